/*
 * oracle.c -- plain FP64 CPU reference for decentralized baseband processing
 * (Li, Sharan, Chen, Goldstein, Cavallaro, Studer, "Decentralized Baseband
 * Processing for Massive MU-MIMO Systems").
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code with the CUDA
 * path and must never be used as a fallback for it.
 *
 * Every routine follows the paper's algorithm steps in the paper's order and
 * notation, one subcarrier / OFDM symbol at a time, in double-precision
 * complex arithmetic.  Matrix inverses are formed explicitly (Gauss-Jordan
 * elimination with partial pivoting), as the algorithms state them.  The only
 * parallelism is an OpenMP loop over independent subcarriers; it does not
 * change the arithmetic of any subcarrier.
 *
 * Layouts (row-major, complex interleaved re/im, i.e. C99 double complex):
 *   H  [W][B][U]   uplink channel; cluster c owns rows c*S .. c*S+S-1, S=B/C
 *   y  [W][N][B]   uplink receive vectors
 *   s  [W][N][U]   downlink transmit vectors / uplink equaliser outputs
 *   x  [W][N][B]   downlink beamforming vectors
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   - gamma is a caller argument (Sec. III-B and IV-B use gamma = 1);
 *   - Alg. 2: the residual update uses e^(t) (standard CG; the printed
 *     e^(t-1) is read as a typo), the consensus sum runs over c = 1..C, the
 *     step size uses the real part of p^H e (the system matrix is Hermitian
 *     positive (semi)definite), and the loop stops early when ||r||^2 or
 *     Re(p^H e) is exactly zero (the iterate is then final);
 *   - Lemma 2 with eps > 0: the scaling uses ||s - w|| with w = sum_c w_c,
 *     the norm that the projection in the proof of Lemma 2 produces.
 *
 * Return codes: 0 ok, -1 bad argument, -2 singular matrix, -3 out of memory.
 */
#include <stdlib.h>
#include <string.h>
#include <tgmath.h>

/* The oracle's arithmetic is double.  The CPU baseline also compiles this
 * same source with ORACLE_REAL=float, as a plain FP32 program that is only
 * timed (the survey's "plain CPU" line); the math functions are the
 * type-generic ones of <tgmath.h>, so both builds run the same steps. */
#ifndef ORACLE_REAL
#define ORACLE_REAL double
#endif
typedef ORACLE_REAL real;
typedef ORACLE_REAL complex cplx;

enum { REG_ZF = 0, REG_MMSE = 1, REG_BOX = 2, REG_BPSK = 3 };
enum { MODE_AUTO = 0, MODE_UXU = 1, MODE_SXS = 2 };
enum { OK = 0, ERR_ARG = -1, ERR_SINGULAR = -2, ERR_NOMEM = -3 };

/* ------------------------------------------------------------------ */
/* Small dense helpers (row-major).                                    */
/* ------------------------------------------------------------------ */

/* Ainv = A^{-1} for an n x n matrix by Gauss-Jordan elimination with
 * partial pivoting on the augmented matrix [A | I].  work holds 2*n*n. */
static int inv_gj(int n, const cplx *A, cplx *Ainv, cplx *work)
{
    const int m = 2 * n;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            work[i * m + j] = A[i * n + j];
            work[i * m + n + j] = (i == j) ? 1.0 : 0.0;
        }
    }
    for (int k = 0; k < n; ++k) {
        int piv = k;
        real best = cabs(work[k * m + k]);
        for (int i = k + 1; i < n; ++i) {
            real a = cabs(work[i * m + k]);
            if (a > best) { best = a; piv = i; }
        }
        if (best == 0.0) return ERR_SINGULAR;
        if (piv != k) {
            for (int j = 0; j < m; ++j) {
                cplx t = work[k * m + j];
                work[k * m + j] = work[piv * m + j];
                work[piv * m + j] = t;
            }
        }
        cplx d = work[k * m + k];
        for (int j = 0; j < m; ++j) work[k * m + j] /= d;
        for (int i = 0; i < n; ++i) {
            if (i == k) continue;
            cplx f = work[i * m + k];
            if (f == 0.0) continue;
            for (int j = 0; j < m; ++j) work[i * m + j] -= f * work[k * m + j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ainv[i * n + j] = work[i * m + n + j];
    return OK;
}

/* out = A x, A is rows x cols. */
static void mv(int rows, int cols, const cplx *A, const cplx *x, cplx *out)
{
    for (int i = 0; i < rows; ++i) {
        cplx acc = 0.0;
        for (int j = 0; j < cols; ++j) acc += A[i * cols + j] * x[j];
        out[i] = acc;
    }
}

/* out = A^H x, A is rows x cols, out has cols entries. */
static void mvh(int rows, int cols, const cplx *A, const cplx *x, cplx *out)
{
    for (int j = 0; j < cols; ++j) {
        cplx acc = 0.0;
        for (int i = 0; i < rows; ++i) acc += conj(A[i * cols + j]) * x[i];
        out[j] = acc;
    }
}

/* G = A^H A + delta I (cols x cols), A is rows x cols. */
static void gram_ha(int rows, int cols, const cplx *A, real delta, cplx *G)
{
    for (int i = 0; i < cols; ++i)
        for (int j = 0; j < cols; ++j) {
            cplx acc = 0.0;
            for (int r = 0; r < rows; ++r) acc += conj(A[r * cols + i]) * A[r * cols + j];
            G[i * cols + j] = acc + ((i == j) ? delta : 0.0);
        }
}

/* G = A A^H + delta I (rows x rows), A is rows x cols. */
static void gram_ah(int rows, int cols, const cplx *A, real delta, cplx *G)
{
    for (int i = 0; i < rows; ++i)
        for (int j = 0; j < rows; ++j) {
            cplx acc = 0.0;
            for (int k = 0; k < cols; ++k) acc += A[i * cols + k] * conj(A[j * cols + k]);
            G[i * rows + j] = acc + ((i == j) ? delta : 0.0);
        }
}

/* At = A^T; A is rows x cols. */
static void transpose(int rows, int cols, const cplx *A, cplx *At)
{
    for (int i = 0; i < rows; ++i)
        for (int j = 0; j < cols; ++j) At[j * rows + i] = A[i * cols + j];
}

static int check_shape(int W, int N, int B, int C, int U)
{
    if (W < 0 || N < 0 || B <= 0 || C <= 0 || U <= 0) return ERR_ARG;
    if (B % C != 0) return ERR_ARG;
    return OK;
}

static void *xmalloc(size_t n) { return malloc(n ? n : 1); }

/* ------------------------------------------------------------------ */
/* Step (E2) via Lemma 1: s = argmin_s g(s) + C rho/2 ||s - v||^2,      */
/* v = w / C.  Closed forms (E2-ZF), (E2-MMSE), (E2-BOX) and BPSK.      */
/* ------------------------------------------------------------------ */
static real clip(real a, real r)
{
    real m = fabs(a) < r ? fabs(a) : r;
    return a < 0.0 ? -m : m;
}

static void prox_e2(int reg, int U, int C, real rho, real N0, real Es,
                    real box_r, const cplx *w, cplx *s)
{
    for (int u = 0; u < U; ++u) {
        cplx v = w[u] / (real)C;
        switch (reg) {
        case REG_ZF:   /* (E2-ZF): s = v */
            s[u] = v;
            break;
        case REG_MMSE: /* Alg. 1 scaling (N0/(rho Es) + C)^{-1} w, i.e. (E2-MMSE) */
            s[u] = w[u] / (N0 / (rho * Es) + (real)C);
            break;
        case REG_BOX:  /* (E2-BOX): per-axis projection onto [-r, r] */
            s[u] = clip(creal(v), box_r) + I * clip(cimag(v), box_r);
            break;
        default:       /* BPSK: projection onto the real segment [-r, r] */
            s[u] = clip(creal(v), box_r);
            break;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Alg. 1: decentralized ADMM-based data detection.                    */
/* mode: 0 = the algorithm's own branch (S x S when S <= U),          */
/*       1 = force the U x U form (E1 closed form with B_c),           */
/*       2 = force the S x S (Woodbury) form with A_c.                 */
/* ------------------------------------------------------------------ */
int oracle_admm_ul(int W, int N, int B, int C, int U,
                   const cplx *H, const cplx *y,
                   real rho, real gamma, real N0, real Es,
                   int T_max, int reg, real box_r, int mode, cplx *s_out)
{
    if (check_shape(W, N, B, C, U) != OK || T_max < 1 || !(rho > 0.0)) return ERR_ARG;
    if (reg < REG_ZF || reg > REG_BPSK) return ERR_ARG;
    if (reg == REG_MMSE && !(Es > 0.0)) return ERR_ARG;
    const int S = B / C;
    const int use_ss = (mode == MODE_AUTO) ? (S <= U) : (mode == MODE_SXS);
    const int D = use_ss ? S : U;
    int status = OK;

#pragma omp parallel for schedule(dynamic)
    for (int w = 0; w < W; ++w) {
        cplx *inv  = xmalloc(sizeof(cplx) * (size_t)C * D * D);
        cplx *mat  = xmalloc(sizeof(cplx) * (size_t)D * D);
        cplx *work = xmalloc(sizeof(cplx) * (size_t)2 * D * D);
        cplx *yreg = xmalloc(sizeof(cplx) * (size_t)C * U);
        cplx *z    = xmalloc(sizeof(cplx) * (size_t)C * U);
        cplx *lam  = xmalloc(sizeof(cplx) * (size_t)C * U);
        cplx *sv   = xmalloc(sizeof(cplx) * (size_t)U);
        cplx *wv   = xmalloc(sizeof(cplx) * (size_t)U);
        cplx *d    = xmalloc(sizeof(cplx) * (size_t)U);
        cplx *tU   = xmalloc(sizeof(cplx) * (size_t)U);
        cplx *tS1  = xmalloc(sizeof(cplx) * (size_t)S);
        cplx *tS2  = xmalloc(sizeof(cplx) * (size_t)S);
        const cplx *Hw = H + (size_t)w * B * U;
        int bad = !inv || !mat || !work || !yreg || !z || !lam || !sv || !wv ||
                  !d || !tU || !tS1 || !tS2;
        if (bad) {
#pragma omp atomic write
            status = ERR_NOMEM;
        }

        /* Preprocessing (per subcarrier; the channel is static over its N
         * symbols): A_c^{-1} = (H_c H_c^H + rho I_S)^{-1} or
         *           B_c^{-1} = (H_c^H H_c + rho I_U)^{-1}. */
        for (int c = 0; c < C && !bad; ++c) {
            const cplx *Hc = Hw + (size_t)c * S * U;
            if (use_ss)
                gram_ah(S, U, Hc, rho, mat);
            else
                gram_ha(S, U, Hc, rho, mat);
            if (inv_gj(D, mat, inv + (size_t)c * D * D, work) != OK) {
                bad = 1;
#pragma omp atomic write
                status = ERR_SINGULAR;
            }
        }

        for (int n = 0; n < N && !bad; ++n) {
            const cplx *yw = y + ((size_t)w * N + n) * B;
            for (int c = 0; c < C; ++c) {
                const cplx *Hc = Hw + (size_t)c * S * U;
                const cplx *yc = yw + (size_t)c * S;
                const cplx *Ic = inv + (size_t)c * D * D;
                if (use_ss) {
                    mv(S, S, Ic, yc, tS1);              /* A_c^{-1} y_c           */
                    mvh(S, U, Hc, tS1, yreg + c * U);   /* y_reg = H_c^H A^{-1} y */
                } else {
                    mvh(S, U, Hc, yc, tU);              /* H_c^H y_c              */
                    mv(U, U, Ic, tU, yreg + c * U);     /* y_reg = B^{-1} H^H y   */
                }
            }
            /* Init: lambda_c = 0, z_c = y_c^reg, s = prox(sum_c z_c). */
            for (int u = 0; u < U; ++u) wv[u] = 0.0;
            for (int c = 0; c < C; ++c)
                for (int u = 0; u < U; ++u) {
                    lam[c * U + u] = 0.0;
                    z[c * U + u] = yreg[c * U + u];
                    wv[u] += z[c * U + u];
                }
            prox_e2(reg, U, C, rho, N0, Es, box_r, wv, sv);

            for (int t = 2; t <= T_max; ++t) {
                for (int u = 0; u < U; ++u) wv[u] = 0.0;
                for (int c = 0; c < C; ++c) {
                    const cplx *Hc = Hw + (size_t)c * S * U;
                    const cplx *Ic = inv + (size_t)c * D * D;
                    cplx *lc = lam + c * U, *zc = z + c * U;
                    /* lambda_c^(t) = lambda_c^(t-1) + gamma (z_c^(t-1) - s^(t-1)) */
                    for (int u = 0; u < U; ++u) lc[u] += gamma * (zc[u] - sv[u]);
                    for (int u = 0; u < U; ++u) d[u] = sv[u] - lc[u];
                    if (use_ss) {
                        /* z_c = y_reg + d - H_c^H A_c^{-1} H_c d */
                        mv(S, U, Hc, d, tS1);
                        mv(S, S, Ic, tS1, tS2);
                        mvh(S, U, Hc, tS2, tU);
                        for (int u = 0; u < U; ++u) zc[u] = yreg[c * U + u] + d[u] - tU[u];
                    } else {
                        /* z_c = y_reg + rho B_c^{-1} d */
                        mv(U, U, Ic, d, tU);
                        for (int u = 0; u < U; ++u) zc[u] = yreg[c * U + u] + rho * tU[u];
                    }
                    /* w_c = z_c + lambda_c; consensus w = sum_c w_c */
                    for (int u = 0; u < U; ++u) wv[u] += zc[u] + lc[u];
                }
                prox_e2(reg, U, C, rho, N0, Es, box_r, wv, sv);
            }
            cplx *so = s_out + ((size_t)w * N + n) * U;
            for (int u = 0; u < U; ++u) so[u] = sv[u];
        }
        free(inv); free(mat); free(work); free(yreg); free(z); free(lam);
        free(sv); free(wv); free(d); free(tU); free(tS1); free(tS2);
    }
    return status;
}

/* ------------------------------------------------------------------ */
/* Alg. 2: decentralized conjugate-gradient data detection.            */
/* rho is the CG regulariser: N0/Es for MMSE, 0 for ZF (Sec. III-D).   */
/* ------------------------------------------------------------------ */
int oracle_cg_ul(int W, int N, int B, int C, int U,
                 const cplx *H, const cplx *y, real rho, int T_max,
                 cplx *x_out)
{
    if (check_shape(W, N, B, C, U) != OK || T_max < 0 || rho < 0.0) return ERR_ARG;
    const int S = B / C;
    int status = OK;

#pragma omp parallel for schedule(dynamic)
    for (int w = 0; w < W; ++w) {
        cplx *r  = xmalloc(sizeof(cplx) * (size_t)U);
        cplx *p  = xmalloc(sizeof(cplx) * (size_t)U);
        cplx *x  = xmalloc(sizeof(cplx) * (size_t)U);
        cplx *e  = xmalloc(sizeof(cplx) * (size_t)U);
        cplx *wv = xmalloc(sizeof(cplx) * (size_t)U);
        cplx *tU = xmalloc(sizeof(cplx) * (size_t)U);
        cplx *tS = xmalloc(sizeof(cplx) * (size_t)S);
        int bad = !r || !p || !x || !e || !wv || !tU || !tS;
        if (bad) {
#pragma omp atomic write
            status = ERR_NOMEM;
        }
        const cplx *Hw = H + (size_t)w * B * U;
        for (int n = 0; n < N && !bad; ++n) {
            const cplx *yw = y + ((size_t)w * N + n) * B;
            /* Preprocessing: y_c^MRC = H_c^H y_c (decentralized),
             * y^MRC = sum_c y_c^MRC (centralized). */
            for (int u = 0; u < U; ++u) r[u] = 0.0;
            for (int c = 0; c < C; ++c) {
                mvh(S, U, Hw + (size_t)c * S * U, yw + (size_t)c * S, tU);
                for (int u = 0; u < U; ++u) r[u] += tU[u];
            }
            /* Init: r = y^MRC, p = r, x = 0. */
            for (int u = 0; u < U; ++u) { p[u] = r[u]; x[u] = 0.0; }
            for (int t = 1; t <= T_max; ++t) {
                /* w_c = H_c^H H_c p (two mat-vecs); w = sum_c w_c */
                for (int u = 0; u < U; ++u) wv[u] = 0.0;
                for (int c = 0; c < C; ++c) {
                    const cplx *Hc = Hw + (size_t)c * S * U;
                    mv(S, U, Hc, p, tS);
                    mvh(S, U, Hc, tS, tU);
                    for (int u = 0; u < U; ++u) wv[u] += tU[u];
                }
                /* e = rho p + w */
                for (int u = 0; u < U; ++u) e[u] = rho * p[u] + wv[u];
                real rr = 0.0, pe = 0.0;
                for (int u = 0; u < U; ++u) {
                    rr += creal(r[u]) * creal(r[u]) + cimag(r[u]) * cimag(r[u]);
                    pe += creal(conj(p[u]) * e[u]);
                }
                if (rr == 0.0 || pe == 0.0) break;
                real alpha = rr / pe;
                for (int u = 0; u < U; ++u) x[u] += alpha * p[u];
                real rr_new = 0.0;
                for (int u = 0; u < U; ++u) {
                    r[u] -= alpha * e[u];
                    rr_new += creal(r[u]) * creal(r[u]) + cimag(r[u]) * cimag(r[u]);
                }
                real beta = rr_new / rr;
                for (int u = 0; u < U; ++u) p[u] = r[u] + beta * p[u];
            }
            cplx *xo = x_out + ((size_t)w * N + n) * U;
            for (int u = 0; u < U; ++u) xo[u] = x[u];
        }
        free(r); free(p); free(x); free(e); free(wv); free(tU); free(tS);
    }
    return status;
}

/* ------------------------------------------------------------------ */
/* Alg. 3: decentralized ADMM-based beamforming, with the (P2) step of  */
/* Lemma 2 (eps >= 0; Alg. 3 as printed is eps = 0).                    */
/* H is given in uplink layout; cluster c uses H^d_c = (H^u_c)^T.       */
/* mode: 0 = the algorithm's branch (S x S when S <= U), 1 = U x U,     */
/*       2 = S x S.                                                     */
/* ------------------------------------------------------------------ */
int oracle_admm_dl(int W, int N, int B, int C, int U,
                   const cplx *H, const cplx *s, real rho, real gamma,
                   real eps, int T_max, int mode, cplx *x_out)
{
    if (check_shape(W, N, B, C, U) != OK || T_max < 1 || !(rho > 0.0) || eps < 0.0)
        return ERR_ARG;
    const int S = B / C;
    const int use_ss = (mode == MODE_AUTO) ? (S <= U) : (mode == MODE_SXS);
    const int D = use_ss ? S : U;
    int status = OK;

#pragma omp parallel for schedule(dynamic)
    for (int w = 0; w < W; ++w) {
        cplx *Hd   = xmalloc(sizeof(cplx) * (size_t)C * U * S);
        cplx *inv  = xmalloc(sizeof(cplx) * (size_t)C * D * D);
        cplx *mat  = xmalloc(sizeof(cplx) * (size_t)D * D);
        cplx *work = xmalloc(sizeof(cplx) * (size_t)2 * D * D);
        cplx *xc   = xmalloc(sizeof(cplx) * (size_t)C * S);
        cplx *z    = xmalloc(sizeof(cplx) * (size_t)C * U);
        cplx *lam  = xmalloc(sizeof(cplx) * (size_t)C * U);
        cplx *m    = xmalloc(sizeof(cplx) * (size_t)C * U);
        cplx *wc   = xmalloc(sizeof(cplx) * (size_t)C * U);
        cplx *wv   = xmalloc(sizeof(cplx) * (size_t)U);
        cplx *v    = xmalloc(sizeof(cplx) * (size_t)U);
        cplx *tU   = xmalloc(sizeof(cplx) * (size_t)U);
        cplx *tS   = xmalloc(sizeof(cplx) * (size_t)S);
        int bad = !Hd || !inv || !mat || !work || !xc || !z || !lam || !m ||
                  !wc || !wv || !v || !tU || !tS;
        if (bad) {
#pragma omp atomic write
            status = ERR_NOMEM;
        }
        const cplx *Hw = H + (size_t)w * B * U;

        /* Preprocessing: H^d_c = (H^u_c)^T (reciprocity, Sec. II-B);
         * A_c^{-1} = (H_c^H H_c + rho^{-1} I_S)^{-1} or
         * B_c^{-1} = (H_c H_c^H + rho^{-1} I_U)^{-1}, H_c the U x S block. */
        for (int c = 0; c < C && !bad; ++c) {
            cplx *Hdc = Hd + (size_t)c * U * S;
            transpose(S, U, Hw + (size_t)c * S * U, Hdc);
            if (use_ss)
                gram_ha(U, S, Hdc, 1.0 / rho, mat);
            else
                gram_ah(U, S, Hdc, 1.0 / rho, mat);
            if (inv_gj(D, mat, inv + (size_t)c * D * D, work) != OK) {
                bad = 1;
#pragma omp atomic write
                status = ERR_SINGULAR;
            }
        }

        /* (P1): x_c = A_c^{-1} H_c^H v  or  H_c^H B_c^{-1} v, v = z_c + lambda_c */
#define DL_P1(c_, vin_, xout_)                                                  \
        do {                                                                    \
            const cplx *Hdc_ = Hd + (size_t)(c_) * U * S;                       \
            const cplx *Ic_ = inv + (size_t)(c_) * D * D;                       \
            if (use_ss) {                                                       \
                mvh(U, S, Hdc_, (vin_), tS);                                    \
                mv(S, S, Ic_, tS, (xout_));                                     \
            } else {                                                            \
                mv(U, U, Ic_, (vin_), tU);                                      \
                mvh(U, S, Hdc_, tU, (xout_));                                   \
            }                                                                   \
        } while (0)

        const real init_scale = fmax((real)U / (real)B, 1.0 / (real)C);
        for (int n = 0; n < N && !bad; ++n) {
            const cplx *sw = s + ((size_t)w * N + n) * U;
            /* Init: z_c = max{U/B, 1/C} s, lambda_c = 0, x_c = P1(z_c). */
            for (int c = 0; c < C; ++c) {
                for (int u = 0; u < U; ++u) {
                    z[c * U + u] = init_scale * sw[u];
                    lam[c * U + u] = 0.0;
                    v[u] = z[c * U + u] + lam[c * U + u];
                }
                DL_P1(c, v, xc + (size_t)c * S);
            }
            for (int t = 2; t <= T_max; ++t) {
                for (int u = 0; u < U; ++u) wv[u] = 0.0;
                for (int c = 0; c < C; ++c) {
                    /* m_c = H_c x_c ; w_c = m_c - lambda_c */
                    mv(U, S, Hd + (size_t)c * U * S, xc + (size_t)c * S, m + c * U);
                    for (int u = 0; u < U; ++u) {
                        wc[c * U + u] = m[c * U + u] - lam[c * U + u];
                        wv[u] += wc[c * U + u];        /* consensus w = sum_c w_c */
                    }
                }
                /* (P2) via Lemma 2: z_c = w_c + k (s/C - w/C),
                 * k = max{0, 1 - eps/||s - w||} (k = 1 for eps = 0). */
                real k = 1.0;
                if (eps > 0.0) {
                    real nrm = 0.0;
                    for (int u = 0; u < U; ++u) {
                        cplx dlt = sw[u] - wv[u];
                        nrm += creal(dlt) * creal(dlt) + cimag(dlt) * cimag(dlt);
                    }
                    nrm = sqrt(nrm);
                    k = (nrm > 0.0) ? fmax(0.0, 1.0 - eps / nrm) : 0.0;
                }
                for (int c = 0; c < C; ++c) {
                    for (int u = 0; u < U; ++u) {
                        z[c * U + u] = wc[c * U + u] + k * (sw[u] - wv[u]) / (real)C;
                        /* (P3): lambda_c = lambda_c - gamma (m_c - z_c) */
                        lam[c * U + u] -= gamma * (m[c * U + u] - z[c * U + u]);
                        v[u] = z[c * U + u] + lam[c * U + u];
                    }
                    DL_P1(c, v, xc + (size_t)c * S);
                }
            }
            cplx *xo = x_out + ((size_t)w * N + n) * B;
            for (int i = 0; i < B; ++i) xo[i] = xc[i];
        }
#undef DL_P1
        free(Hd); free(inv); free(mat); free(work); free(xc); free(z); free(lam);
        free(m); free(wc); free(wv); free(v); free(tU); free(tS);
    }
    return status;
}

/* ------------------------------------------------------------------ */
/* Centralized references (Sec. III-A, Sec. IV-A).                     */
/* ------------------------------------------------------------------ */

/* x = (H^H H + delta I)^{-1} H^H y; delta = N0/Es (MMSE) or 0 (ZF). */
int oracle_lmmse_ul(int W, int N, int B, int U, const cplx *H, const cplx *y,
                    real delta, cplx *x_out)
{
    if (W < 0 || N < 0 || B <= 0 || U <= 0 || delta < 0.0) return ERR_ARG;
    int status = OK;
#pragma omp parallel for schedule(dynamic)
    for (int w = 0; w < W; ++w) {
        cplx *G = xmalloc(sizeof(cplx) * (size_t)U * U);
        cplx *Gi = xmalloc(sizeof(cplx) * (size_t)U * U);
        cplx *work = xmalloc(sizeof(cplx) * (size_t)2 * U * U);
        cplx *t = xmalloc(sizeof(cplx) * (size_t)U);
        int bad = !G || !Gi || !work || !t;
        const cplx *Hw = H + (size_t)w * B * U;
        if (!bad) {
            gram_ha(B, U, Hw, delta, G);
            if (inv_gj(U, G, Gi, work) != OK) bad = 1;
        }
        if (bad) {
#pragma omp atomic write
            status = ERR_SINGULAR;
        }
        for (int n = 0; n < N && !bad; ++n) {
            mvh(B, U, Hw, y + ((size_t)w * N + n) * B, t);
            mv(U, U, Gi, t, x_out + ((size_t)w * N + n) * U);
        }
        free(G); free(Gi); free(work); free(t);
    }
    return status;
}

/* ZF beamformer x = H^H (H H^H)^{-1} s with the downlink H = (H^u)^T. */
int oracle_zf_dl(int W, int N, int B, int U, const cplx *H, const cplx *s,
                 cplx *x_out)
{
    if (W < 0 || N < 0 || B <= 0 || U <= 0 || U > B) return ERR_ARG;
    int status = OK;
#pragma omp parallel for schedule(dynamic)
    for (int w = 0; w < W; ++w) {
        cplx *Hd = xmalloc(sizeof(cplx) * (size_t)U * B);
        cplx *G = xmalloc(sizeof(cplx) * (size_t)U * U);
        cplx *Gi = xmalloc(sizeof(cplx) * (size_t)U * U);
        cplx *work = xmalloc(sizeof(cplx) * (size_t)2 * U * U);
        cplx *t = xmalloc(sizeof(cplx) * (size_t)U);
        int bad = !Hd || !G || !Gi || !work || !t;
        if (!bad) {
            transpose(B, U, H + (size_t)w * B * U, Hd);
            gram_ah(U, B, Hd, 0.0, G);
            if (inv_gj(U, G, Gi, work) != OK) bad = 1;
        }
        if (bad) {
#pragma omp atomic write
            status = ERR_SINGULAR;
        }
        for (int n = 0; n < N && !bad; ++n) {
            mv(U, U, Gi, s + ((size_t)w * N + n) * U, t);
            mvh(U, B, Hd, t, x_out + ((size_t)w * N + n) * B);
        }
        free(Hd); free(G); free(Gi); free(work); free(t);
    }
    return status;
}
