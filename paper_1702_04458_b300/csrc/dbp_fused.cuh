// dbp_fused.cuh -- fused per-subcarrier kernels for decentralized baseband
// processing on sm_103a.
//
// Mapping.  One warp owns one (subcarrier w, antenna cluster c) pair: it is
// the "processing element" of cluster c (Sec. II-A.2) and only ever reads its
// own block H_c (rows c*S .. c*S+S-1 of H[w]) and its own receive data y_c.
// The C warps of a subcarrier sit in one CTA; the fusion node of the paper
// (consensus sum w = sum_c w_c, Lemma 1 / Lemma 2) becomes a shared-memory
// exchange of U-vectors between those warps, after which every warp applies
// the consensus step itself (early broadcast of w, Sec. III-C).  A CTA holds P
// subcarriers (P*C warps) when C is small.  When the C warps of one
// subcarrier need more registers than one CTA can have, the subcarrier is
// spread over the CL CTAs of a thread-block cluster (CPB = C/CL clusters per
// CTA) and the consensus reads the other CTAs' vectors through distributed
// shared memory (DSMEM) after a cluster barrier.
//
// Lane layout inside a warp: UT (a power of two >= U) lanes per symbol group,
// G = 32/UT groups; lane (u, g) owns user row u and the symbols
// n = n0 + g + G*j, j < NN, of the current symbol chunk (NCH = G*NN symbols).
// Per-cluster operators (Gram, inverse) live in registers, one matrix row per
// lane; vectors are exchanged through a small per-warp shared-memory buffer.
//
// Everything a subcarrier needs (Gram + regularisation, explicit inverse,
// matched filter, all iterations, consensus, slicer) runs in one launch; no
// intermediate result leaves the chip.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dbp {

enum Alg { ALG_ADMM_UL = 0, ALG_CG_UL = 1, ALG_ADMM_DL = 2 };

struct FusedParams;
template <typename T> struct ParamSel;
template <> struct ParamSel<float> {
    static __device__ __forceinline__ float get(double, float f) { return f; }
};
template <> struct ParamSel<double> {
    static __device__ __forceinline__ double get(double d, float) { return d; }
};

struct FusedParams {
    const void *H;       // [W][B][U] complex
    const void *vin;     // uplink: y [W][N][B]; downlink: s [W][N][U]
    void *out;           // uplink: x_hat [W][N][U]; downlink: x [W][N][B]
    uint8_t *labels;     // [W][N][U] or nullptr
    double *energy;      // downlink: accumulates sum |x|^2, or nullptr
    int W, N, B, C, U, S, T;
    int P;               // subcarriers per CTA (CTA mapping)
    int CPB;             // antenna clusters per CTA (cluster mapping)
    int CL;              // CTAs per thread-block cluster (cluster mapping)
    int reg;             // 0 ZF, 1 MMSE, 2 BOX (uplink ADMM prox)
    double delta;        // diagonal loading of the Gram: rho (UL ADMM),
                         // 0 (CG), 1/rho (DL)
    double rho;          // ADMM penalty
    double gamma;        // dual step
    double e2_scale;     // (E2): 1/C (ZF) or 1/(N0/(rho Es) + C) (MMSE)
    double invC;         // 1/C
    double box_r;        // (E2-BOX) radius
    double eps;          // downlink residual bound (Lemma 2); 0 = Alg. 3 as printed
    double rho_cg;       // CG regulariser N0/Es or 0
    double kappa;        // DL init max{U/B, 1/C}
    double inv_rho;      // 1/rho
    int qam_M, qam_L, qam_half;
    double qam_inv_a;    // 1 / sqrt(3 / (2 (M - 1)))
    // The same scalars rounded to FP32 on the host, so FP32 kernels read
    // them from the parameter bank without a double conversion.
    float f_delta, f_rho, f_gamma, f_e2_scale, f_invC, f_box_r, f_rho_cg, f_kappa, f_inv_rho, f_qam_inv_a, f_eps;
    // Persistent bulk-copy kernel only:
    int *status;         // device word: bit 0 = a bounded wait gave up
    unsigned int *retries;   // device counter of FP64 inverse retries
    int tiles;           // subcarrier tiles (ceil(W / P))
    int single_buf;      // 1: one staging buffer (uplink), the next subcarrier
                         // is fetched after the matched filter has read it
    int hp;              // staged H row pitch, in input elements
    int yp;              // staged receive-row pitch, in input elements
    int h_rows;          // staged H rows (S, or S rounded up to 8)
    int y_rows;          // staged receive rows per buffer (N rounded up)
    int ms_rows;         // rows of the matched-filter result buffer
    // per-warp shared-memory layout, byte offsets from the warp's base
    int off_h1, off_y0, off_y1, off_g, off_v, warp_bytes;
    // Resident per-cluster operator of a coherence block (bulk-copy kernel):
    // 0 = compute, 1 = compute and store, 2 = load instead of computing.
    // Layout [W][C][UT][UT] float2: B_c^{-1} (uplink and downlink ADMM) or
    // G_c (CG).
    float2 *factor;
    int factor_mode;
    // Test hook of the bounded waits (0 = off): bytes added to every input
    // copy's expected transaction count (so that its barrier never
    // completes) and the wait limit in polling iterations.
    int starve_bytes;
    int wait_iters;
};

// ---------------------------------------------------------------------------
// Complex helpers (float2 / double2).
// ---------------------------------------------------------------------------
template <typename T> struct C2Of;
template <> struct C2Of<float>  { typedef float2 type; };
template <> struct C2Of<double> { typedef double2 type; };

__device__ __forceinline__ float2 cz(float2) { return make_float2(0.f, 0.f); }
__device__ __forceinline__ double2 cz(double2) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }

// acc += a * b
template <typename C2> __device__ __forceinline__ void cmac(C2 &acc, C2 a, C2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename C2> __device__ __forceinline__ void cmacc(C2 &acc, C2 a, C2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
template <typename C2> __device__ __forceinline__ C2 cmul(C2 a, C2 b) {
    C2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C2> __device__ __forceinline__ C2 cadd(C2 a, C2 b) { a.x += b.x; a.y += b.y; return a; }
template <typename C2> __device__ __forceinline__ C2 csub(C2 a, C2 b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C2, typename T> __device__ __forceinline__ C2 cscale(C2 a, T s) { a.x *= s; a.y *= s; return a; }
template <typename C2> __device__ __forceinline__ C2 crcp(C2 a) {
    auto d = a.x * a.x + a.y * a.y;
    auto inv = decltype(d)(1) / d;
    C2 r; r.x = a.x * inv; r.y = -a.y * inv;
    return r;
}
// 1 / x by the hardware approximation (rcp.approx.ftz.f32: within one ulp,
// subnormal arguments and results flushed to zero).  The FP32 eliminations
// take their pivots' reciprocals with it: it sits on each step's dependent
// chain, where the correctly rounded reciprocal adds a refinement sequence.
// Exponent e of m = f 2^e with f in [0.5, 1) (the frexp exponent) for a
// positive finite m, from its IEEE-754 fields: biased exponent - 126 for a
// normal m; for a subnormal m = k 2^-149, the position of k's leading bit.
__device__ __forceinline__ int frexp_exponent(float m) {
    const int b = __float_as_int(m);
    return (b >> 23) ? (b >> 23) - 126 : -117 - __clz(b);
}
// Largest value over the full warp in one instruction (redux.sync.max.f32;
// max is exact, so any order of reduction gives the same result).
__device__ __forceinline__ float warp_redux_max(float v) {
    float r;
    asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Two consecutive complex values from shared memory (16-byte aligned for
// float: one 128-bit load).
__device__ __forceinline__ void ld2(const float2 *p, float2 &a, float2 &b) {
    float4 v = *reinterpret_cast<const float4 *>(p);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld2(const double2 *p, double2 &a, double2 &b) {
    a = p[0];
    b = p[1];
}

template <typename T> __device__ __forceinline__ T shfl_x(T v, int m) {
    return __shfl_xor_sync(0xffffffffu, v, m);
}

// Sum over the UT lanes of one symbol group (butterfly; every lane of the
// group ends with the bit-identical sum).
template <int UT, typename T> __device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int m = 1; m < UT; m <<= 1) v += shfl_x(v, m);
    return v;
}

// ---------------------------------------------------------------------------
// Slicer (Sec. III-A): nearest point of the square QAM alphabet per axis,
// Gray label out.  t = (x * inv_a + (L-1)) / 2, k = ceil(t - 1/2) clamped to
// [0, L-1] (an exact boundary goes to the lower level).  Every operation is
// rounded separately (no contraction) so the decision is reproducible.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pam_index(float x, float inv_a, float off, int L) {
    float t = __fmul_rn(__fadd_rn(__fmul_rn(x, inv_a), off), 0.5f);
    float k = ceilf(__fadd_rn(t, -0.5f));
    k = fminf(fmaxf(k, 0.f), (float)(L - 1));
    return (int)k;
}
__device__ __forceinline__ int pam_index(double x, double inv_a, double off, int L) {
    double t = __dmul_rn(__dadd_rn(__dmul_rn(x, inv_a), off), 0.5);
    double k = ceil(__dadd_rn(t, -0.5));
    k = fmin(fmax(k, 0.0), (double)(L - 1));
    return (int)k;
}
template <typename T>
__device__ __forceinline__ uint8_t qam_label(T xr, T xi, T inv_a, int L, int half) {
    int kI = pam_index(xr, inv_a, (T)(L - 1), L);
    int kQ = pam_index(xi, inv_a, (T)(L - 1), L);
    int gI = kI ^ (kI >> 1), gQ = kQ ^ (kQ >> 1);
    return (uint8_t)((gI << half) | gQ);
}

template <typename T> __device__ __forceinline__ T clip_r(T a, T r) {
    T m = fabs(a) < r ? fabs(a) : r;
    return a < (T)0 ? -m : m;
}

// ---------------------------------------------------------------------------
// Compile-time tiling per padded user count UT.
// ---------------------------------------------------------------------------
template <int UT> struct Tile {
    static constexpr int G = 32 / UT;                       // symbol groups
    static constexpr int NN = (UT == 4) ? 2 : (UT == 8) ? 4 : 7;
    static constexpr int NCH = G * NN;                      // symbols per chunk
    static constexpr int SCH = (UT == 32) ? 16 : 32;        // H rows per stage
    static constexpr int HS_LD = UT + 2;                    // padded strides
    static constexpr int YS_LD = SCH + 2;                   //  (complex units,
    static constexpr int V_LD = UT + 2;                     //   16 B aligned)
    static constexpr int WARP_ELEMS = SCH * HS_LD + NCH * YS_LD + NCH * V_LD;
    static constexpr int CONS_ELEMS = NCH * UT;             // per warp, per buffer
};

template <int UT> __host__ __device__ constexpr int fused_smem_elems(int nwarps, int subcarriers) {
    // per warp: staging and contribution buffers; per subcarrier of the CTA:
    // the reduced consensus sums, two buffers of CONS_ELEMS
    return nwarps * (Tile<UT>::WARP_ELEMS + 2 * Tile<UT>::CONS_ELEMS) + subcarriers * 2 * Tile<UT>::CONS_ELEMS;
}

// Stage rows s0 .. s0+rows-1 of the cluster block H_c into Hs[SCH][HS_LD],
// zero-filling padded rows and users.
template <int UT, typename C2>
__device__ __forceinline__ void stage_h(C2 *Hs, const C2 *Hc, int s0, int rows, int U,
                                        bool valid, int lane) {
    using K = Tile<UT>;
#pragma unroll 4
    for (int i = lane; i < K::SCH * UT; i += 32) {
        const int r = i / UT, uu = i % UT;
        C2 v = cz(C2());
        if (valid && r < rows && uu < U) v = Hc[(size_t)(s0 + r) * U + uu];
        Hs[r * K::HS_LD + uu] = v;
    }
}

// Stage y[w][n0+nl][c*S + s0 + sl] into Ys[nl][sl] (zero padded).
template <int UT, typename C2>
__device__ __forceinline__ void stage_y(C2 *Ys, const C2 *yw, int n0, int N, int B, int col0,
                                        int rows, bool valid, int lane) {
    using K = Tile<UT>;
#pragma unroll 4
    for (int i = lane; i < K::NCH * K::SCH; i += 32) {
        const int nl = i / K::SCH, sl = i % K::SCH;
        C2 v = cz(C2());
        if (valid && sl < rows && n0 + nl < N) v = yw[(size_t)(n0 + nl) * B + col0 + sl];
        Ys[nl * K::YS_LD + sl] = v;
    }
}

// out[j] = sum_k R[k] * V[n_j][k]  (row u of the operator times the lane's
// symbol vectors, read from the warp's exchange buffer).
template <int UT, typename C2>
__device__ __forceinline__ void matvec(const C2 (&R)[UT], const C2 *Vb, int g, C2 (&out)[Tile<UT>::NN]) {
    using K = Tile<UT>;
#pragma unroll
    for (int j = 0; j < K::NN; ++j) {
        const int nl = g + K::G * j;
        C2 acc = cz(C2());
#pragma unroll
        for (int k = 0; k < UT; k += 2) {
            C2 a, b;
            ld2(&Vb[nl * K::V_LD + k], a, b);
            cmac(acc, R[k], a);
            cmac(acc, R[k + 1], b);
        }
        out[j] = acc;
    }
}

template <int UT, typename C2>
__device__ __forceinline__ void put_vec(C2 *Vb, int u, int g, const C2 (&v)[Tile<UT>::NN]) {
    using K = Tile<UT>;
#pragma unroll
    for (int j = 0; j < K::NN; ++j) Vb[(g + K::G * j) * K::V_LD + u] = v[j];
}

// In-register Gauss-Jordan inversion of the Hermitian positive definite
// matrix whose row u is held by lane (u, g) (all groups hold copies).  No
// pivoting is needed: every pivot is a Schur complement of an HPD matrix.
template <int UT, typename C2>
__device__ __forceinline__ void gj_invert(C2 (&R)[UT], C2 *scratch, int u, int lane) {
#pragma unroll
    for (int k = 0; k < UT; ++k) {
        if (lane == k) {
#pragma unroll
            for (int j = 0; j < UT; ++j) scratch[j] = R[j];
        }
        __syncwarp();
        const C2 inv = crcp(scratch[k]);
        const bool me = (u == k);
        const C2 f = me ? mkc(-inv.x, -inv.y) : cmul(R[k], inv);
#pragma unroll
        for (int j = 0; j < UT; j += 2) {
            C2 a, b;
            ld2(&scratch[j], a, b);
            if (j != k) {
                C2 base = me ? cz(C2()) : R[j];
                cmac(base, mkc(-f.x, -f.y), a);
                R[j] = base;
            }
            if (j + 1 != k) {
                C2 base = me ? cz(C2()) : R[j + 1];
                cmac(base, mkc(-f.x, -f.y), b);
                R[j + 1] = base;
            }
        }
        R[k] = me ? inv : mkc(-f.x, -f.y);
        __syncwarp();
    }
}

// Threads per CTA the register budget allows (65536 registers per SM; one
// operator row of UT complex values plus the symbol state per lane).
template <typename T, int UT> struct Bounds {
    static constexpr int threads = (sizeof(T) == 4)
        ? ((UT <= 4) ? 1024 : (UT <= 16) ? 512 : 256)
        : ((UT <= 4) ? 512 : 256);
    static constexpr int max_warps = threads / 32;
};

// ---------------------------------------------------------------------------
// The fused kernel.  CLU = false: one CTA holds P whole subcarriers.
// CLU = true: one thread-block cluster of CL CTAs holds one subcarrier.
// ---------------------------------------------------------------------------
template <typename T, int UT, int ALG, bool CLU>
__global__ void __launch_bounds__(Bounds<T, UT>::threads) dbp_fused_kernel(const FusedParams p) {
    using C2 = typename C2Of<T>::type;
    using K = Tile<UT>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *smem = reinterpret_cast<C2 *>(smem_raw);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    int pl, c, w;
    if (CLU) {
        const int rank = blockIdx.x % p.CL;  // CTA rank in the cluster
        pl = 0;
        c = rank * p.CPB + warp;             // antenna cluster of this warp
        w = blockIdx.x / p.CL;               // subcarrier
    } else {
        pl = warp / p.C;                     // subcarrier slot in the CTA
        c = warp - pl * p.C;                 // antenna cluster of this warp
        w = blockIdx.x * p.P + pl;           // subcarrier
    }
    const bool valid = (w < p.W);
    const int u = lane % UT, g = lane / UT;

    C2 *Hs = smem + warp * K::WARP_ELEMS;
    C2 *Ys = Hs + K::SCH * K::HS_LD;
    C2 *Vb = Ys + K::NCH * K::YS_LD;
    C2 *cons = smem + nwarps * K::WARP_ELEMS;          // [2][nwarps][NCH][UT]
    C2 *cons_grp = cons + (size_t)(pl * p.C) * K::CONS_ELEMS;
    // reduced consensus sums [2][subcarriers of the CTA][NCH][UT]
    C2 *wsum = cons + (size_t)2 * nwarps * K::CONS_ELEMS;
    const int nsub = CLU ? 1 : p.P;

    const int S = p.S, U = p.U, N = p.N, B = p.B;
    const C2 *Hc = reinterpret_cast<const C2 *>(p.H) + ((size_t)(valid ? w : 0) * B + (size_t)c * S) * U;

    // ---- Per-cluster operator: Gram (+ diagonal loading), row u per lane ----
    C2 R[UT];
#pragma unroll
    for (int v = 0; v < UT; ++v) R[v] = cz(C2());
    for (int s0 = 0; s0 < S; s0 += K::SCH) {
        const int rows = min(K::SCH, S - s0);
        stage_h<UT>(Hs, Hc, s0, rows, U, valid, lane);
        __syncwarp();
        for (int r = g; r < rows; r += K::G) {
            const C2 hu = Hs[r * K::HS_LD + u];
#pragma unroll
            for (int v = 0; v < UT; v += 2) {
                C2 a, b;
                ld2(&Hs[r * K::HS_LD + v], a, b);
                if (ALG == ALG_ADMM_DL) {
                    // B_c = H^d H^dH = conj(H^H H): entry sum_s H[s][u] conj(H[s][v])
                    cmacc(R[v], a, hu);
                    cmacc(R[v + 1], b, hu);
                } else {
                    // G_c = H^H H: entry sum_s conj(H[s][u]) H[s][v]
                    cmacc(R[v], hu, a);
                    cmacc(R[v + 1], hu, b);
                }
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int m = UT; m < 32; m <<= 1) {
#pragma unroll
        for (int v = 0; v < UT; ++v) {
            R[v].x += shfl_x(R[v].x, m);
            R[v].y += shfl_x(R[v].y, m);
        }
    }
    const T delta = ParamSel<T>::get(p.delta, p.f_delta);
#pragma unroll
    for (int v = 0; v < UT; ++v)
        if (v == u) R[v].x += delta;

    if (ALG == ALG_ADMM_UL) {
        gj_invert<UT>(R, Vb, u, lane);                   // row u of B_c^{-1}
    } else if (ALG == ALG_ADMM_DL) {
        gj_invert<UT>(R, Vb, u, lane);                   // row u of B_c^{-1}
    }
    // (CG keeps G_c = H_c^H H_c in R.)

    const bool single_stage = (S <= K::SCH);   // H_c still staged in Hs
    int buf = 0;
    const C2 *yw = reinterpret_cast<const C2 *>(p.vin) + (size_t)(valid ? w : 0) * N * (ALG == ALG_ADMM_DL ? U : B);

    for (int n0 = 0; n0 < N; n0 += K::NCH) {
        C2 s_[K::NN];
        C2 acc[K::NN];

        // Consensus over the C clusters of this subcarrier: every warp
        // publishes its U-vector and every entry is summed in cluster order,
        // in two phases: warp c sums its slice of the entries over the C
        // contributions, then every warp reads its entries' sums.  Across the
        // CTAs of a thread-block cluster the contributions and the sums are
        // read through DSMEM, each contribution crossing CTAs once.
        auto consensus = [&](const C2 (&val)[K::NN], C2 (&sum)[K::NN]) {
            C2 *mine = cons + ((size_t)buf * nwarps + warp) * K::CONS_ELEMS;
#pragma unroll
            for (int j = 0; j < K::NN; ++j) mine[(g + K::G * j) * UT + u] = val[j];
            if (CLU) {
                cooperative_groups::cluster_group cg_cl = cooperative_groups::this_cluster();
                constexpr int E = K::CONS_ELEMS;
                const int per = (E + p.C - 1) / p.C;
                cg_cl.sync();
                for (int e = c * per + lane; e < min(E, (c + 1) * per); e += 32) {
                    C2 a = cz(C2());
                    for (int rk = 0; rk < p.CL; ++rk) {
                        const C2 *rb = cg_cl.map_shared_rank(cons + (size_t)buf * nwarps * E, rk);
                        for (int lw = 0; lw < p.CPB; ++lw) {
                            const C2 t = rb[(size_t)lw * E + e];
                            a.x += t.x;
                            a.y += t.y;
                        }
                    }
                    wsum[buf * E + e] = a;
                }
                cg_cl.sync();
#pragma unroll
                for (int j = 0; j < K::NN; ++j) {
                    const int idx = (g + K::G * j) * UT + u;
                    sum[j] = *cg_cl.map_shared_rank(wsum + buf * E + idx, (idx / per) / p.CPB);
                }
            } else {
                constexpr int E = K::CONS_ELEMS;
                const int per = (E + p.C - 1) / p.C;
                C2 *ws = wsum + ((size_t)buf * nsub + pl) * E;
                __syncthreads();
                const C2 *grp = cons_grp + (size_t)buf * nwarps * E;
                for (int e = c * per + lane; e < min(E, (c + 1) * per); e += 32) {
                    C2 a = cz(C2());
                    for (int cc = 0; cc < p.C; ++cc) {
                        const C2 t = grp[(size_t)cc * E + e];
                        a.x += t.x;
                        a.y += t.y;
                    }
                    ws[e] = a;
                }
                __syncthreads();
#pragma unroll
                for (int j = 0; j < K::NN; ++j) sum[j] = ws[(g + K::G * j) * UT + u];
            }
            buf ^= 1;
        };

        if (ALG == ALG_ADMM_UL || ALG == ALG_CG_UL) {
            // ---- Matched filter m_c = H_c^H y_c for the chunk's symbols ----
#pragma unroll
            for (int j = 0; j < K::NN; ++j) acc[j] = cz(C2());
            for (int s0 = 0; s0 < S; s0 += K::SCH) {
                const int rows = min(K::SCH, S - s0);
                if (!single_stage) stage_h<UT>(Hs, Hc, s0, rows, U, valid, lane);
                stage_y<UT>(Ys, yw, n0, N, B, c * S + s0, rows, valid, lane);
                __syncwarp();
                for (int r = 0; r < rows; r += 2) {
                    const C2 h0 = Hs[r * K::HS_LD + u];
                    const C2 h1 = Hs[(r + 1) * K::HS_LD + u];
#pragma unroll
                    for (int j = 0; j < K::NN; ++j) {
                        C2 a, b;
                        ld2(&Ys[(g + K::G * j) * K::YS_LD + r], a, b);
                        cmacc(acc[j], h0, a);
                        cmacc(acc[j], h1, b);
                    }
                }
                __syncwarp();
            }
        }

        if (ALG == ALG_ADMM_UL) {
            // y_c^reg = B_c^{-1} H_c^H y_c
            C2 yreg[K::NN], lam[K::NN], z[K::NN];
            put_vec<UT>(Vb, u, g, acc);
            __syncwarp();
            matvec<UT>(R, Vb, g, yreg);
            __syncwarp();
            // Init: lambda = 0, z = y_reg, s = prox(sum_c z_c)
#pragma unroll
            for (int j = 0; j < K::NN; ++j) { lam[j] = cz(C2()); z[j] = yreg[j]; }
            auto prox = [&](C2 (&sum)[K::NN]) {
#pragma unroll
                for (int j = 0; j < K::NN; ++j) {
                    if (p.reg >= 2) {   // (E2-BOX); BPSK: the real segment [-r, r]
                        const T r = ParamSel<T>::get(p.box_r, p.f_box_r), ic = ParamSel<T>::get(p.invC, p.f_invC);
                        s_[j].x = clip_r(sum[j].x * ic, r);
                        s_[j].y = (p.reg == 2) ? clip_r(sum[j].y * ic, r) : (T)0;
                    } else {
                        s_[j] = cscale(sum[j], ParamSel<T>::get(p.e2_scale, p.f_e2_scale));
                    }
                }
            };
            consensus(z, acc);
            prox(acc);
            const T gam = ParamSel<T>::get(p.gamma, p.f_gamma), rho = ParamSel<T>::get(p.rho, p.f_rho);
            for (int t = 2; t <= p.T; ++t) {
                C2 d[K::NN];
#pragma unroll
                for (int j = 0; j < K::NN; ++j) {
                    // lambda_c += gamma (z_c - s);  d = rho (s - lambda_c)
                    lam[j].x = fma(gam, z[j].x - s_[j].x, lam[j].x);
                    lam[j].y = fma(gam, z[j].y - s_[j].y, lam[j].y);
                    d[j] = cscale(csub(s_[j], lam[j]), rho);
                }
                put_vec<UT>(Vb, u, g, d);
                __syncwarp();
                matvec<UT>(R, Vb, g, z);          // rho B_c^{-1} (s - lambda_c)
                __syncwarp();
                C2 wv[K::NN];
#pragma unroll
                for (int j = 0; j < K::NN; ++j) {
                    z[j] = cadd(z[j], yreg[j]);   // z_c = y_reg + ...
                    wv[j] = cadd(z[j], lam[j]);   // w_c = z_c + lambda_c
                }
                consensus(wv, acc);
                prox(acc);
            }
        } else if (ALG == ALG_CG_UL) {
            C2 r[K::NN], pv[K::NN], x[K::NN];
            T rr[K::NN];
            bool live[K::NN];
            consensus(acc, r);                    // y^MRC = sum_c H_c^H y_c
#pragma unroll
            for (int j = 0; j < K::NN; ++j) {
                pv[j] = r[j];
                x[j] = cz(C2());
                rr[j] = group_sum<UT>(r[j].x * r[j].x + r[j].y * r[j].y);
                live[j] = true;
            }
            const T rcg = ParamSel<T>::get(p.rho_cg, p.f_rho_cg);
            for (int t = 1; t <= p.T; ++t) {
                C2 wc[K::NN], e[K::NN];
                put_vec<UT>(Vb, u, g, pv);
                __syncwarp();
                matvec<UT>(R, Vb, g, wc);         // w_c = H_c^H H_c p
                __syncwarp();
                consensus(wc, e);                 // w = sum_c w_c
#pragma unroll
                for (int j = 0; j < K::NN; ++j) {
                    e[j].x = fma(rcg, pv[j].x, e[j].x);   // e = rho p + w
                    e[j].y = fma(rcg, pv[j].y, e[j].y);
                    const T pe = group_sum<UT>(pv[j].x * e[j].x + pv[j].y * e[j].y);
                    const bool go = live[j] && rr[j] != (T)0 && pe != (T)0;
                    const T alpha = go ? rr[j] / pe : (T)0;
                    x[j].x = fma(alpha, pv[j].x, x[j].x);
                    x[j].y = fma(alpha, pv[j].y, x[j].y);
                    r[j].x = fma(-alpha, e[j].x, r[j].x);
                    r[j].y = fma(-alpha, e[j].y, r[j].y);
                    const T rn = group_sum<UT>(r[j].x * r[j].x + r[j].y * r[j].y);
                    const T beta = go ? rn / rr[j] : (T)0;
                    if (go) {
                        pv[j].x = fma(beta, pv[j].x, r[j].x);
                        pv[j].y = fma(beta, pv[j].y, r[j].y);
                        rr[j] = rn;
                    }
                    live[j] = go;
                }
            }
#pragma unroll
            for (int j = 0; j < K::NN; ++j) s_[j] = x[j];
        } else {  // ALG_ADMM_DL
            C2 sv[K::NN], z[K::NN], lam[K::NN], v[K::NN], m[K::NN];
            const T kap = ParamSel<T>::get(p.kappa, p.f_kappa), gam = ParamSel<T>::get(p.gamma, p.f_gamma), ic = ParamSel<T>::get(p.invC, p.f_invC);
#pragma unroll
            for (int j = 0; j < K::NN; ++j) {
                const int n = n0 + g + K::G * j;
                sv[j] = (valid && u < U && n < N) ? yw[(size_t)n * U + u] : cz(C2());
                z[j] = cscale(sv[j], kap);        // z_c = max{U/B, 1/C} s
                lam[j] = cz(C2());
                v[j] = z[j];
            }
            const T ir = ParamSel<T>::get(p.inv_rho, p.f_inv_rho);
            for (int t = 2; t <= p.T; ++t) {
                put_vec<UT>(Vb, u, g, v);
                __syncwarp();
                matvec<UT>(R, Vb, g, m);          // B_c^{-1} v_c
                __syncwarp();
                // m_c = H_c x_c = v_c - rho^{-1} B_c^{-1} v_c  (v_c = z_c + lambda_c)
#pragma unroll
                for (int j = 0; j < K::NN; ++j) {
                    m[j].x = fma(-ir, m[j].x, v[j].x);
                    m[j].y = fma(-ir, m[j].y, v[j].y);
                }
                C2 wc[K::NN], wsum[K::NN];
#pragma unroll
                for (int j = 0; j < K::NN; ++j) wc[j] = csub(m[j], lam[j]);   // w_c
                consensus(wc, wsum);              // w = sum_c w_c
                if (p.eps > 0.0) {
                    // (P2) by Lemma 2: s - w scaled by max{0, 1 - eps / ||s - w||}
                    const T eps = ParamSel<T>::get(p.eps, p.f_eps);
#pragma unroll
                    for (int j = 0; j < K::NN; ++j) {
                        const C2 dl = csub(sv[j], wsum[j]);
                        const T nrm = sqrt(group_sum<UT>(dl.x * dl.x + dl.y * dl.y));
                        const T k = (nrm > (T)0) ? fmax((T)0, (T)1 - eps / nrm) : (T)0;
                        wsum[j] = csub(sv[j], cscale(dl, k));
                    }
                }
#pragma unroll
                for (int j = 0; j < K::NN; ++j) {
                    // (P2): z_c = w_c + k (s - w) / C (k = 1 for eps = 0)
                    z[j].x = fma(sv[j].x - wsum[j].x, ic, wc[j].x);
                    z[j].y = fma(sv[j].y - wsum[j].y, ic, wc[j].y);
                    // (P3): lambda_c -= gamma (m_c - z_c)
                    lam[j].x = fma(-gam, m[j].x - z[j].x, lam[j].x);
                    lam[j].y = fma(-gam, m[j].y - z[j].y, lam[j].y);
                    v[j] = cadd(z[j], lam[j]);
                }
            }
            // (P1) output: x_c = H^dH_c B_c^{-1} v
            put_vec<UT>(Vb, u, g, v);
            __syncwarp();
            matvec<UT>(R, Vb, g, m);
            __syncwarp();
            put_vec<UT>(Vb, u, g, m);
            __syncwarp();
            // x_c[s'][n] = sum_u conj(H_c[s'][u]) t[u][n]; lanes run over s'.
            C2 *xo = reinterpret_cast<C2 *>(p.out);
            T energy = (T)0;
            for (int r0 = 0; r0 < S; r0 += 32) {
                const int sr = r0 + lane;
                C2 h[UT];
#pragma unroll
                for (int k = 0; k < UT; ++k)
                    h[k] = (valid && sr < S && k < U) ? Hc[(size_t)sr * U + k] : cz(C2());
                for (int nl = 0; nl < K::NCH; ++nl) {
                    const int n = n0 + nl;
                    if (n >= N) break;
                    C2 a = cz(C2());
#pragma unroll
                    for (int k = 0; k < UT; k += 2) {
                        C2 t0, t1;
                        ld2(&Vb[nl * K::V_LD + k], t0, t1);
                        cmacc(a, h[k], t0);
                        cmacc(a, h[k + 1], t1);
                    }
                    if (valid && sr < S) {
                        xo[((size_t)w * N + n) * B + (size_t)c * S + sr] = a;
                        energy += a.x * a.x + a.y * a.y;
                    }
                }
            }
            __syncwarp();
            if (p.energy != nullptr) {
#pragma unroll
                for (int m2 = 16; m2 > 0; m2 >>= 1) energy += shfl_x(energy, m2);
                if (lane == 0 && valid) atomicAdd(p.energy, (double)energy);
            }
        }

        // ---- Uplink output: x_hat and labels, written by cluster 0 ----
        if (ALG != ALG_ADMM_DL && c == 0 && valid && u < U) {
            C2 *xo = reinterpret_cast<C2 *>(p.out);
#pragma unroll
            for (int j = 0; j < K::NN; ++j) {
                const int n = n0 + g + K::G * j;
                if (n < N) {
                    const size_t o = ((size_t)w * N + n) * U + u;
                    xo[o] = s_[j];
                    if (p.labels != nullptr)
                        p.labels[o] = qam_label<T>(s_[j].x, s_[j].y, ParamSel<T>::get(p.qam_inv_a, p.f_qam_inv_a), p.qam_L, p.qam_half);
                }
            }
        }
    }
    // Keep this CTA's shared memory alive until every CTA of the cluster has
    // finished reading it.
    if (CLU) cooperative_groups::this_cluster().sync();
}

// Downlink power normalisation: x *= beta, beta = sqrt(count / sum |x|^2).
template <typename T>
__global__ void dbp_scale_kernel(typename C2Of<T>::type *x, size_t n, const double *energy,
                                 double count, double *beta_out) {
    const double e = *energy;
    const double beta = (e > 0.0) ? sqrt(count / e) : 0.0;
    const T b = (T)beta;
    // four independent loads in flight per thread before the stores
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        auto a0 = x[i], a1 = x[i + stride], a2 = x[i + 2 * stride], a3 = x[i + 3 * stride];
        a0.x *= b; a0.y *= b;
        a1.x *= b; a1.y *= b;
        a2.x *= b; a2.y *= b;
        a3.x *= b; a3.y *= b;
        x[i] = a0;
        x[i + stride] = a1;
        x[i + 2 * stride] = a2;
        x[i + 3 * stride] = a3;
    }
    for (; i < n; i += stride) {
        x[i].x *= b;
        x[i].y *= b;
    }
    if (beta_out != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *beta_out = beta;
}

}  // namespace dbp
