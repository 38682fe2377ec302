// dbp_mma8.cuh -- uplink kernel for U = 8 users with FP32 inputs in which every
// dense complex product runs on the tensor cores: the Gram H_c^H H_c, the
// matched filter H_c^H y_c and, in every iteration, the product of the
// per-cluster operator (B_c^{-1} for Alg. 1, G_c for Alg. 2) with the
// cluster's 8 x N state.
//
// FP32 accuracy from TF32 tensor cores: every operand x is split into
// x_hi = tf32(x) and x_lo = tf32(x - x_hi), and a product is accumulated as
// a_lo b_hi + a_hi b_lo + a_hi b_hi in FP32 (the a_lo b_lo term, ~2^-22
// relative, is dropped) -- three mma.sync.m16n8k8.tf32 per product.
//
// Complex products are embedded in real ones with real/imaginary parts
// interleaved along the contraction, k' = 2k + a:
//   Re C[u][n] = sum_k' A_re[u][k'] B'[k'][n],  Im C[u][n] = sum_k' A_im[u][k'] B'[k'][n]
//   A_re[u][2k:2k+2] = (Re A[u][k], -Im A[u][k]),  A_im[u][2k:2k+2] = (Im A[u][k], Re A[u][k]),
//   B'[2k:2k+2][n] = (Re B[k][n], Im B[k][n]),
// and one m16 tile holds the 8 real rows over the 8 imaginary rows, so the
// accumulator gives lane (g, t) = (lane / 4, lane % 4) the complex results
// C[g][8nt + 2t] = (d0, d2) and C[g][8nt + 2t + 1] = (d1, d3).
//
// Every per-cluster vector therefore lives in that accumulator layout: lane
// (g, t) holds user u = g and the symbols n = 8 (q >> 1) + 2t + (q & 1),
// q = 0..3 (16 symbol slots; N <= 16 per pass).  The matched filter lands
// there directly; the operator is inverted in place by a shuffle-based
// Gauss-Jordan elimination with each lane holding row g, columns 2t, 2t+1;
// state vectors go back into B fragments through a small shared-memory
// transpose.  Everything else (staging, consensus, prox, CG scalars, slicer,
// resident operator, FP64 retry) follows dbp_tma_kernel.
#pragma once

#include "dbp_tma.cuh"

namespace dbp {

__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void split3(float x, uint32_t &hi, uint32_t &lo) {
    hi = tf32_bits(x);
    lo = tf32_bits(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// d += A B with A = ah + al and B = bh + bl (three TF32 products).
__device__ __forceinline__ void mma3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4], uint32_t bh0,
                                     uint32_t bh1, uint32_t bl0, uint32_t bl1) {
    mma_tf32(d, al[0], al[1], al[2], al[3], bh0, bh1);
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bl0, bl1);
    mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bh0, bh1);
}

// A fragment of H_c^H for one k-step (complex rows s0..s0+3 of H_c):
// lane (g, t) takes H[s0 + t/2][g] and H[s0 + 2 + t/2][g], component t & 1
// for the real rows and the matching component of the rotation for the
// imaginary rows.  Returns the raw values (a0..a3) before splitting.
__device__ __forceinline__ void hh_frag(const float2 *Hs, int s0, int g, int t, float (&a)[4]) {
    const float2 h0 = Hs[(s0 + (t >> 1)) * 8 + g];
    const float2 h1 = Hs[(s0 + 2 + (t >> 1)) * 8 + g];
    const bool odd = t & 1;
    // conj(H)^T: Re-block (Re, -Im of conj(H)) = (Re H, Im H); Im-block = (-Im H, Re H)
    a[0] = odd ? h0.y : h0.x;
    a[1] = odd ? h0.x : -h0.y;
    a[2] = odd ? h1.y : h1.x;
    a[3] = odd ? h1.x : -h1.y;
}

// Gauss-Jordan inversion of the 8 x 8 Hermitian positive definite matrix
// whose row g, columns 2t and 2t+1, lane (g, t) holds in (e0, e1).  No
// pivoting (every pivot is a Schur complement of an HPD matrix).  The pivot
// row reaches the other lanes by shuffles.  Returns the smallest pivot's
// real part.
template <typename C2, typename T>
__device__ __forceinline__ T gj8(C2 &e0, C2 &e1, int g, int t) {
    T min_piv = (T)3.0e38;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        C2 P0, P1, pk, mk;
        const int src_row = 4 * k + t;            // row k, my two columns
        P0.x = __shfl_sync(0xffffffffu, e0.x, src_row);
        P0.y = __shfl_sync(0xffffffffu, e0.y, src_row);
        P1.x = __shfl_sync(0xffffffffu, e1.x, src_row);
        P1.y = __shfl_sync(0xffffffffu, e1.y, src_row);
        const int piv_lane = 4 * k + (k >> 1);    // A[k][k]
        const T pkx = __shfl_sync(0xffffffffu, (k & 1) ? e1.x : e0.x, piv_lane);
        const T pky = __shfl_sync(0xffffffffu, (k & 1) ? e1.y : e0.y, piv_lane);
        pk.x = pkx;
        pk.y = pky;
        const int my_k = 4 * g + (k >> 1);        // A[g][k]
        mk.x = __shfl_sync(0xffffffffu, (k & 1) ? e1.x : e0.x, my_k);
        mk.y = __shfl_sync(0xffffffffu, (k & 1) ? e1.y : e0.y, my_k);
        min_piv = (pk.x < min_piv) ? pk.x : min_piv;
        C2 inv;
        if constexpr (sizeof(T) == 4) {
            const float dd = __frcp_rn(fmaf(pk.x, pk.x, pk.y * pk.y));
            inv.x = pk.x * dd;
            inv.y = -pk.y * dd;
        } else {
            inv = crcp(pk);
        }
        const bool me = (g == k);
        C2 f;
        if (me) {
            f.x = (T)1 - inv.x;
            f.y = -inv.y;
        } else {
            f = cmul(mk, inv);
        }
        const C2 nf = mkc(-f.x, -f.y);
        const C2 colk = me ? inv : nf;
        if (2 * t == k) e0 = colk;
        else cmac(e0, nf, P0);
        if (2 * t + 1 == k) e1 = colk;
        else cmac(e1, nf, P1);
    }
    return min_piv;
}

template <int ALG>
__global__ void __launch_bounds__(512) dbp_mma8_kernel(const FusedParams p) {
    using C2 = float2;
    constexpr int E = 16 * 8;                         // consensus entries (16 symbol slots x 8 users)
    constexpr int VP = 10;                            // transpose buffer pitch (float2): conflict-free B loads
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int C = p.C, P = p.P, S = p.S, N = p.N, B = p.B, W = p.W;
    const int pl = warp / C, c = warp - pl * C;
    const int g = lane >> 2, t = lane & 3;
    const int yp = p.yp;

    unsigned char *wb = smem_raw + (size_t)warp * p.warp_bytes;
    C2 *Vs = reinterpret_cast<C2 *>(wb + p.off_v);    // [16][VP]
    C2 *contrib = reinterpret_cast<C2 *>(smem_raw + (size_t)nwarps * p.warp_bytes);   // [2][nwarps][E]
    C2 *wsum = contrib + 2 * (size_t)nwarps * E;                                        // [2][P][E]
    uint64_t *bars = reinterpret_cast<uint64_t *>(wsum + 2 * (size_t)P * E) + 2 * warp;

    for (int i = lane * 16; i < p.warp_bytes; i += 32 * 16)
        *reinterpret_cast<float4 *>(wb + i) = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    fence_proxy_async();

    const C2 *Hg = reinterpret_cast<const C2 *>(p.H);
    const C2 *Yg = reinterpret_cast<const C2 *>(p.vin);

    auto issue = [&](int w, int b) {
        const uint32_t hbytes = (uint32_t)(S * 8 * sizeof(C2));
        const uint32_t ybytes = (uint32_t)(S * sizeof(C2));
        fence_proxy_async();
        if (lane == 0) mbar_arrive_expect_tx(&bars[b], hbytes + (uint32_t)N * ybytes);
        __syncwarp();
        if (lane == 0)
            bulk_g2s(wb + (b ? p.off_h1 : 0), Hg + ((size_t)w * B + (size_t)c * S) * 8, hbytes, &bars[b]);
        unsigned char *ydst = wb + (b ? p.off_y1 : p.off_y0);
        for (int n = lane; n < N; n += 32)
            bulk_g2s(ydst + (size_t)n * yp * sizeof(C2), Yg + ((size_t)w * N + n) * B + (size_t)c * S, ybytes,
                     &bars[b]);
    };

    // state entry q of this lane: user g, symbol n0 + 8 (q >> 1) + 2t + (q & 1)
    auto nof = [&](int q) { return 8 * (q >> 1) + 2 * t + (q & 1); };

    uint32_t parity = 0u;
    int tile = blockIdx.x;
    if (tile < p.tiles && tile * P + pl < W) issue(tile * P + pl, 0);
    int buf = 0;

    for (int it = 0; tile < p.tiles; ++it, tile += gridDim.x) {
        const int b = it & 1;
        const int w = tile * P + pl;
        const bool valid = (w < W);
        const int ntile = tile + gridDim.x;
        if (ntile < p.tiles && ntile * P + pl < W) issue(ntile * P + pl, b ^ 1);
        if (valid) {
            mbar_wait_bounded(&bars[b], (parity >> b) & 1u, p.status);
            parity ^= (1u << b);
        }
        const C2 *Hs = reinterpret_cast<const C2 *>(wb + (b ? p.off_h1 : 0));
        const C2 *Ys = reinterpret_cast<const C2 *>(wb + (b ? p.off_y1 : p.off_y0));

        // ---- Gram and matched filter on the tensor cores (k-steps of 4 antennas) ----
        const int nblk = (N + 15) / 16;               // symbol passes of 16
        float gacc[4] = {0.f, 0.f, 0.f, 0.f};
        float macc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
        const bool need_gram = (p.factor_mode != 2);
        for (int s0 = 0; s0 < p.h_rows; s0 += 4) {
            float a[4];
            hh_frag(Hs, s0, g, t, a);
            uint32_t ah[4], al[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) split3(a[i], ah[i], al[i]);
            if (need_gram) mma3(gacc, ah, al, ah[0], ah[2], al[0], al[2]);   // B = H_c: same values
            if (nblk == 1) {
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    const float2 y0 = Ys[(8 * nt + g) * yp + s0 + (t >> 1)];
                    const float2 y1 = Ys[(8 * nt + g) * yp + s0 + 2 + (t >> 1)];
                    uint32_t bh0, bl0, bh1, bl1;
                    split3((t & 1) ? y0.y : y0.x, bh0, bl0);
                    split3((t & 1) ? y1.y : y1.x, bh1, bl1);
                    mma3(macc[nt], ah, al, bh0, bh1, bl0, bl1);
                }
            }
        }

        // ---- Per-cluster operator, entries (g, 2t) and (g, 2t+1) ----
        C2 e0, e1;
        C2 *frow = (p.factor != nullptr && valid) ? p.factor + (((size_t)w * C + c) * 8 + g) * 8 + 2 * t : nullptr;
        if (!need_gram) {
            if (frow != nullptr) {
                const float4 q = *reinterpret_cast<const float4 *>(frow);
                e0 = make_float2(q.x, q.y);
                e1 = make_float2(q.z, q.w);
            } else {
                e0 = e1 = make_float2(0.f, 0.f);
            }
        } else {
            e0 = make_float2(gacc[0], gacc[2]);
            e1 = make_float2(gacc[1], gacc[3]);
            if (ALG == ALG_ADMM_UL) {
                const float delta = p.f_delta;
                if (2 * t == g) e0.x += delta;
                if (2 * t + 1 == g) e1.x += delta;
                float dmax = (2 * t == g) ? e0.x : ((2 * t + 1 == g) ? e1.x : 0.f);
#pragma unroll
                for (int m = 16; m > 0; m >>= 1) dmax = fmaxf(dmax, shfl_x(dmax, m));
                const float min_piv = gj8<float2, float>(e0, e1, g, t);
                if (valid && !(min_piv >= 0x1p-12f * dmax)) {
                    // FP64 retry of this cluster's Gram and inverse
                    double2 d0 = make_double2(0.0, 0.0), d1 = make_double2(0.0, 0.0);
                    for (int r = 0; r < S; ++r) {
                        const float2 hu = Hs[r * 8 + g], h0 = Hs[r * 8 + 2 * t], h1 = Hs[r * 8 + 2 * t + 1];
                        const double2 hd = make_double2(hu.x, hu.y);
                        cmacc(d0, hd, make_double2(h0.x, h0.y));
                        cmacc(d1, hd, make_double2(h1.x, h1.y));
                    }
                    if (2 * t == g) d0.x += p.delta;
                    if (2 * t + 1 == g) d1.x += p.delta;
                    gj8<double2, double>(d0, d1, g, t);
                    e0 = make_float2((float)d0.x, (float)d0.y);
                    e1 = make_float2((float)d1.x, (float)d1.y);
                    if (lane == 0 && p.retries) atomicAdd(p.retries, 1u);
                }
            }
            if (p.factor_mode == 1 && frow != nullptr)
                *reinterpret_cast<float4 *>(frow) = make_float4(e0.x, e0.y, e1.x, e1.y);
        }
        // A fragments (hi, lo) of the operator for the two k-steps (users 0-3, 4-7):
        // lane (g, t) needs Op[g][4ks + t/2] and Op[g][4ks + 2 + t/2].
        uint32_t oh[2][4], ol[2][4];
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                // columns 4ks + 2 half + {0, 1} sit in lane (g, 2 ks + half)
                const int srcl = 4 * g + 2 * ks + half;
                C2 v0, v1;
                v0.x = __shfl_sync(0xffffffffu, e0.x, srcl);
                v0.y = __shfl_sync(0xffffffffu, e0.y, srcl);
                v1.x = __shfl_sync(0xffffffffu, e1.x, srcl);
                v1.y = __shfl_sync(0xffffffffu, e1.y, srcl);
                const C2 o = (t >> 1) ? v1 : v0;      // Op[g][4ks + 2 half + t/2]
                const bool odd = t & 1;
                // A_re = (Re, -Im), A_im = (Im, Re) of a general complex operator
                const float are = odd ? -o.y : o.x;
                const float aim = odd ? o.x : o.y;
                split3(are, oh[ks][2 * half], ol[ks][2 * half]);
                split3(aim, oh[ks][2 * half + 1], ol[ks][2 * half + 1]);
            }
        }

        // Operator times the state X (accumulator layout) -> out (same layout).
        auto apply = [&](const C2 (&x)[4], C2 (&out)[4]) {
#pragma unroll
            for (int q = 0; q < 4; ++q) Vs[nof(q) * VP + g] = x[q];
            __syncwarp();
            float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
            const float *Vf = reinterpret_cast<const float *>(Vs);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    const int n = 8 * nt + g;
                    const float b0 = Vf[(n * VP + 4 * ks + (t >> 1)) * 2 + (t & 1)];
                    const float b1 = Vf[(n * VP + 4 * ks + 2 + (t >> 1)) * 2 + (t & 1)];
                    uint32_t bh0, bl0, bh1, bl1;
                    split3(b0, bh0, bl0);
                    split3(b1, bh1, bl1);
                    mma3(acc[nt], oh[ks], ol[ks], bh0, bh1, bl0, bl1);
                }
            }
            __syncwarp();
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                out[2 * nt] = make_float2(acc[nt][0], acc[nt][2]);
                out[2 * nt + 1] = make_float2(acc[nt][1], acc[nt][3]);
            }
        };

        for (int blk = 0; blk < nblk; ++blk) {
            const int n0 = 16 * blk;
            C2 m[4];
            if (nblk == 1) {
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    m[2 * nt] = make_float2(macc[nt][0], macc[nt][2]);
                    m[2 * nt + 1] = make_float2(macc[nt][1], macc[nt][3]);
                }
            } else {
                float ma[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
                for (int s0 = 0; s0 < p.h_rows; s0 += 4) {
                    float a[4];
                    hh_frag(Hs, s0, g, t, a);
                    uint32_t ah[4], al[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) split3(a[i], ah[i], al[i]);
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) {
                        const float2 y0 = Ys[(n0 + 8 * nt + g) * yp + s0 + (t >> 1)];
                        const float2 y1 = Ys[(n0 + 8 * nt + g) * yp + s0 + 2 + (t >> 1)];
                        uint32_t bh0, bl0, bh1, bl1;
                        split3((t & 1) ? y0.y : y0.x, bh0, bl0);
                        split3((t & 1) ? y1.y : y1.x, bh1, bl1);
                        mma3(ma[nt], ah, al, bh0, bh1, bl0, bl1);
                    }
                }
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    m[2 * nt] = make_float2(ma[nt][0], ma[nt][2]);
                    m[2 * nt + 1] = make_float2(ma[nt][1], ma[nt][3]);
                }
            }

            // Two-phase consensus over the C clusters of this subcarrier.
            auto consensus = [&](const C2 (&val)[4], C2 (&sum)[4]) {
                C2 *mine = contrib + ((size_t)buf * nwarps + warp) * E;
#pragma unroll
                for (int q = 0; q < 4; ++q) mine[nof(q) * 8 + g] = val[q];
                __syncthreads();
                const C2 *grp = contrib + ((size_t)buf * nwarps + pl * C) * E;
                C2 *ws = wsum + ((size_t)buf * P + pl) * E;
                const int per = (E + C - 1) / C;
                for (int e = c * per + lane; e < min(E, (c + 1) * per); e += 32) {
                    C2 a2 = make_float2(0.f, 0.f);
                    for (int cc = 0; cc < C; ++cc) {
                        const C2 tv = grp[(size_t)cc * E + e];
                        a2.x += tv.x;
                        a2.y += tv.y;
                    }
                    ws[e] = a2;
                }
                __syncthreads();
#pragma unroll
                for (int q = 0; q < 4; ++q) sum[q] = ws[nof(q) * 8 + g];
                buf ^= 1;
            };

            C2 s_[4];
            if (ALG == ALG_ADMM_UL) {
                C2 yreg[4], lam[4], z[4], acc[4];
                apply(m, yreg);                       // y_reg = B_c^{-1} H_c^H y_c
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    lam[q] = make_float2(0.f, 0.f);
                    z[q] = yreg[q];
                }
                auto prox = [&](C2 (&sum)[4]) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (p.reg == 2) {
                            const float r = p.f_box_r, ic = p.f_invC;
                            s_[q].x = clip_r(sum[q].x * ic, r);
                            s_[q].y = clip_r(sum[q].y * ic, r);
                        } else {
                            s_[q] = cscale(sum[q], p.f_e2_scale);
                        }
                    }
                };
                consensus(z, acc);
                prox(acc);
                const float gam = p.f_gamma, rho = p.f_rho;
                for (int it2 = 2; it2 <= p.T; ++it2) {
                    C2 d[4], wv[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        lam[q].x = fmaf(gam, z[q].x - s_[q].x, lam[q].x);
                        lam[q].y = fmaf(gam, z[q].y - s_[q].y, lam[q].y);
                        d[q] = cscale(csub(s_[q], lam[q]), rho);
                    }
                    apply(d, z);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        z[q] = cadd(z[q], yreg[q]);
                        wv[q] = cadd(z[q], lam[q]);
                    }
                    consensus(wv, acc);
                    prox(acc);
                }
            } else {  // ALG_CG_UL: operator = G_c
                C2 r[4], pv[4], x[4];
                float rr[4];
                consensus(m, r);                      // y^MRC
                // dot products over the 8 users: lanes with the same t
                auto usum = [&](float v) {
                    v += shfl_x(v, 4);
                    v += shfl_x(v, 8);
                    v += shfl_x(v, 16);
                    return v;
                };
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    pv[q] = r[q];
                    x[q] = make_float2(0.f, 0.f);
                    rr[q] = usum(r[q].x * r[q].x + r[q].y * r[q].y);
                }
                const float rcg = p.f_rho_cg;
                for (int it2 = 1; it2 <= p.T; ++it2) {
                    C2 wc[4], e[4];
                    apply(pv, wc);                    // w_c = G_c p
                    consensus(wc, e);                 // w = sum_c w_c
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        e[q].x = fmaf(rcg, pv[q].x, e[q].x);
                        e[q].y = fmaf(rcg, pv[q].y, e[q].y);
                        const float pe = usum(pv[q].x * e[q].x + pv[q].y * e[q].y);
                        // a symbol whose residual or curvature is exactly zero keeps its iterate
                        const bool go = rr[q] != 0.f && pe != 0.f;
                        const float alpha = go ? __fdividef(rr[q], pe) : 0.f;
                        x[q].x = fmaf(alpha, pv[q].x, x[q].x);
                        x[q].y = fmaf(alpha, pv[q].y, x[q].y);
                        r[q].x = fmaf(-alpha, e[q].x, r[q].x);
                        r[q].y = fmaf(-alpha, e[q].y, r[q].y);
                        const float rn = usum(r[q].x * r[q].x + r[q].y * r[q].y);
                        const float beta = go ? __fdividef(rn, rr[q]) : 0.f;
                        if (go) {
                            pv[q].x = fmaf(beta, pv[q].x, r[q].x);
                            pv[q].y = fmaf(beta, pv[q].y, r[q].y);
                            rr[q] = rn;
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) s_[q] = x[q];
            }

            // outputs: warp c writes the entries q with q % C == c
            if (valid) {
                C2 *xo = reinterpret_cast<C2 *>(p.out);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int n = n0 + nof(q);
                    if ((q % C) == c && n < N) {
                        const size_t o = ((size_t)w * N + n) * 8 + g;
                        xo[o] = s_[q];
                        if (p.labels != nullptr)
                            p.labels[o] = qam_label<float>(s_[q].x, s_[q].y, p.f_qam_inv_a, p.qam_L, p.qam_half);
                    }
                }
            }
        }
    }
}

}  // namespace dbp
