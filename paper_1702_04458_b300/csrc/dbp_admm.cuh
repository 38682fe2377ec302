// dbp_admm.cuh -- decentralized consensus-ADMM uplink detection (Alg. 1) on
// CUDA cores: one warp per (subcarrier, cluster), register budget of 64 per
// thread so that four 8-warp CTAs share an SM, one staging buffer per warp.
//
// Per cluster c (all local, Sec. III-B): B_c = H_c^H H_c + rho I, its inverse,
// the matched filter m_c = H_c^H y_c, y_c^reg = B_c^{-1} m_c, and per
// iteration lambda_c += gamma (z_c - s), z_c = y_c^reg + rho B_c^{-1}(s -
// lambda_c).  The consensus w = sum_c (z_c + lambda_c) and the (E2) prox of
// Lemma 1 run once per symbol: warp c reduces and applies the prox to the
// units c, c + C, ... of 32 (symbol, user) entries of the chunk and s is
// broadcast through shared memory (the centralized unit, spread over the
// cluster warps).
//
// The Gram and the Gauss-Jordan inverse run in a column-split layout: lane
// (u, g) holds columns [g*CPG, (g+1)*CPG) of row u, so the UT / CPG groups of
// a warp share the elimination instead of repeating it.  The pivot, the
// multiplier of each row and the pivot row travel by warp shuffles.  The
// inverse is then gathered into row u per lane for the mat-vecs.
#pragma once

#include "dbp_fused.cuh"
#include "dbp_tma.cuh"
#include "dbp_cg.cuh"

namespace dbp {

template <int UT> struct Split {
    static constexpr int G = 32 / UT;                          // lane groups
    static constexpr int CPG = (UT / G) > 0 ? UT / G : 1;      // columns per group
    static constexpr int NG = UT / CPG;                        // groups with distinct columns
};

template <int UT> struct AdmmCfg {
    using K = Tile<UT>;
    static constexpr int E = K::NCH * UT;                       // (symbol, user) entries per chunk
    static constexpr int VB = (K::NCH * K::V_LD > UT * UT) ? K::NCH * K::V_LD : UT * UT;   // scratch, complex
};

// Shared memory after the warps' regions (host computes the same):
//   contrib[nwarps][E] float2 | s[P][E] float2 | mbarrier[nwarps]
template <int UT> __host__ __device__ constexpr size_t admm_cta_bytes(int nwarps, int P) {
    return (size_t)nwarps * AdmmCfg<UT>::E * 8 + (size_t)P * AdmmCfg<UT>::E * 8 + (size_t)nwarps * 8;
}

// Gauss-Jordan inversion (no pivoting: every pivot is a Schur complement of
// an HPD matrix) in the column-split layout.  A[i] = entry (u, g*CPG + i) on
// entry and of the inverse on exit; returns the smallest pivot's real part
// (identical on every lane).
//
// Step k with pivot p = A[k][k] and f_u = A[u][k]: every other row takes
// A[u][j] -= (f_u / p) A[k][j] for j != k and A[u][k] = -f_u / p.  The pivot
// row is left as it is, with A[k][k] = 1, and is divided by its pivot once,
// after the last step: a row that has been a pivot row stays p times the
// row of the textbook order through every later step, so the result is the
// same, and no step forms 1 - 1/p (which loses the row's significant bits
// when |p| is large).
template <int UT>
__device__ __forceinline__ float gj_split(float2 (&A)[Split<UT>::CPG], int u, int g) {
    using SP = Split<UT>;
    float min_piv = 3.4e38f;
    float2 myinv = make_float2(1.f, 0.f);     // 1 / the pivot of row u's own step
#pragma unroll
    for (int k = 0; k < UT; ++k) {
        const int gk = k / SP::CPG, ik = k % SP::CPG;
        float2 piv, f, rk[SP::CPG];
        piv.x = __shfl_sync(0xffffffffu, A[ik].x, k + UT * gk);
        piv.y = __shfl_sync(0xffffffffu, A[ik].y, k + UT * gk);
        f.x = __shfl_sync(0xffffffffu, A[ik].x, u + UT * gk);
        f.y = __shfl_sync(0xffffffffu, A[ik].y, u + UT * gk);
#pragma unroll
        for (int i = 0; i < SP::CPG; ++i) {
            rk[i].x = __shfl_sync(0xffffffffu, A[i].x, k + UT * g);
            rk[i].y = __shfl_sync(0xffffffffu, A[i].y, k + UT * g);
        }
        min_piv = fminf(min_piv, piv.x);
        const float dd = rcp_approx(fmaf(piv.x, piv.x, piv.y * piv.y));
        const float2 inv = make_float2(piv.x * dd, -piv.y * dd);
        const bool me = (u == k);
        const float2 fi = cmul(f, inv);                  // f_u / p
        const float2 nm = me ? make_float2(0.f, 0.f) : make_float2(-fi.x, -fi.y);
        if (me) myinv = inv;
#pragma unroll
        for (int i = 0; i < SP::CPG; ++i) cmac(A[i], nm, rk[i]);
        if (g % SP::NG == gk) A[ik] = me ? make_float2(1.f, 0.f) : make_float2(-fi.x, -fi.y);
    }
#pragma unroll
    for (int i = 0; i < SP::CPG; ++i) A[i] = cmul(A[i], myinv);
    return min_piv;
}

template <int UT>
__global__ void __launch_bounds__(512, (UT <= 8) ? 2 : 1) dbp_admm_kernel(const FusedParams p) {
    using C2 = float2;
    using K = Tile<UT>;
    using SP = Split<UT>;
    constexpr int E = AdmmCfg<UT>::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int C = p.C, P = p.P, S = p.S, N = p.N, B = p.B, W = p.W;
    const int pl = warp / C, c = warp - pl * C;
    const int u = lane % UT, g = lane / UT;
    const int yp = p.yp;

    unsigned char *wb = smem_raw + (size_t)warp * p.warp_bytes;
    const C2 *Hs = reinterpret_cast<const C2 *>(wb);
    const C2 *Ys = reinterpret_cast<const C2 *>(wb + p.off_y0);
    C2 *Vb = reinterpret_cast<C2 *>(wb + p.off_v);
    C2 *Yr = reinterpret_cast<C2 *>(wb + p.off_g);                                      // y_c^reg [NCH][UT]
    C2 *contrib = reinterpret_cast<C2 *>(smem_raw + (size_t)nwarps * p.warp_bytes);   // [nwarps][E]
    C2 *sb = contrib + (size_t)nwarps * E + (size_t)pl * E;                             // this subcarrier's s
    uint64_t *bar = reinterpret_cast<uint64_t *>(contrib + (size_t)nwarps * E + (size_t)P * E) + warp;
    const C2 *grp = contrib + pl * C * E;

    for (int i = lane * 16; i < p.warp_bytes; i += 32 * 16)
        *reinterpret_cast<float4 *>(wb + i) = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    fence_proxy_async();

    const C2 *Hg = reinterpret_cast<const C2 *>(p.H);
    const C2 *Yg = reinterpret_cast<const C2 *>(p.vin);
    auto issue = [&](int w) {
        const uint32_t hbytes = (uint32_t)(S * UT * 8);
        const uint32_t ybytes = (uint32_t)(S * 8);
        fence_proxy_async();
        if (lane == 0) mbar_arrive_expect_tx(bar, hbytes + (uint32_t)N * ybytes + p.starve_bytes);
        __syncwarp();
        if (lane == 0) bulk_g2s(wb, Hg + ((size_t)w * B + (size_t)c * S) * UT, hbytes, bar);
        for (int n = lane; n < N; n += 32)
            bulk_g2s(wb + p.off_y0 + (size_t)n * yp * 8, Yg + ((size_t)w * N + n) * B + (size_t)c * S, ybytes, bar);
    };

    grid_dependency_wait();
    grid_dependents_launch();
    uint32_t phase = 0u;
    int tile = blockIdx.x;
    if (tile < p.tiles && tile * P + pl < W) issue(tile * P + pl);

    for (; tile < p.tiles; tile += gridDim.x) {
        const int w = tile * P + pl;
        const bool valid = (w < W);
        const int nw = (tile + (int)gridDim.x) * P + pl;
        const bool prefetch = (tile + (int)gridDim.x < p.tiles) && nw < W;
        if (valid) {
            mbar_wait_bounded(bar, phase, p.status, p.wait_iters);
            phase ^= 1u;
        }

        // ---- B_c^{-1}, row u per lane ----
        C2 R[UT];
        C2 *frow = (p.factor != nullptr && valid) ? p.factor + (((size_t)w * C + c) * UT + u) * UT : nullptr;
        if (p.factor_mode == 2) {
#pragma unroll
            for (int v = 0; v < UT; v += 2) {
                float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                if (frow != nullptr) q = *reinterpret_cast<const float4 *>(&frow[v]);
                R[v] = make_float2(q.x, q.y);
                R[v + 1] = make_float2(q.z, q.w);
            }
        } else {
            // Gram B_c = H_c^H H_c + rho I in the column-split layout.
            const int col0 = (g % SP::NG) * SP::CPG;
            C2 A[SP::CPG];
#pragma unroll
            for (int i = 0; i < SP::CPG; ++i) A[i] = make_float2(0.f, 0.f);
            for (int r = 0; r < S; ++r) {
                const C2 hu = Hs[r * UT + u];
                if constexpr (SP::CPG == 1) {
                    cmacc(A[0], hu, Hs[r * UT + col0]);
                } else {
#pragma unroll
                    for (int i = 0; i < SP::CPG; i += 2) {
                        C2 a, b;
                        ld2(&Hs[r * UT + col0 + i], a, b);
                        cmacc(A[i], hu, a);
                        cmacc(A[i + 1], hu, b);
                    }
                }
            }
            const float delta = p.f_delta;
            float dmax = 0.f;
#pragma unroll
            for (int i = 0; i < SP::CPG; ++i)
                if (col0 + i == u) {
                    A[i].x += delta;
                    dmax = A[i].x;
                }
            dmax = warp_redux_max(dmax);
            const float min_piv = gj_split<UT>(A, u, g);
            if (!(min_piv >= 0x1p-12f * dmax) && valid) {
                // FP64 retry: Gram and inverse of this cluster again in FP64
                // (row u per lane, every group a copy).
                double2 D[UT];
#pragma unroll
                for (int v = 0; v < UT; ++v) D[v] = make_double2(0.0, 0.0);
                for (int r = 0; r < S; ++r) {
                    const C2 hu = Hs[r * UT + u];
                    const double2 hd = make_double2(hu.x, hu.y);
#pragma unroll
                    for (int v = 0; v < UT; ++v) {
                        const C2 hv = Hs[r * UT + v];
                        cmacc(D[v], hd, make_double2(hv.x, hv.y));
                    }
                }
#pragma unroll
                for (int v = 0; v < UT; ++v)
                    if (v == u) D[v].x += p.delta;
                __syncwarp();
                gj_invert<UT>(D, reinterpret_cast<double2 *>(Vb), u, lane);
#pragma unroll
                for (int v = 0; v < UT; ++v) R[v] = make_float2((float)D[v].x, (float)D[v].y);
                if (lane == 0 && p.retries) atomicAdd(p.retries, 1u);
                __syncwarp();
            } else {
                // gather row u of the inverse
                if (g < SP::NG) {
#pragma unroll
                    for (int i = 0; i < SP::CPG; ++i) Vb[u * UT + col0 + i] = A[i];
                }
                __syncwarp();
#pragma unroll
                for (int v = 0; v < UT; v += 2) ld2(&Vb[u * UT + v], R[v], R[v + 1]);
                __syncwarp();
            }
            if (p.factor_mode == 1 && frow != nullptr && g == 0) {
#pragma unroll
                for (int v = 0; v < UT; v += 2)
                    *reinterpret_cast<float4 *>(&frow[v]) = make_float4(R[v].x, R[v].y, R[v + 1].x, R[v + 1].y);
            }
        }

        for (int n0 = 0; n0 < N; n0 += K::NCH) {
            const int nvu = min(K::NCH, N - n0) * UT;     // (symbol, user) entries in this chunk

            // Matched filter and regularised estimate y_c^reg = B_c^{-1} H_c^H y_c
            // (kept in shared memory; z_c starts from it).
            C2 z[K::NN], lam[K::NN], s[K::NN];
            {
                C2 acc[K::NN];
#pragma unroll
                for (int j = 0; j < K::NN; ++j) acc[j] = make_float2(0.f, 0.f);
                const C2 *yr = Ys + (n0 + g) * yp;
                const int js = K::G * yp;                 // row step between a lane's symbols
                for (int r = 0; r < S; r += 2) {
                    const C2 h0 = Hs[r * UT + u];
                    const C2 h1 = Hs[(r + 1) * UT + u];
#pragma unroll
                    for (int j = 0; j < K::NN; ++j) {
                        C2 a, b;
                        ld2(&yr[j * js + r], a, b);
                        cmacc(acc[j], h0, a);
                        cmacc(acc[j], h1, b);
                    }
                }
                if (n0 + K::NCH >= N) {
                    __syncwarp();
                    if (prefetch) issue(nw);
                }
                put_vec<UT>(Vb, u, g, acc);
                __syncwarp();
                matvec<UT>(R, Vb, g, z);
                __syncwarp();
#pragma unroll
                for (int j = 0; j < K::NN; ++j) Yr[(g + K::G * j) * UT + u] = z[j];
            }

            // Consensus and (E2) prox for the owned symbols, s broadcast.
            // w_c = z_c + lambda_c is published, s = prox(sum_c w_c) returned.
            auto consensus = [&](const C2 (&zz)[K::NN], const C2 (&ll)[K::NN], C2 (&s)[K::NN]) {
                C2 *mine = contrib + warp * E;
#pragma unroll
                for (int j = 0; j < K::NN; ++j) mine[(g + K::G * j) * UT + u] = cadd(zz[j], ll[j]);
                __syncthreads();
                for (int base = c * 32; base < nvu; base += C * 32) {
                    const int e = base + lane;
                    if (e < nvu) {
                        C2 a = consensus_sum<E>(grp, e, C);
                        if (p.reg >= 2) {   // (E2-BOX); BPSK: the real segment [-r, r]
                            const float r = p.f_box_r, ic = p.f_invC;
                            a.x = clip_r(a.x * ic, r);
                            a.y = (p.reg == 2) ? clip_r(a.y * ic, r) : 0.f;
                        } else {
                            a = cscale(a, p.f_e2_scale);
                        }
                        sb[e] = a;
                    }
                }
                __syncthreads();
#pragma unroll
                for (int j = 0; j < K::NN; ++j) s[j] = sb[(g + K::G * j) * UT + u];
            };

            // Init: lambda_c = 0, z_c = y_c^reg, s = prox(sum_c z_c).
#pragma unroll
            for (int j = 0; j < K::NN; ++j) lam[j] = make_float2(0.f, 0.f);
            consensus(z, lam, s);
            const float gam = p.f_gamma, rho = p.f_rho;
            for (int t = 2; t <= p.T; ++t) {
                C2 d[K::NN];
#pragma unroll
                for (int j = 0; j < K::NN; ++j) {
                    lam[j].x = fmaf(gam, z[j].x - s[j].x, lam[j].x);
                    lam[j].y = fmaf(gam, z[j].y - s[j].y, lam[j].y);
                    d[j] = cscale(csub(s[j], lam[j]), rho);
                }
                put_vec<UT>(Vb, u, g, d);
                __syncwarp();
                matvec<UT>(R, Vb, g, z);
                __syncwarp();
#pragma unroll
                for (int j = 0; j < K::NN; ++j) z[j] = cadd(z[j], Yr[(g + K::G * j) * UT + u]);
                consensus(z, lam, s);
            }

            // Output s^(T) and its label, written by the warp that formed it.
            if (valid) {
                C2 *xo = reinterpret_cast<C2 *>(p.out);
                for (int base = c * 32; base < nvu; base += C * 32) {
                    const int e = base + lane;
                    if (e < nvu) {
                        const C2 sv = sb[e];
                        const size_t o = ((size_t)w * N + n0) * UT + e;
                        xo[o] = sv;
                        if (p.labels != nullptr)
                            p.labels[o] = qam_label<float>(sv.x, sv.y, p.f_qam_inv_a, p.qam_L, p.qam_half);
                    }
                }
            }
        }
    }
}

}  // namespace dbp
