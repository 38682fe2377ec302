// dbp_cg.cuh -- decentralized CG uplink detection (Alg. 2, Sec. III-D) with
// the consensus vector reduced once and the CG vector updates done once per
// subcarrier, then p^(t) broadcast to the clusters.
//
// Sec. III-D gives two placements for the updates of e, x, r and p: on the
// centralized unit after the consensus w = sum_c w_c, followed by a broadcast
// of p^(t) to every cluster; or in every cluster on its own copy after a
// broadcast of w.  The bulk-copy kernel (dbp_tma.cuh) follows the second;
// this kernel follows the first.  On one GPU the "centralized unit" for a
// subcarrier is spread over its C cluster warps in units of 32 (symbol, user)
// entries: warp c reduces and updates the units c, c + C, ... of each chunk,
// so each update runs once instead of C times and on full warps.  Per (subcarrier, cluster) the local work is what
// Alg. 2 assigns to cluster c: the matched filter H_c^H y_c and, per
// iteration, w_c = G_c p with the local Gram G_c = H_c^H H_c (the footnote to
// Alg. 2).
//
// Layout: one warp per (subcarrier, cluster), P subcarriers x C warps per
// CTA, persistent CTAs.  Each warp owns one staging buffer for its cluster
// block H_c (S x U, dense) and its receive rows (N x S); the copies for the
// next subcarrier are issued as soon as the matched filter of the last chunk
// has read the buffer, so they overlap the CG iterations.
//
// Shared memory after the warps' staging regions (host computes the same):
//   contrib[nwarps][E] float2 | p, r, x [P][E] float2 | rr [P][E] float |
//   mbarrier[nwarps]
#pragma once

#include "dbp_fused.cuh"
#include "dbp_tma.cuh"

namespace dbp {

template <int UT> struct CgCfg {
    using K = Tile<UT>;
    static constexpr int E = K::NCH * UT;   // entries (symbol, user) per chunk
};

// Consensus sum over the C cluster contributions of entry e (stride E in
// shared memory), in cluster order.
template <int E>
__device__ __forceinline__ float2 consensus_sum(const float2 *grp, int e, int C) {
    float2 a = make_float2(0.f, 0.f);
    const float2 *q = grp + e;
    int cc = 0;
    for (; cc + 4 <= C; cc += 4, q += 4 * E) {
        const float2 t0 = q[0], t1 = q[E], t2 = q[2 * E], t3 = q[3 * E];
        a.x += t0.x; a.y += t0.y;
        a.x += t1.x; a.y += t1.y;
        a.x += t2.x; a.y += t2.y;
        a.x += t3.x; a.y += t3.y;
    }
    for (; cc < C; ++cc, q += E) {
        a.x += q[0].x;
        a.y += q[0].y;
    }
    return a;
}

template <int UT> __host__ __device__ constexpr size_t cg_cta_bytes(int nwarps, int P) {
    return (size_t)nwarps * CgCfg<UT>::E * 8 + (size_t)P * CgCfg<UT>::E * (3 * 8 + 4) + (size_t)nwarps * 8;
}

template <int UT>
__global__ void __launch_bounds__(512, (UT <= 8) ? 2 : 1) dbp_cg_kernel(const FusedParams p) {
    using C2 = float2;
    using K = Tile<UT>;
    constexpr int E = CgCfg<UT>::E;
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
    C2 *contrib = reinterpret_cast<C2 *>(smem_raw + (size_t)nwarps * p.warp_bytes);   // [nwarps][E]
    C2 *pb = contrib + (size_t)nwarps * E + (size_t)pl * E;                             // this subcarrier's p
    C2 *rb = pb + (size_t)P * E;
    C2 *xb = rb + (size_t)P * E;
    float *rrb = reinterpret_cast<float *>(contrib + (size_t)nwarps * E + 3 * (size_t)P * E) + (size_t)pl * E;
    uint64_t *bar = reinterpret_cast<uint64_t *>(reinterpret_cast<float *>(contrib + (size_t)nwarps * E +
                                                                           3 * (size_t)P * E) +
                                                 (size_t)P * E) + warp;
    const C2 *grp = contrib + pl * C * E;           // the C contributions of this subcarrier

    // Zero the staging region (receive rows past N stay zero), set up the
    // mbarrier.
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

    const float rcg = p.f_rho_cg;
    for (; tile < p.tiles; tile += gridDim.x) {
        const int w = tile * P + pl;
        const bool valid = (w < W);
        const int nw = (tile + (int)gridDim.x) * P + pl;
        const bool prefetch = (tile + (int)gridDim.x < p.tiles) && nw < W;
        if (valid) {
            mbar_wait_bounded(bar, phase, p.status, p.wait_iters);
            phase ^= 1u;
        }

        // ---- Local Gram G_c = H_c^H H_c (+ delta I), row u per lane ----
        C2 R[UT];
        C2 *frow = (p.factor != nullptr && valid) ? p.factor + (((size_t)w * C + c) * UT + u) * UT : nullptr;
        if (p.factor_mode == 2) {
            // resident Gram of this coherence block
#pragma unroll
            for (int v = 0; v < UT; v += 2) {
                float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                if (frow != nullptr) q = *reinterpret_cast<const float4 *>(&frow[v]);
                R[v] = make_float2(q.x, q.y);
                R[v + 1] = make_float2(q.z, q.w);
            }
        } else {
#pragma unroll
            for (int v = 0; v < UT; ++v) R[v] = make_float2(0.f, 0.f);
            for (int r = g; r < S; r += K::G) {
                const C2 hu = Hs[r * UT + u];
#pragma unroll
                for (int v = 0; v < UT; v += 2) {
                    C2 a, b;
                    ld2(&Hs[r * UT + v], a, b);
                    cmacc(R[v], hu, a);
                    cmacc(R[v + 1], hu, b);
                }
            }
#pragma unroll
            for (int m = UT; m < 32; m <<= 1) {
#pragma unroll
                for (int v = 0; v < UT; ++v) {
                    R[v].x += shfl_x(R[v].x, m);
                    R[v].y += shfl_x(R[v].y, m);
                }
            }
            const float delta = p.f_delta;
#pragma unroll
            for (int v = 0; v < UT; ++v)
                if (v == u) R[v].x += delta;
            if (p.factor_mode == 1 && frow != nullptr && g == 0) {
#pragma unroll
                for (int v = 0; v < UT; v += 2)
                    *reinterpret_cast<float4 *>(&frow[v]) = make_float4(R[v].x, R[v].y, R[v + 1].x, R[v + 1].y);
            }
        }

        for (int n0 = 0; n0 < N; n0 += K::NCH) {
            const int nv = min(K::NCH, N - n0);          // symbols in this chunk
            const int nvu = nv * UT;                      // (symbol, user) entries in this chunk

            // Matched filter m_c = H_c^H y_c for the chunk, published for the
            // consensus y_MRC = sum_c m_c (Alg. 2, preprocessing).
            {
                C2 acc[K::NN];
#pragma unroll
                for (int j = 0; j < K::NN; ++j) acc[j] = make_float2(0.f, 0.f);
                const C2 *yr = Ys + (n0 + g) * yp;
                const int js = K::G * yp;                 // row step between a lane's symbols
#pragma unroll 2
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
                C2 *mine = contrib + warp * E;
#pragma unroll
                for (int j = 0; j < K::NN; ++j) mine[(g + K::G * j) * UT + u] = acc[j];
            }
            if (n0 + K::NCH >= N) {
                // Last read of the staging buffer: fetch the next subcarrier.
                __syncwarp();
                if (prefetch) issue(nw);
            }
            __syncthreads();

            // Init (Alg. 2): r = y_MRC, p = r, x = 0.
            for (int base = c * 32; base < nvu; base += C * 32) {
                const int e = base + lane;
                const bool ok = e < nvu;
                C2 y = make_float2(0.f, 0.f);
                if (ok) y = consensus_sum<E>(grp, e, C);
                const float rr = group_sum<UT>(y.x * y.x + y.y * y.y);
                if (ok) {
                    pb[e] = y;
                    rb[e] = y;
                    xb[e] = make_float2(0.f, 0.f);
                    rrb[e] = rr;
                }
            }
            __syncthreads();

            for (int t = 1; t <= p.T; ++t) {
                // Decentralized: w_c = G_c p^(t-1) in every cluster.
                {
                    C2 wc[K::NN];
#pragma unroll
                    for (int j = 0; j < K::NN; ++j) {
                        const C2 *pv = pb + (g + K::G * j) * UT;
                        wc[j] = make_float2(0.f, 0.f);
#pragma unroll
                        for (int v = 0; v < UT; v += 2) {
                            C2 a, b;
                            ld2(&pv[v], a, b);
                            cmac(wc[j], R[v], a);
                            cmac(wc[j], R[v + 1], b);
                        }
                    }
                    C2 *mine = contrib + warp * E;
#pragma unroll
                    for (int j = 0; j < K::NN; ++j) mine[(g + K::G * j) * UT + u] = wc[j];
                }
                __syncthreads();
                // Centralized, once per symbol: w = sum_c w_c, then the CG
                // updates of e, alpha, x, r, beta and p; p^(t) is broadcast
                // through shared memory.  A symbol whose ||r||^2 or Re(p^H e)
                // is zero stops (its iterate is final); rr < 0 marks it.
                for (int base = c * 32; base < nvu; base += C * 32) {
                    const int e = base + lane;
                    const bool ok = e < nvu;
                    C2 ws = make_float2(0.f, 0.f), pv = ws, rv = ws, xv = ws;
                    float rr = -1.f;
                    if (ok) {
                        ws = consensus_sum<E>(grp, e, C);
                        pv = pb[e];
                        rv = rb[e];
                        xv = xb[e];
                        rr = rrb[e];
                    }
                    C2 ev;
                    ev.x = fmaf(rcg, pv.x, ws.x);
                    ev.y = fmaf(rcg, pv.y, ws.y);
                    const float pe = group_sum<UT>(pv.x * ev.x + pv.y * ev.y);
                    const bool go = !(rr < 0.f) && rr != 0.f && pe != 0.f;
                    const float alpha = go ? __fdiv_rn(rr, pe) : 0.f;
                    if (go) {
                        xv.x = fmaf(alpha, pv.x, xv.x);
                        xv.y = fmaf(alpha, pv.y, xv.y);
                        rv.x = fmaf(-alpha, ev.x, rv.x);
                        rv.y = fmaf(-alpha, ev.y, rv.y);
                    }
                    const float rn = group_sum<UT>(rv.x * rv.x + rv.y * rv.y);
                    if (ok) {
                        if (go) {
                            const float beta = __fdiv_rn(rn, rr);
                            pv.x = fmaf(beta, pv.x, rv.x);
                            pv.y = fmaf(beta, pv.y, rv.y);
                            pb[e] = pv;
                            rb[e] = rv;
                            xb[e] = xv;
                            rrb[e] = rn;
                        } else {
                            rrb[e] = -1.f;
                        }
                    }
                }
                __syncthreads();
            }

            // Output x^(T) and its label, written by the updating warp.
            if (valid) {
                C2 *xo = reinterpret_cast<C2 *>(p.out);
                for (int base = c * 32; base < nvu; base += C * 32) {
                    const int e = base + lane;
                    if (e < nvu) {
                        const C2 xv = xb[e];
                        const size_t o = ((size_t)w * N + n0) * UT + e;
                        xo[o] = xv;
                        if (p.labels != nullptr)
                            p.labels[o] = qam_label<float>(xv.x, xv.y, p.f_qam_inv_a, p.qam_L, p.qam_half);
                    }
                }
            }
        }
    }
}

}  // namespace dbp
