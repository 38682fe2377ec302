// dbp_tc8.cuh -- uplink detection for U = 8 users, FP32 inputs, with every
// dense complex product on the tensor cores and the consensus step once per
// symbol (the broadcast structure of dbp_admm.cuh / dbp_cg.cuh).
//
// Per (subcarrier, cluster) warp, Alg. 1 and Alg. 2 need the same three
// products with K = 2S (antenna rows) or 2U (users) real contraction terms:
// the Gram H_c^H H_c, the matched filter H_c^H y_c for 16 symbol slots, and
// per iteration the operator (B_c^{-1} for Alg. 1, G_c for Alg. 2) times the
// cluster's 8 x 16 state.  Each is a 16 x 16 real product (rows: the real
// parts of the 8 outputs over their imaginary parts) computed as three
// mma.sync.m16n8k8 TF32 products per k-step (split operands, FP32 accuracy;
// the split is in dbp_tma.cuh, the real embedding in dbp_mma8.cuh).  Lane
// (g, t) = (lane / 4, lane % 4) holds user g of symbols
// n = 8 (q >> 1) + 2t + (q & 1), q = 0..3, of the accumulator.
//
// Consensus: warps publish their contributions, warp c reduces the units c,
// c + C, ... of 32 (symbol, user) entries and forms the centralized step (the
// (E2) prox of Alg. 1; the e, alpha, x, r, beta, p updates of Alg. 2), and s
// or p comes back through shared memory.  For CG the B fragments of p are
// read straight from that broadcast buffer.
//
// Shared memory per warp: H_c (h_rows x 8), receive rows (y_rows x yp), and
// for ADMM y_c^reg in the accumulator layout.
// After the warps: contrib[nwarps][CE] | ADMM: s[P][CE] | CG: p[P][CE],
// r[P][E], x[P][E], rr[P][E] | mbarrier[nwarps].  contrib and s rows have
// PITCH complex per symbol, p rows VP; the ADMM transpose buffer is the
// warp's own contrib slot.
#pragma once

#include "dbp_mma8.cuh"
#include "dbp_cg.cuh"

namespace dbp {

struct Tc8 {
    static constexpr int E = 128;      // 16 symbol slots x 8 users
    static constexpr int PITCH = 12;   // complex per symbol row in contrib and s
    static constexpr int CE = 16 * PITCH;
    static constexpr int VP = 10;      // transpose buffer and CG p pitch (complex):
                                       // conflict-free B fragment loads
};

// entry e = 8 n + u of a 16-symbol pass -> padded shared-memory index
template <int PITCH> __device__ __forceinline__ int tc8_idx(int e) { return (e >> 3) * PITCH + (e & 7); }

template <int ALG> __host__ __device__ constexpr size_t tc8_cta_bytes(int nwarps, int P) {
    return (size_t)nwarps * Tc8::CE * 8 +
           ((ALG == ALG_ADMM_UL) ? (size_t)P * Tc8::CE * 8 : (size_t)P * (Tc8::CE * 8 + Tc8::E * (8 + 8 + 4))) +
           (size_t)nwarps * 8;
}

// Operator (A fragments, hi and lo, for the k-steps of users 0-3 and 4-7)
// times a state whose complex entry (n, k) sits at src[n * PITCH + k] in
// shared memory; the result lands in the accumulator layout.
template <int PITCH>
__device__ __forceinline__ void tc8_apply(const uint32_t (&oh)[2][4], const uint32_t (&ol)[2][4], const float2 *src,
                                          int g, int t, float2 (&out)[4]) {
    const float *sf = reinterpret_cast<const float *>(src) + (g * PITCH + (t >> 1)) * 2 + (t & 1);
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const float b0 = sf[(8 * nt * PITCH + 4 * ks) * 2];
            const float b1 = sf[(8 * nt * PITCH + 4 * ks + 2) * 2];
            uint32_t bh0, bl0, bh1, bl1;
            split3(b0, bh0, bl0);
            split3(b1, bh1, bl1);
            mma3(acc[nt], oh[ks], ol[ks], bh0, bh1, bl0, bl1);
        }
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        out[2 * nt] = make_float2(acc[nt][0], acc[nt][2]);
        out[2 * nt + 1] = make_float2(acc[nt][1], acc[nt][3]);
    }
}

// Sum of the C contributions of one entry (stride CE), in cluster order; C = 8
// unrolled.
template <int CE>
__device__ __forceinline__ float2 tc8_sum(const float2 *grp, int idx, int C) {
    if (C == 8) {
        const float2 *q = grp + idx;
        float2 a = q[0];
#pragma unroll
        for (int cc = 1; cc < 8; ++cc) {
            a.x += q[cc * CE].x;
            a.y += q[cc * CE].y;
        }
        return a;
    }
    return consensus_sum<CE>(grp, idx, C);
}

template <int ALG>
__global__ void __launch_bounds__(512, 2) dbp_tc8_kernel(const FusedParams p) {
    using C2 = float2;
    constexpr int E = Tc8::E, CE = Tc8::CE, VP = Tc8::VP, PITCH = Tc8::PITCH;
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int C = p.C, P = p.P, S = p.S, N = p.N, B = p.B, W = p.W;
    const int pl = warp / C, c = warp - pl * C;
    const int g = lane >> 2, t = lane & 3;
    const int yp = p.yp;

    unsigned char *wb = smem_raw + (size_t)warp * p.warp_bytes;
    const C2 *Hs = reinterpret_cast<const C2 *>(wb);
    const float *Yf = reinterpret_cast<const float *>(wb + p.off_y0);
    C2 *Yr = reinterpret_cast<C2 *>(wb + p.off_g);            // ADMM: y_c^reg [4][32]
    C2 *contrib = reinterpret_cast<C2 *>(smem_raw + (size_t)nwarps * p.warp_bytes);   // [nwarps][CE]
    // ADMM transpose buffer [16][VP]: this warp's contribution slot, free
    // between the consensus rounds
    C2 *Vs = contrib + warp * CE;
    C2 *bc = contrib + nwarps * CE + pl * CE;                 // broadcast s or p of this subcarrier
    C2 *rb = contrib + nwarps * CE + P * CE + pl * E;         // CG: r
    C2 *xb = rb + P * E;                                      // CG: x
    float *rrb = reinterpret_cast<float *>(contrib + nwarps * CE + P * CE + 2 * P * E) + pl * E;
    unsigned char *tail = smem_raw + (size_t)nwarps * p.warp_bytes +
                          ((ALG == ALG_ADMM_UL) ? ((size_t)nwarps * CE + (size_t)P * CE) * 8
                                                : ((size_t)nwarps * CE + (size_t)P * CE + 2 * (size_t)P * E) * 8 +
                                                      (size_t)P * E * 4);
    uint64_t *bar = reinterpret_cast<uint64_t *>(tail) + warp;
    const C2 *grp = contrib + pl * C * CE;

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
        const uint32_t hbytes = (uint32_t)(S * 8 * 8);
        const uint32_t ybytes = (uint32_t)(S * 8);
        fence_proxy_async();
        if (lane == 0) mbar_arrive_expect_tx(bar, hbytes + (uint32_t)N * ybytes + p.starve_bytes);
        __syncwarp();
        if (lane == 0) bulk_g2s(wb, Hg + ((size_t)w * B + (size_t)c * S) * 8, hbytes, bar);
        for (int n = lane; n < N; n += 32)
            bulk_g2s(wb + p.off_y0 + (size_t)n * yp * 8, Yg + ((size_t)w * N + n) * B + (size_t)c * S, ybytes, bar);
    };
    // symbol of accumulator entry q of this lane (within a 16-symbol pass)
    auto nof = [&](int q) { return 8 * (q >> 1) + 2 * t + (q & 1); };

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
        const int npass = (N + 15) / 16;
        const bool need_gram = (p.factor_mode != 2);

        // ---- Gram (and the matched filter of a single pass) ----
        float gacc[4] = {0.f, 0.f, 0.f, 0.f};
        float macc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
        if (need_gram || npass == 1) {
            for (int s0 = 0; s0 < p.h_rows; s0 += 4) {
                float a[4];
                hh_frag(Hs, s0, g, t, a);
                uint32_t ah[4], al[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) split3(a[i], ah[i], al[i]);
                if (need_gram) mma3(gacc, ah, al, ah[0], ah[2], al[0], al[2]);   // B = H_c: same values
                if (npass == 1) {
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) {
                        const float *yr = Yf + ((8 * nt + g) * yp + s0 + (t >> 1)) * 2 + (t & 1);
                        uint32_t bh0, bl0, bh1, bl1;
                        split3(yr[0], bh0, bl0);
                        split3(yr[4], bh1, bl1);
                        mma3(macc[nt], ah, al, bh0, bh1, bl0, bl1);
                    }
                }
            }
        }

        // ---- Operator: lane (g, t) holds entries (g, 2t), (g, 2t + 1) ----
        C2 e0, e1;
        C2 *frow = (p.factor != nullptr && valid) ? p.factor + (((size_t)w * C + c) * 8 + g) * 8 + 2 * t : nullptr;
        if (!need_gram) {
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            if (frow != nullptr) q = *reinterpret_cast<const float4 *>(frow);
            e0 = make_float2(q.x, q.y);
            e1 = make_float2(q.z, q.w);
        } else {
            e0 = make_float2(gacc[0], gacc[2]);
            e1 = make_float2(gacc[1], gacc[3]);
            if (ALG == ALG_ADMM_UL) {
                const float delta = p.f_delta;
                if (2 * t == g) e0.x += delta;
                if (2 * t + 1 == g) e1.x += delta;
                float dmax = (2 * t == g) ? e0.x : ((2 * t + 1 == g) ? e1.x : 0.f);
                dmax = warp_redux_max(dmax);
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
        if (npass == 1) {
            // H_c and y_c are no longer read: fetch the next subcarrier.
            __syncwarp();
            if (prefetch) issue(nw);
        }

        // A fragments (hi, lo) of the operator for the k-steps of users 0-3
        // and 4-7: lane (g, t) needs Op[g][4 ks + t/2] and Op[g][4 ks + 2 + t/2].
        uint32_t oh[2][4], ol[2][4];
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int srcl = 4 * g + 2 * ks + half;
                C2 v0, v1;
                v0.x = __shfl_sync(0xffffffffu, e0.x, srcl);
                v0.y = __shfl_sync(0xffffffffu, e0.y, srcl);
                v1.x = __shfl_sync(0xffffffffu, e1.x, srcl);
                v1.y = __shfl_sync(0xffffffffu, e1.y, srcl);
                const C2 o = (t >> 1) ? v1 : v0;
                const bool odd = t & 1;
                const float are = odd ? -o.y : o.x;
                const float aim = odd ? o.x : o.y;
                split3(are, oh[ks][2 * half], ol[ks][2 * half]);
                split3(aim, oh[ks][2 * half + 1], ol[ks][2 * half + 1]);
            }
        }

        // Operator times a state whose complex entry (n, k) sits at
        // src[n * pitch + k] in shared memory -> accumulator layout.
        for (int pass = 0; pass < npass; ++pass) {
            const int n0 = 16 * pass;
            const int nvu = min(16, N - n0) * 8;            // valid (symbol, user) entries
            C2 m[4];
            if (npass == 1) {
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
                        const float *yr = Yf + ((n0 + 8 * nt + g) * yp + s0 + (t >> 1)) * 2 + (t & 1);
                        uint32_t bh0, bl0, bh1, bl1;
                        split3(yr[0], bh0, bl0);
                        split3(yr[4], bh1, bl1);
                        mma3(ma[nt], ah, al, bh0, bh1, bl0, bl1);
                    }
                }
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    m[2 * nt] = make_float2(ma[nt][0], ma[nt][2]);
                    m[2 * nt + 1] = make_float2(ma[nt][1], ma[nt][3]);
                }
                if (pass == npass - 1) {
                    __syncwarp();
                    if (prefetch) issue(nw);
                }
            }
            C2 *mine = contrib + warp * CE;

            if (ALG == ALG_ADMM_UL) {
                // y_c^reg = B_c^{-1} m_c (transpose through Vs into B fragments)
                C2 z[4], lam[4], s[4];
                auto apply_regs = [&](const C2 (&x)[4], C2 (&out)[4]) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) Vs[nof(q) * VP + g] = x[q];
                    __syncwarp();
                    tc8_apply<VP>(oh, ol, Vs, g, t, out);
                    __syncwarp();
                };
                apply_regs(m, z);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    Yr[q * 32 + lane] = z[q];
                    lam[q] = make_float2(0.f, 0.f);
                }
                // symbol slots past N read s = 0 (the owners write only valid slots)
                for (int e = nvu + lane; e < E; e += 32) bc[tc8_idx<PITCH>(e)] = make_float2(0.f, 0.f);
                // publish w_c = z_c + lambda_c, reduce and prox the owned
                // entries, read s back
                auto consensus = [&]() {
#pragma unroll
                    for (int q = 0; q < 4; ++q) mine[nof(q) * PITCH + g] = cadd(z[q], lam[q]);
                    __syncthreads();
                    for (int base = c * 32; base < nvu; base += C * 32) {
                        const int e = base + lane;            // < E: in the buffers
                        C2 a = tc8_sum<CE>(grp, tc8_idx<PITCH>(e), C);
                        if (p.reg >= 2) {   // (E2-BOX); BPSK: the real segment [-r, r]
                            const float r = p.f_box_r, ic = p.f_invC;
                            a.x = clip_r(a.x * ic, r);
                            a.y = (p.reg == 2) ? clip_r(a.y * ic, r) : 0.f;
                        } else {
                            a = cscale(a, p.f_e2_scale);
                        }
                        if (e < nvu) bc[tc8_idx<PITCH>(e)] = a;
                    }
                    __syncthreads();
#pragma unroll
                    for (int q = 0; q < 4; ++q) s[q] = bc[nof(q) * PITCH + g];
                };
                consensus();
                const float gam = p.f_gamma, rho = p.f_rho;
                for (int it = 2; it <= p.T; ++it) {
                    C2 d[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        lam[q].x = fmaf(gam, z[q].x - s[q].x, lam[q].x);
                        lam[q].y = fmaf(gam, z[q].y - s[q].y, lam[q].y);
                        d[q] = cscale(csub(s[q], lam[q]), rho);
                    }
                    apply_regs(d, z);
#pragma unroll
                    for (int q = 0; q < 4; ++q) z[q] = cadd(z[q], Yr[q * 32 + lane]);
                    consensus();
                }
                // output s^(T) and its label from the owning warp
                if (valid) {
                    C2 *xo = reinterpret_cast<C2 *>(p.out);
                    for (int base = c * 32; base < nvu; base += C * 32) {
                        const int e = base + lane;
                        if (e < nvu) {
                            const C2 sv = bc[tc8_idx<PITCH>(e)];
                            const size_t o = ((size_t)w * N + n0) * 8 + e;
                            xo[o] = sv;
                            if (p.labels != nullptr)
                                p.labels[o] = qam_label<float>(sv.x, sv.y, p.f_qam_inv_a, p.qam_L, p.qam_half);
                        }
                    }
                }
            } else {
                // CG: y_MRC = sum_c m_c; r = p = y_MRC, x = 0
#pragma unroll
                for (int q = 0; q < 4; ++q) mine[nof(q) * PITCH + g] = m[q];
                __syncthreads();
                for (int base = c * 32; base < nvu; base += C * 32) {
                    const int e = base + lane;
                    const bool ok = e < nvu;
                    C2 y = make_float2(0.f, 0.f);
                    if (ok) y = tc8_sum<CE>(grp, tc8_idx<PITCH>(e), C);
                    const float rr = group_sum<8>(y.x * y.x + y.y * y.y);
                    if (ok) {
                        bc[tc8_idx<VP>(e)] = y;
                        rb[e] = y;
                        xb[e] = make_float2(0.f, 0.f);
                        rrb[e] = rr;
                    }
                }
                if (nvu < E) {
                    // symbol slots past N: p = 0 keeps the products finite
                    for (int e = nvu + lane; e < E; e += 32) bc[tc8_idx<VP>(e)] = make_float2(0.f, 0.f);
                }
                __syncthreads();
                const float rcg = p.f_rho_cg;
                for (int it = 1; it <= p.T; ++it) {
                    C2 wc[4];
                    tc8_apply<VP>(oh, ol, bc, g, t, wc);                 // w_c = G_c p
#pragma unroll
                    for (int q = 0; q < 4; ++q) mine[nof(q) * PITCH + g] = wc[q];
                    __syncthreads();
                    // e < E always (base < nvu <= E): the loads stay in the
                    // buffers; entries past N compute on stale values that no
                    // valid symbol group reads, and only valid entries store.
                    for (int base = c * 32; base < nvu; base += C * 32) {
                        const int e = base + lane;
                        const bool ok = e < nvu;
                        const int ie = tc8_idx<VP>(e);
                        const C2 ws = tc8_sum<CE>(grp, tc8_idx<PITCH>(e), C);
                        C2 pv = bc[ie], rv = rb[e], xv = xb[e];
                        const float rr = rrb[e];
                        C2 ev;
                        ev.x = fmaf(rcg, pv.x, ws.x);
                        ev.y = fmaf(rcg, pv.y, ws.y);
                        const float pe = group_sum<8>(pv.x * ev.x + pv.y * ev.y);
                        const bool go = !(rr < 0.f) && rr != 0.f && pe != 0.f;
                        const float alpha = go ? __fdiv_rn(rr, pe) : 0.f;
                        // a stopped symbol (alpha = 0) keeps x and r
                        xv.x = fmaf(alpha, pv.x, xv.x);
                        xv.y = fmaf(alpha, pv.y, xv.y);
                        rv.x = fmaf(-alpha, ev.x, rv.x);
                        rv.y = fmaf(-alpha, ev.y, rv.y);
                        const float rn = group_sum<8>(rv.x * rv.x + rv.y * rv.y);
                        const float beta = go ? __fdiv_rn(rn, rr) : 0.f;
                        if (go) {
                            pv.x = fmaf(beta, pv.x, rv.x);
                            pv.y = fmaf(beta, pv.y, rv.y);
                        }
                        if (ok) {
                            bc[ie] = pv;
                            rb[e] = rv;
                            xb[e] = xv;
                            rrb[e] = go ? rn : -1.f;
                        }
                    }
                    __syncthreads();
                }
                if (valid) {
                    C2 *xo = reinterpret_cast<C2 *>(p.out);
                    for (int base = c * 32; base < nvu; base += C * 32) {
                        const int e = base + lane;
                        if (e < nvu) {
                            const C2 xv = xb[e];
                            const size_t o = ((size_t)w * N + n0) * 8 + e;
                            xo[o] = xv;
                            if (p.labels != nullptr)
                                p.labels[o] = qam_label<float>(xv.x, xv.y, p.f_qam_inv_a, p.qam_L, p.qam_half);
                        }
                    }
                }
            }
        }
    }
}

}  // namespace dbp
