// dbp_tcdl.cuh -- decentralized ADMM downlink beamforming (Alg. 3) for U = 16
// users with FP32 inputs, every dense complex product on the tensor cores.
//
// Per (subcarrier, cluster) warp, in the U x U form of Alg. 3 with
// H^d_c = (H_c)^T (reciprocity):
//   * B_c = H^d_c H^{dH}_c + rho^{-1} I = conj(H_c^H H_c) + rho^{-1} I: the
//     Gram on the tensor cores, its inverse by the column-split Gauss-Jordan
//     of dbp_admm.cuh (lane (u, g) holds columns 8g..8g+7 of row u);
//   * per iteration m_c = H^d_c x_c = v_c - rho^{-1} B_c^{-1} v_c with
//     v_c = z_c + lambda_c (x_c = H^{dH}_c B_c^{-1} v_c, push-through), the
//     product B_c^{-1} v_c for 16 symbol slots being a 32 x 32 x 16 real
//     product (2 m-tiles of 8 users, real parts over imaginary parts, 2
//     k-steps of 8 complex entries, 2 n-tiles of 8 symbols);
//   * the output x_c = H^{dH}_c B_c^{-1} v_c, an (S x 16) x (16 x 16) product.
// Every product is mma.sync.m16n8k16 with FP16 operands and FP32
// accumulators, three per k-step: each FP32 operand is scaled by a power of
// two (its warp's largest magnitude into [2^13, 2^14)), split into FP16 hi
// and lo halves, and the products lo hi, hi lo, hi hi are accumulated in
// that order (small terms first); the scales are exact and are divided out.
// In a k-step of the complex embedding, lane (g, t) holds one complex entry
// per register: (re, im) for a real row and (-im, re) for the imaginary
// row below it, so one hi / lo split serves both rows.
// The consensus w = sum_c (m_c - lambda_c) and (s - w)/C run once per symbol:
// warp c reduces the units c, c + C, ... of 32 (symbol, user) entries and
// broadcasts d = (s - w)/C, scaled by max{0, 1 - eps/||s - w||} for eps > 0
// (Lemma 2); every cluster then forms z_c = w_c + d and its dual update
// (Alg. 3, the consensus step of Sec. IV-B).
//
// Lane (g, t) = (lane / 4, lane % 4) holds, for m-tile mt and n-tile nt, user
// 8 mt + g of symbols 8 nt + 2t and 8 nt + 2t + 1 (8 complex state entries).
//
// Shared memory per warp: two H_c buffers (S x 16, double-buffered bulk
// copies), the state v [16][VPD] and B_c^{-1} [16][QP].  After the warps:
// contrib[nwarps][CE] | d[P][CE] | s[P][CE] | mbarrier[nwarps][2].
#pragma once

#include "dbp_mma8.cuh"
#include "dbp_admm.cuh"

namespace dbp {

struct TcDl {
    static constexpr int U = 16;
    static constexpr int NS = 16;            // symbol slots per pass
    static constexpr int VPD = 20;           // state pitch (complex), 4 mod 16: conflict-free B fragment loads
    static constexpr int QP = 18;            // operator pitch (complex)
    static constexpr int CP = 20;            // contrib / broadcast pitch (complex)
    static constexpr int CE = NS * CP;
};

__host__ __device__ constexpr size_t tcdl_cta_bytes(int nwarps, int P) {
    return (size_t)nwarps * TcDl::CE * 8 + 2 * (size_t)P * TcDl::CE * 8 + (size_t)nwarps * 16;
}

// Power-of-two exponent e with m 2^e in [2^13, 2^14) (0 for 0 or a
// non-finite m), clamped to [-60, 60] so that the sum of two exponents is a
// normal power of two: FP16 operands keep 11 significant bits in hi and 11
// more in lo for every entry within 2^-17 of the largest.
__device__ __forceinline__ int dl16_scale_exp(float m) {
    if (!(m > 0.f) || !(m < 3.0e38f)) return 0;
    const int e = 14 - frexp_exponent(m);
    return e < -60 ? -60 : (e > 60 ? 60 : e);
}
__device__ __forceinline__ float dl16_exp2i(int e) { return __int_as_float((127 + e) << 23); }
__device__ __forceinline__ float dl16_warp_max(float m) { return warp_redux_max(m); }
__device__ __forceinline__ float cabsmax(float2 v) { return fmaxf(fabsf(v.x), fabsf(v.y)); }

// FP16 hi / lo halves of (re, im) scaled by sc, packed as f16x2 (re in the
// low half): hi = fp16(x sc), lo = fp16(x sc - hi).
__device__ __forceinline__ void dl16_split(float re, float im, float sc, uint32_t &hi, uint32_t &lo) {
    const float a = re * sc, b = im * sc;
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}
// (re, im) -> (-im, re) on a packed f16x2 (exact; the halves of a negated
// value are the negated halves).
__device__ __forceinline__ uint32_t dl16_rot(uint32_t x) { return __byte_perm(x, 0u, 0x1032) ^ 0x00008000u; }

__device__ __forceinline__ void mma_f16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// D += A B over K = 16 from hi / lo halves: lo hi, hi lo, then hi hi.
__device__ __forceinline__ void mma3h(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4], uint32_t bh0,
                                      uint32_t bh1, uint32_t bl0, uint32_t bl1) {
    mma_f16(d, al, bh0, bh1);
    mma_f16(d, ah, bl0, bl1);
    mma_f16(d, ah, bh0, bh1);
}
// A fragment of one k-step from two complex entries x0 (column 2t, 2t + 1 of
// the real embedding) and x1 (the same, 8 further), given as the real row's
// (re, im) coefficients: registers 1 and 3 are the imaginary row's.
__device__ __forceinline__ void dl16_afrag(float2 x0, float2 x1, float sc, uint32_t (&ah)[4], uint32_t (&al)[4]) {
    dl16_split(x0.x, x0.y, sc, ah[0], al[0]);
    dl16_split(x1.x, x1.y, sc, ah[2], al[2]);
    ah[1] = dl16_rot(ah[0]);
    al[1] = dl16_rot(al[0]);
    ah[3] = dl16_rot(ah[2]);
    al[3] = dl16_rot(al[2]);
}

// Position of entry (n, u) of a 16-symbol state or consensus buffer with
// rows `pitch` (20) entries apart: columns XOR 4 on rows 4-7 and 12-15.  The
// accumulator layout's 8-byte accesses (lane (g, t): rows 2t + q, column g)
// and the B fragments' (row g, columns t, t + 4) then both hit 16 distinct
// bank pairs per half-warp; unswizzled, rows n and n + 4 of the first met
// in the same banks (2-way conflicts).
__device__ __forceinline__ int sw20(int n, int u, int pitch) { return n * pitch + (u ^ (((n >> 2) & 1) << 2)); }

// Scale exponent of H_c (S x 16, row pitch 16) for its FP16 split.
__device__ __forceinline__ int tcdl_h_scale(const float2 *Hs, int S, int lane) {
    float m = 0.f;
    for (int i = lane; i < S * TcDl::U; i += 32) m = fmaxf(m, cabsmax(Hs[i]));
    return dl16_scale_exp(dl16_warp_max(m));
}

// B fragments of a 16 x 16 state held as [symbol][VPD] (complex): lane (g, t)
// of n-tile nt, k-step ks takes symbol 8 nt + g, entries 8 ks + t and
// 8 ks + t + 4, split with one scale for the warp; returns the exponent.
__device__ __forceinline__ int dl16_bfrag(const float2 *Vb, int g, int t, uint32_t (&bh)[2][2][2],
                                          uint32_t (&bl)[2][2][2]) {
    float2 v[2][2][2];
    float mv = 0.f;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                v[nt][ks][hh] = Vb[sw20(8 * nt + g, 8 * ks + 4 * hh + t, TcDl::VPD)];
                mv = fmaxf(mv, cabsmax(v[nt][ks][hh]));
            }
    const int ev = dl16_scale_exp(dl16_warp_max(mv));
    const float sv = dl16_exp2i(ev);
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) dl16_split(v[nt][ks][hh].x, v[nt][ks][hh].y, sv, bh[nt][ks][hh], bl[nt][ks][hh]);
    return ev;
}

// m = Q v: Q (B_c^{-1}, scale 2^eq) as A fragments (hi, lo) [m-tile][k-step][4],
// v [16 symbols][VPD] in shared memory; result in the accumulator layout
// m[mt][nt][q] (user 8 mt + g, symbol 8 nt + 2 t + q).
__device__ __forceinline__ void tcdl_apply(const uint32_t (&qh)[2][2][4], const uint32_t (&ql)[2][2][4], int eq,
                                           const float2 *Vb, int g, int t, float2 (&m)[2][2][2]) {
    uint32_t bh[2][2][2], bl[2][2][2];
    const int ev = dl16_bfrag(Vb, g, t, bh, bl);
    float acc[2][2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[mt][nt][i] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
                mma3h(acc[mt][nt], qh[mt][ks], ql[mt][ks], bh[nt][ks][0], bh[nt][ks][1], bl[nt][ks][0], bl[nt][ks][1]);
    const float us = dl16_exp2i(-(eq + ev));
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            m[mt][nt][0] = make_float2(acc[mt][nt][0] * us, acc[mt][nt][2] * us);
            m[mt][nt][1] = make_float2(acc[mt][nt][1] * us, acc[mt][nt][3] * us);
        }
}

// Column-split Gauss-Jordan inversion of the 16 x 16 HPD matrix held as in
// gj_split<16> (lane (u, g) holds row u, columns 8 g .. 8 g + 7), with the
// pivot row and the pivot column published through shared memory instead of
// 20 shuffles per step: the two lanes of row k store its 16 entries, the
// lanes of column k's group store that column, and every lane reads back
// the row (four 16-byte broadcast loads), its multiplier and the pivot.  The
// values and the arithmetic are those of gj_split<16>, so the results are
// bit-identical.  sc: 64 complex, 16-byte aligned, two buffers used in
// turn, so one __syncwarp per step suffices.
__device__ __forceinline__ float gj_split16_s(float2 (&A)[8], int u, int g, float2 *sc) {
    float min_piv = 3.4e38f;
    float2 myinv = make_float2(1.f, 0.f);     // 1 / the pivot of row u's own step
    __syncwarp();   // every lane has loaded its row before the buffers are written
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int gk = k >> 3, ik = k & 7;
        float2 *buf = sc + (k & 1) * 32;   // [0, 16): row k; [16, 32): column k
        if (u == k) {
#pragma unroll
            for (int i = 0; i < 8; i += 2)
                *reinterpret_cast<float4 *>(&buf[8 * g + i]) = make_float4(A[i].x, A[i].y, A[i + 1].x, A[i + 1].y);
        }
        if (g == gk) buf[16 + u] = A[ik];
        __syncwarp();
        const float2 piv = buf[16 + k];
        const float2 f = buf[16 + u];
        float2 rk[8];
#pragma unroll
        for (int i = 0; i < 8; i += 2) ld2(&buf[8 * g + i], rk[i], rk[i + 1]);
        min_piv = fminf(min_piv, piv.x);
        const float dd = rcp_approx(fmaf(piv.x, piv.x, piv.y * piv.y));
        const float2 inv = make_float2(piv.x * dd, -piv.y * dd);
        const bool me = (u == k);
        const float2 fi = cmul(f, inv);                  // f_u / p
        const float2 nm = me ? make_float2(0.f, 0.f) : make_float2(-fi.x, -fi.y);
        if (me) myinv = inv;
#pragma unroll
        for (int i = 0; i < 8; ++i) cmac(A[i], nm, rk[i]);
        if (g == gk) A[ik] = me ? make_float2(1.f, 0.f) : make_float2(-fi.x, -fi.y);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) A[i] = cmul(A[i], myinv);
    return min_piv;
}


// B_c^{-1} of Alg. 3 for one cluster from the staged H_c (S x 16, row pitch
// 16, scale exponent eh from tcdl_h_scale): the Gram conj(H_c^H H_c) on the
// tensor cores (FP16 hi / lo, three products per k-step of 8 antennas), plus
// delta on the diagonal, row-major into Qs (pitch QP), then the column-split
// Gauss-Jordan; lane (ur, gc) returns entries (ur, 8 gc + i) of the inverse in
// A.  An FP32 pivot below 2^-12 of the largest diagonal entry recomputes this
// cluster's B_c and its inverse in FP64 (counted in *retries; Vb is scratch).
// Shared by the downlink kernel and the operator kernel (dbp_factor.cuh).
__device__ __forceinline__ void tcdl_operator(const float2 *Hs, int S, int eh, float2 *Qs, float2 *Vb, int lane,
                                              float f_delta, double delta, bool valid, unsigned int *retries,
                                              float2 (&A)[8]) {
    using C2 = float2;
    constexpr int QP = TcDl::QP;
    const int g = lane >> 2, t = lane & 3;
    const int ur = lane & 15, gc = lane >> 4;
    // Gram G = H_c^H H_c on the tensor cores: m-tile mt = users
    // 8 mt .. 8 mt + 7 (rows), n-tile nt = users 8 nt .. (columns), K =
    // antennas s0 + t and s0 + t + 4 of each k-step (re, im interleaved).
    const float sh = dl16_exp2i(eh);
    float gacc[2][2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) gacc[mt][nt][i] = 0.f;
    for (int s0 = 0; s0 < S; s0 += 8) {
        uint32_t ah[2][4], al[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
            dl16_afrag(Hs[(s0 + t) * 16 + 8 * mt + g], Hs[(s0 + t + 4) * 16 + 8 * mt + g], sh, ah[mt], al[mt]);
        // the B fragment of H_c for n-tile nt is registers 0 and 2 of m-tile
        // nt's A fragment; block (1, 0) is the conjugate transpose of block
        // (0, 1) (the Gram is Hermitian) and is not multiplied
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = mt; nt < 2; ++nt)
                mma3h(gacc[mt][nt], ah[mt], al[mt], ah[nt][0], ah[nt][2], al[nt][0], al[nt][2]);
    }
    const float ug = dl16_exp2i(-2 * eh);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) gacc[mt][nt][i] *= ug;
    // B_c = conj(G) + delta I, row-major into Qs
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = mt; nt < 2; ++nt)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int row = 8 * mt + g, col = 8 * nt + 2 * t + q;
                C2 v = make_float2(gacc[mt][nt][q], -gacc[mt][nt][2 + q]);
                if (row == col) v.x += f_delta;
                Qs[row * QP + col] = v;
                // conj(G)[col][row] = G[row][col]
                if (nt != mt) Qs[col * QP + row] = make_float2(gacc[mt][nt][q], gacc[mt][nt][2 + q]);
            }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; i += 2) ld2(&Qs[ur * QP + 8 * gc + i], A[i], A[i + 1]);
    float dmax = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        if (8 * gc + i == ur) dmax = A[i].x;
    dmax = warp_redux_max(dmax);
    const float min_piv = gj_split16_s(A, ur, gc, Qs);   // B_c in Qs is no longer read
    __syncwarp();
    if (!(min_piv >= 0x1p-12f * dmax) && valid) {
        // FP64 retry: B_c and its inverse again in FP64 (row ur per lane)
        double2 D[16];
#pragma unroll
        for (int v = 0; v < 16; ++v) D[v] = make_double2(0.0, 0.0);
        for (int r = 0; r < S; ++r) {
            const C2 hu = Hs[r * 16 + ur];
            const double2 hd = make_double2(hu.x, hu.y);
#pragma unroll
            for (int v = 0; v < 16; ++v) {
                const C2 hv = Hs[r * 16 + v];
                cmacc(D[v], make_double2(hv.x, hv.y), hd);      // conj(H[r][v]) H[r][ur]
            }
        }
#pragma unroll
        for (int v = 0; v < 16; ++v)
            if (v == ur) D[v].x += delta;
        gj_invert<16>(D, reinterpret_cast<double2 *>(Vb), ur, lane);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const double2 dv = gc ? D[8 + i] : D[i];
            A[i] = make_float2((float)dv.x, (float)dv.y);
        }
        if (lane == 0 && retries) atomicAdd(retries, 1u);
        __syncwarp();
    }
}

// (a template only so that every translation unit may include it)
template <int UT>
__global__ void __launch_bounds__(512, 1) dbp_tcdl_kernel(const FusedParams p) {
    static_assert(UT == TcDl::U, "the downlink tensor-core kernel is for 16 users");
    using C2 = float2;
    constexpr int U = TcDl::U, VPD = TcDl::VPD, QP = TcDl::QP, CP = TcDl::CP, CE = TcDl::CE;
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int C = p.C, P = p.P, S = p.S, N = p.N, B = p.B, W = p.W;
    const int pl = warp / C, c = warp - pl * C;
    const int g = lane >> 2, t = lane & 3;          // MMA layout
    const int ur = lane & 15, gc = lane >> 4;       // column-split layout: row ur, columns 8 gc + i

    unsigned char *wb = smem_raw + (size_t)warp * p.warp_bytes;
    C2 *Vb = reinterpret_cast<C2 *>(wb + p.off_v);
    C2 *Qs = reinterpret_cast<C2 *>(wb + p.off_g);
    C2 *contrib = reinterpret_cast<C2 *>(smem_raw + (size_t)nwarps * p.warp_bytes);   // [nwarps][CE]
    C2 *db = contrib + nwarps * CE + pl * CE;                 // d = (s - w) / C of this subcarrier
    C2 *ss = contrib + nwarps * CE + P * CE + pl * CE;        // s of this subcarrier, this pass
    uint64_t *bars = reinterpret_cast<uint64_t *>(contrib + nwarps * CE + 2 * P * CE) + 2 * warp;
    const C2 *grp = contrib + pl * C * CE;
    C2 *mine = contrib + warp * CE;

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
    const C2 *Sg = reinterpret_cast<const C2 *>(p.vin);
    auto issue = [&](int w, int b) {
        const uint32_t hbytes = (uint32_t)(S * U * 8);
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) {
            mbar_arrive_expect_tx(&bars[b], hbytes + p.starve_bytes);
            bulk_g2s(wb + (b ? p.off_h1 : 0), Hg + ((size_t)w * B + (size_t)c * S) * U, hbytes, &bars[b]);
        }
    };

    const float kap = p.f_kappa, gam = p.f_gamma, ic = p.f_invC, ir = p.f_inv_rho, eps = p.f_eps;
    grid_dependency_wait();
    grid_dependents_launch();
    float energy = 0.f;
    uint32_t parity = 0u;
    int tile = blockIdx.x;
    if (tile < p.tiles && tile * P + pl < W) issue(tile * P + pl, 0);

    for (int it = 0; tile < p.tiles; ++it, tile += gridDim.x) {
        const int b = it & 1;
        const int w = tile * P + pl;
        const bool valid = (w < W);
        const int ntile = tile + gridDim.x;
        if (ntile < p.tiles && ntile * P + pl < W) issue(ntile * P + pl, b ^ 1);
        if (valid) {
            mbar_wait_bounded(&bars[b], (parity >> b) & 1u, p.status, p.wait_iters);
            parity ^= (1u << b);
        }
        const C2 *Hs = reinterpret_cast<const C2 *>(wb + (b ? p.off_h1 : 0));

        const int eh = tcdl_h_scale(Hs, S, lane);       // H_c's FP16 scale (Gram and output)

        // ---- B_c^{-1} into Qs ----
        C2 *frow = (p.factor != nullptr && valid) ? p.factor + (((size_t)w * C + c) * U + ur) * U + 8 * gc : nullptr;
        if (p.factor_mode == 2) {
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
                float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                if (frow != nullptr) q = *reinterpret_cast<const float4 *>(&frow[i]);
                Qs[ur * QP + 8 * gc + i] = make_float2(q.x, q.y);
                Qs[ur * QP + 8 * gc + i + 1] = make_float2(q.z, q.w);
            }
        } else {
            C2 A[8];
            tcdl_operator(Hs, S, eh, Qs, Vb, lane, p.f_delta, p.delta, valid, p.retries, A);
#pragma unroll
            for (int i = 0; i < 8; ++i) Qs[ur * QP + 8 * gc + i] = A[i];
            if (p.factor_mode == 1 && frow != nullptr) {
#pragma unroll
                for (int i = 0; i < 8; i += 2)
                    *reinterpret_cast<float4 *>(&frow[i]) = make_float4(A[i].x, A[i].y, A[i + 1].x, A[i + 1].y);
            }
        }
        __syncwarp();

        // A fragments (hi, lo) of B_c^{-1}: lane (g, t) takes entries
        // [8 mt + g][8 ks + t] and [8 mt + g][8 ks + t + 4] as the real row's
        // coefficients (Re Q, -Im Q); one scale for the warp
        uint32_t qh[2][2][4], ql[2][2][4];
        int eq;
        {
            C2 qv[2][2][2];
            float mq = 0.f;
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int ks = 0; ks < 2; ++ks)
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        qv[mt][ks][hh] = Qs[(8 * mt + g) * QP + 8 * ks + 4 * hh + t];
                        mq = fmaxf(mq, cabsmax(qv[mt][ks][hh]));
                    }
            eq = dl16_scale_exp(dl16_warp_max(mq));
            const float sq = dl16_exp2i(eq);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int ks = 0; ks < 2; ++ks)
                    dl16_afrag(make_float2(qv[mt][ks][0].x, -qv[mt][ks][0].y),
                               make_float2(qv[mt][ks][1].x, -qv[mt][ks][1].y), sq, qh[mt][ks], ql[mt][ks]);
        }

        for (int n0 = 0; n0 < N; n0 += TcDl::NS) {
            const int nv = min(TcDl::NS, N - n0);
            const int nvu = nv * U;
            // stage s of this pass (zero past N) for every warp of the subcarrier
            __syncthreads();
            for (int e = c * 32 + lane; e < TcDl::NS * U; e += C * 32) {
                const int n = e >> 4, u = e & 15;
                ss[sw20(n, u, CP)] = (valid && n < nv) ? Sg[((size_t)w * N + n0 + n) * U + u] : make_float2(0.f, 0.f);
                db[sw20(n, u, CP)] = make_float2(0.f, 0.f);   // slots past N keep d = 0
            }
            __syncthreads();

            // Init: z_c = kappa s, lambda_c = 0, v_c = z_c (v_c also kept in
            // registers, in the accumulator layout)
            C2 lam[2][2][2], vr[2][2][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const int u = 8 * mt + g, n = 8 * nt + 2 * t + q;
                        vr[mt][nt][q] = cscale(ss[sw20(n, u, CP)], kap);
                        Vb[sw20(n, u, VPD)] = vr[mt][nt][q];
                        lam[mt][nt][q] = make_float2(0.f, 0.f);
                    }
            __syncwarp();

            for (int iter = 2; iter <= p.T; ++iter) {
                C2 m[2][2][2];
                tcdl_apply(qh, ql, eq, Vb, g, t, m);              // B_c^{-1} v_c
                // m_c = H_c x_c = v_c - rho^{-1} B_c^{-1} v_c
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const C2 v = vr[mt][nt][q];
                            m[mt][nt][q].x = fmaf(-ir, m[mt][nt][q].x, v.x);
                            m[mt][nt][q].y = fmaf(-ir, m[mt][nt][q].y, v.y);
                        }
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const int u = 8 * mt + g, n = 8 * nt + 2 * t + q;
                            mine[sw20(n, u, CP)] = csub(m[mt][nt][q], lam[mt][nt][q]);   // w_c
                        }
                __syncthreads();
                for (int base = c * 32; base < nvu; base += C * 32) {
                    const int e = base + lane;                    // < NS U: in the buffers
                    const int idx = sw20(e >> 4, e & 15, CP);
                    // the C <= 16 contributions loaded together, then added in
                    // cluster order (the order of consensus_sum)
                    C2 tv[16];
#pragma unroll
                    for (int cc = 0; cc < 16; ++cc) tv[cc] = (cc < C) ? grp[idx + cc * CE] : make_float2(0.f, 0.f);
                    C2 ws = make_float2(0.f, 0.f);
#pragma unroll
                    for (int cc = 0; cc < 16; ++cc)
                        if (cc < C) {
                            ws.x += tv[cc].x;
                            ws.y += tv[cc].y;
                        }
                    const C2 sv = ss[idx];
                    C2 dl = csub(sv, ws);
                    if (eps > 0.f) {
                        // Lemma 2: (s - w)/C scaled by max{0, 1 - eps / ||s - w||}
                        // (the 16 users of a symbol are 16 aligned lanes)
                        const float nrm = sqrtf(group_sum<16>(dl.x * dl.x + dl.y * dl.y));
                        const float k = (nrm > 0.f) ? fmaxf(0.f, 1.f - eps / nrm) : 0.f;
                        dl = cscale(dl, k);
                    }
                    if (e < nvu) db[idx] = make_float2(dl.x * ic, dl.y * ic);
                }
                __syncthreads();
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const int u = 8 * mt + g, n = 8 * nt + 2 * t + q;
                            const C2 wc = csub(m[mt][nt][q], lam[mt][nt][q]);
                            const C2 d = db[sw20(n, u, CP)];
                            C2 z = cadd(wc, d);                   // z_c = w_c + (s - w) / C
                            C2 &l = lam[mt][nt][q];
                            l.x = fmaf(-gam, m[mt][nt][q].x - z.x, l.x);
                            l.y = fmaf(-gam, m[mt][nt][q].y - z.y, l.y);
                            vr[mt][nt][q] = cadd(z, l);           // v_c = z_c + lambda_c
                            Vb[sw20(n, u, VPD)] = vr[mt][nt][q];
                        }
                __syncwarp();
            }

            // Output x_c = H^{dH}_c B_c^{-1} v_c
            {
                C2 tt[2][2][2];
                tcdl_apply(qh, ql, eq, Vb, g, t, tt);
                __syncwarp();
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                        for (int q = 0; q < 2; ++q) Vb[sw20(8 * nt + 2 * t + q, 8 * mt + g, VPD)] = tt[mt][nt][q];
                __syncwarp();
            }
            C2 *xo = reinterpret_cast<C2 *>(p.out);
            uint32_t th[2][2][2], tl[2][2][2];          // B fragments of B_c^{-1} v_c
            const int et = dl16_bfrag(Vb, g, t, th, tl);
            const float sh = dl16_exp2i(eh), ux = dl16_exp2i(-eh) * dl16_exp2i(-et);
            for (int sa = 0; sa < S; sa += 8) {
                // m-tile of antennas sa .. sa+7: A = H^{dH}_c, A[s'][u] = conj(H_c[s'][u]),
                // the real row's coefficients (Re H, Im H)
                float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    uint32_t ah[4], al[4];
                    dl16_afrag(Hs[(sa + g) * U + 8 * ks + t], Hs[(sa + g) * U + 8 * ks + 4 + t], sh, ah, al);
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) mma3h(acc[nt], ah, al, th[nt][ks][0], th[nt][ks][1], tl[nt][ks][0], tl[nt][ks][1]);
                }
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[nt][i] *= ux;
                if (valid) {
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const int n = 8 * nt + 2 * t + q;
                            if (n < nv) {
                                const C2 xv = make_float2(acc[nt][q], acc[nt][2 + q]);
                                xo[((size_t)w * N + n0 + n) * B + (size_t)c * S + sa + g] = xv;
                                energy += xv.x * xv.x + xv.y * xv.y;
                            }
                        }
                }
            }
            __syncwarp();
        }
    }
    if (p.energy != nullptr) {
#pragma unroll
        for (int m2 = 16; m2 > 0; m2 >>= 1) energy += shfl_x(energy, m2);
        if (lane == 0) atomicAdd(p.energy, (double)energy);
    }
}

}  // namespace dbp
