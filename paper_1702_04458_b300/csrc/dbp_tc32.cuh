// dbp_tc32.cuh -- decentralized ADMM uplink detection (Alg. 1, U x U form)
// for square clusters S = U = 32 on the fifth-generation tensor cores
// (tcgen05, accumulators in tensor memory).
//
// One CTA of 8 warps owns one subcarrier at a time (persistent over
// subcarriers, two CTAs per SM); warp c is the processing element of
// antenna cluster c for the per-cluster scalar work.  Every dense product of
// the cluster -- the Gram H_c^H H_c, the matched filter H_c^H y_c, the
// regularised estimate B_c^{-1} m_c and each iteration's B_c^{-1} (s -
// lambda_c) -- runs as one tcgen05.mma chain issued by a single thread;
// the explicit inverse B_c^{-1} (the paper's getrf/getri, Sec. VII-A) is the
// in-register Gauss-Jordan elimination of the bulk-copy kernel, with its
// pivot check and FP64 retry.
//
// Products in FP32 from FP16 tensor cores.  Every FP32 operand x is scaled
// by a power of two (so that the operand's largest magnitude lies in
// [2^13, 2^14)) and split into two FP16 values, hi = fp16(x) and lo =
// fp16(x - hi), so that |x - hi - lo| <= 2^-24 |x| for every value that is
// not 2^17 times smaller than the operand's largest; a product is
// accumulated in FP32 as hi_a hi_b + hi_a lo_b + lo_a hi_b (the dropped
// lo_a lo_b term is below 2^-22 of the product).  The scale factors are
// exact and are divided out of the accumulators.  16-bit inputs (FP16 /
// BF16 H and y) enter the Gram and the matched filter as they are, with one
// product (every product of two 16-bit values is exact in FP32).
//
// Complex products as real ones: a cluster's operand tile has 64 rows, the
// real and the imaginary part of each of the 32 users (row 32h + 16p + i
// holds component p of user 16h + i), and the contraction over antennas or
// users in K.  D = A B^T then holds every product of components, and the
// complex result is Re = D_00 + D_11 (or D_00 - D_11), Im = D_01 - D_10 (or
// D_10 + D_01): component p = 0 and p = 1 of a user sit in lanes l and l + 16
// of the same warp, so one shuffle per value completes it.  The two clusters
// of a pair are stacked into one M = 128 MMA (cluster 2j in rows 0-63,
// cluster 2j+1 in rows 64-127) against both clusters' B operands side by
// side, so every tensor-memory lane holds a needed row; the cross-cluster
// half of the result is not read.
//
// Per subcarrier: bulk copies of H[w] and y[w] into shared memory; operand
// conversion; matched filter (all pairs, one chain each); Gram (two rounds of
// two pairs); Gauss-Jordan per warp; y_reg = B_c^{-1} m_c; the consensus
// (fusion step of Alg. 1) summed over the clusters in a fixed order through
// shared memory, the (E2) prox, then T_max - 1 iterations of the lambda
// update (E3), the operator product (E1) and the consensus; slicer and
// outputs.  Waits on mbarriers are bounded: a wait that gives up raises bit 0
// of the status word and the CTA leaves its subcarrier loop, frees its
// tensor memory and returns.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dbp_tc5.cuh"
#include "dbp_tma.cuh"

namespace dbp {
namespace tc32 {

constexpr int THREADS = 256;
constexpr int HT = 0;              // 4 pairs x 16 KB: raw H[w] | A/B tiles (hi, lo) | Gram rows | B_c^{-1} tiles
constexpr int HT_PAIR = 16384;
constexpr int HT_LO = 8192;
constexpr int VT = 65536;          // 4 pairs x 8 KB: raw y[w] | y / state tiles (hi, lo) | consensus partials
constexpr int VT_PAIR = 8192;
constexpr int VT_LO = 4096;
constexpr int SCR = 98304;         // per-warp Gauss-Jordan pivot buffers (FP64 rows on retry)
constexpr int SCR_WARP = 1024;
constexpr int SLOTS = SCR + 8 * SCR_WARP;   // scale exponents and warp maxima
constexpr int PARAMS = SLOTS + 160;        // OpParams of the operator phase (64 B)
constexpr int BARS = SLOTS + 256;
constexpr int SMEM = BARS + 64;
constexpr int TMEM_COLS = 256;
constexpr int PART_LD = 20;        // floats per consensus partial row (16 used, padded against bank conflicts)

// Byte offset of 16-bit element (row, k) of a K-major operand tile with 32
// contraction elements per row: 8 x 16-byte core matrices, K-direction core
// matrices 128 B apart (LBO), 8-row groups 512 B apart (SBO).
__device__ __forceinline__ int off16(int row, int k) {
    return (row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}
// Row of component p of user u inside a cluster's 64-row tile.
__device__ __forceinline__ int arow(int p, int u) { return 32 * (u >> 4) + 16 * p + (u & 15); }

// Power-of-two exponent e with m 2^e in [2^13, 2^14) (0 for 0 / non-finite).
__device__ __forceinline__ int scale_exp(float m) {
    if (!(m > 0.f) || !(m < 3.0e38f)) return 0;
    int e;
    frexpf(m, &e);
    e = 14 - e;
    return e < -100 ? -100 : (e > 100 ? 100 : e);
}
__device__ __forceinline__ float exp2i(int e) { return __int_as_float((127 + e) << 23); }

template <typename T> struct Op16;
template <> struct Op16<__half> {
    static constexpr int fmt = tc5::FMT_F16;
    static __device__ __forceinline__ uint16_t bits(float x) { return __half_as_ushort(__float2half_rn(x)); }
    static __device__ __forceinline__ float back(uint16_t b) { return __half2float(__ushort_as_half(b)); }
};
template <> struct Op16<__nv_bfloat16> {
    static constexpr int fmt = tc5::FMT_BF16;
    static __device__ __forceinline__ uint16_t bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
    static __device__ __forceinline__ float back(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }
};
// Operand type of the Gram / matched filter for an input type.
template <typename TIn> struct GramOp { using type = __half; };
template <> struct GramOp<__nv_bfloat162> { using type = __nv_bfloat16; };

// hi / lo FP16 split of x (already scaled).
__device__ __forceinline__ void split16(float x, uint32_t &hi, uint32_t &lo) {
    const __half h = __float2half_rn(x);
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
}
__device__ __forceinline__ uint32_t pack2(uint32_t a, uint32_t b) { return a | (b << 16); }

// D (+)= A B^T over K = 32 (two K steps of 16): A tile of 128 rows at a_hi /
// a_lo, B tile at b_hi / b_lo (shared-memory byte addresses); three products
// with the split, one (hi only) without.
__device__ __forceinline__ void mma_k32(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo,
                                        uint32_t id, bool split) {
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
        const uint32_t o = ks * 256;
        const uint64_t ah = tc5::sdesc(a_hi + o, 128, 512), bh = tc5::sdesc(b_hi + o, 128, 512);
        tc5::mma_f16(d, ah, bh, id, ks > 0 ? 1u : 0u);
        if (split) {
            tc5::mma_f16(d, ah, tc5::sdesc(b_lo + o, 128, 512), id, 1u);
            tc5::mma_f16(d, tc5::sdesc(a_lo + o, 128, 512), bh, id, 1u);
        }
    }
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, m));
    return v;
}

// Load 32 consecutive accumulator columns of this warp's lane quadrant.
__device__ __forceinline__ void ld32(uint32_t taddr, float (&a)[32]) {
    tc5::ld_x32(taddr, a);
    tc5::ld_wait();
}

}  // namespace tc32

// In-register Gauss-Jordan inversion of a 32 x 32 Hermitian positive
// definite matrix held by one warp as 4 x 8 blocks: lane l = 4 rg + cg owns
// rows 4 rg .. 4 rg + 3 and columns 8 cg .. 8 cg + 7 (A[r][c]).
// Step k: the lanes holding column k publish it (colbuf), the lanes holding
// row k publish it (rowbuf), every lane updates its block with the rank-1
// term f_i a_kj, f_i = a_ik / a_kk, and the owners of column k write the new
// column (-f_i; 1 on the pivot row, whose row stays multiplied by its pivot
// until the final scaling).  Buffers alternate between steps, so one warp
// barrier per step orders writes and reads.  The step loop is unrolled by 8
// so every register index is static.  Returns the smallest pivot (real part).
__device__ __forceinline__ float gj2d_invert(float2 (&A)[4][8], float2 *buf, int lane) {
    const int rg = lane >> 2, cg = lane & 3;
    float min_piv = 3.0e38f;
    float2 myinv[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) myinv[r] = make_float2(1.f, 0.f);
#pragma unroll 1
    for (int k0 = 0; k0 < 32; k0 += 8) {
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const int k = k0 + kk;
            float2 *colbuf = buf + (kk & 1) * 64, *rowbuf = colbuf + 32;
            const bool ownc = (cg == (k >> 3)), ownr = (rg == (k >> 2));
            if (ownc) {
                *reinterpret_cast<float4 *>(&colbuf[4 * rg]) = make_float4(A[0][kk].x, A[0][kk].y, A[1][kk].x, A[1][kk].y);
                *reinterpret_cast<float4 *>(&colbuf[4 * rg + 2]) = make_float4(A[2][kk].x, A[2][kk].y, A[3][kk].x, A[3][kk].y);
            }
            if (ownr) {
#pragma unroll
                for (int c = 0; c < 8; c += 2)
                    *reinterpret_cast<float4 *>(&rowbuf[8 * cg + c]) =
                        make_float4(A[kk & 3][c].x, A[kk & 3][c].y, A[kk & 3][c + 1].x, A[kk & 3][c + 1].y);
            }
            __syncwarp();
            const float2 pk = colbuf[k];
            min_piv = fminf(min_piv, pk.x);
            const float d = __frcp_rn(fmaf(pk.x, pk.x, pk.y * pk.y));
            const float2 inv = make_float2(pk.x * d, -pk.y * d);
            float2 f[4], p[8];
            {
                float2 a, b;
                ld2(&colbuf[4 * rg], a, b);
                f[0] = a; f[1] = b;
                ld2(&colbuf[4 * rg + 2], a, b);
                f[2] = a; f[3] = b;
#pragma unroll
                for (int c = 0; c < 8; c += 2) {
                    ld2(&rowbuf[8 * cg + c], a, b);
                    p[c] = a; p[c + 1] = b;
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const bool piv = ownr && (r == (kk & 3));
                const float2 a = f[r];
                f[r] = piv ? make_float2(0.f, 0.f) : make_float2(a.x * inv.x - a.y * inv.y, a.x * inv.y + a.y * inv.x);
                if (piv) myinv[r] = inv;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float2 nf = make_float2(-f[r].x, -f[r].y);
#pragma unroll
                for (int c = 0; c < 8; ++c) cmac(A[r][c], nf, p[c]);
            }
            if (ownc) {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const bool piv = ownr && (r == (kk & 3));
                    A[r][kk] = piv ? make_float2(1.f, 0.f) : make_float2(-f[r].x, -f[r].y);
                }
            }
            __syncwarp();
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float2 a = A[r][c];
            A[r][c] = make_float2(a.x * myinv[r].x - a.y * myinv[r].y, a.x * myinv[r].y + a.y * myinv[r].x);
        }
    return min_piv;
}

// Write B_c^{-1} (row `lane` in R) as the cluster's operator tile (hi / lo,
// scaled by 2^e with e from the warp's largest magnitude, stored at *eslot).
__device__ __forceinline__ void tc32_put_operator(const float2 (&R)[32], unsigned char *th, int clw, int *eslot,
                                                  int lane) {
    using namespace tc32;
    float mb = 0.f;
#pragma unroll
    for (int v = 0; v < 32; ++v) mb = fmaxf(mb, fmaxf(fabsf(R[v].x), fabsf(R[v].y)));
    const int eb = scale_exp(warp_max(mb));
    if (lane == 0) *eslot = eb;
    const float sb = exp2i(eb);
#pragma unroll
    for (int pc = 0; pc < 2; ++pc) {
        const int row = 64 * clw + arow(pc, lane);
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const float2 a = R[8 * k4 + 2 * t], b = R[8 * k4 + 2 * t + 1];
                uint32_t ha, la, hb, lb;
                split16((pc ? a.y : a.x) * sb, ha, la);
                split16((pc ? b.y : b.x) * sb, hb, lb);
                hw[t] = pack2(ha, hb);
                lw[t] = pack2(la, lb);
            }
            const int o = off16(row, 8 * k4);
            *reinterpret_cast<uint4 *>(th + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4 *>(th + HT_LO + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
    }
}

// Write B_c^{-1} held as 4 x 8 blocks (lane 4 rg + cg: rows 4 rg .. + 3,
// columns 8 cg .. + 7) as the cluster's operator tile (hi / lo, scaled by
// 2^e with e from the warp's largest magnitude, stored at *eslot): the
// lane's 8 columns are one 16-byte K chunk of each of its tile rows.
__device__ __forceinline__ void tc32_put_operator_2d(const float2 (&A)[4][8], unsigned char *th, int clw, int *eslot,
                                                     int lane) {
    using namespace tc32;
    const int rg = lane >> 2, cg = lane & 3;
    float mb = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) mb = fmaxf(mb, fmaxf(fabsf(A[r][c].x), fabsf(A[r][c].y)));
    const int eb = scale_exp(warp_max(mb));
    if (lane == 0) *eslot = eb;
    const float sb = exp2i(eb);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int pc = 0; pc < 2; ++pc) {
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const float2 a = A[r][2 * t], b = A[r][2 * t + 1];
                uint32_t ha, la, hb, lb;
                split16((pc ? a.y : a.x) * sb, ha, la);
                split16((pc ? b.y : b.x) * sb, hb, lb);
                hw[t] = pack2(ha, hb);
                lw[t] = pack2(la, lb);
            }
            const int o = off16(64 * clw + arow(pc, 4 * rg + r), 8 * cg);
            *reinterpret_cast<uint4 *>(th + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4 *>(th + HT_LO + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
}

// FP64 recomputation of one cluster's operator (whole warp): the Gram
// H_c^H H_c + delta I from the cluster block in global memory (row u per
// lane), its Gauss-Jordan inverse in FP64, rounded to FP32 and written as
// the operator tile.  Out of line: it runs only when an FP32 pivot was too
// small, and its FP64 rows must not weigh on the kernel's registers.
template <typename TIn>
__device__ __noinline__ void tc32_fp64_operator(const TIn *Hg, double delta, double2 *scr, unsigned char *th, int clw,
                                                int *eslot, int lane) {
    double2 D[32];
#pragma unroll
    for (int v = 0; v < 32; ++v) D[v] = make_double2(0.0, 0.0);
    for (int s = 0; s < 32; ++s) {
        const float2 hu = to_f2(Hg[s * 32 + lane]);
        const double2 hd = make_double2(hu.x, hu.y);
#pragma unroll
        for (int v = 0; v < 32; ++v) {
            const float2 hv = to_f2(Hg[s * 32 + v]);
            cmacc(D[v], hd, make_double2(hv.x, hv.y));
        }
    }
#pragma unroll
    for (int v = 0; v < 32; ++v)
        if (v == lane) D[v].x += delta;
    __syncwarp();
    gj_invert<32>(D, scr, lane, lane);
    float2 R[32];
#pragma unroll
    for (int v = 0; v < 32; ++v) R[v] = make_float2((float)D[v].x, (float)D[v].y);
    tc32_put_operator(R, th, clw, eslot, lane);
}

// What the operator phase needs besides shared memory, kept in shared
// memory by the kernel so that the phase is called without arguments.
struct OpParams {
    const void *H;              // inputs in global memory (FP64 retry)
    unsigned int *retries;      // FP64 retry counter
    double delta;               // diagonal loading rho
    long long row0;             // first H row of the subcarrier (w B)
    int C;
};

// The operator phase of one subcarrier (whole CTA): warp c < C loads its
// cluster's Gram as 4 x 8 blocks (from the XOR-swizzled planes Gr, Gi of the
// Gram readout), waits until every warp has, inverts it by Gauss-Jordan
// elimination with the pivot check, recomputes it in FP64 if a pivot was too
// small, and writes B_c^{-1} as the cluster's operator tile.
template <typename TIn>
__device__ __forceinline__ void tc32_operator_phase() {
    using namespace tc32;
    extern __shared__ __align__(1024) unsigned char sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rg = lane >> 2, cg = lane & 3;
    const OpParams &op = *reinterpret_cast<const OpParams *>(sm + PARAMS);
    int *eslot = reinterpret_cast<int *>(sm + SLOTS);
    const int C = op.C;
    float2 A[4][8];
    if (warp < C) {
        const float *gr = reinterpret_cast<const float *>(sm + HT + (warp >> 1) * HT_PAIR + (warp & 1) * 8192);
        const float *gi = gr + 1024;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = 4 * rg + r;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ch = 2 * cg + h;
                const float4 a = *reinterpret_cast<const float4 *>(gr + i * 32 + 4 * (ch ^ (i & 7)));
                const float4 b = *reinterpret_cast<const float4 *>(gi + i * 32 + 4 * (ch ^ (i & 7)));
                A[r][4 * h + 0] = make_float2(a.x, b.x);
                A[r][4 * h + 1] = make_float2(a.y, b.y);
                A[r][4 * h + 2] = make_float2(a.z, b.z);
                A[r][4 * h + 3] = make_float2(a.w, b.w);
            }
        }
    }
    __syncthreads();        // every Gram block is in registers
    if (warp < C) {
        float dmax = 0.f;
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (4 * rg + r == 8 * cg + c) dmax = fmaxf(dmax, A[r][c].x);
        dmax = warp_max(dmax);
        float2 *scr = reinterpret_cast<float2 *>(sm + SCR + warp * SCR_WARP);
        const float min_piv = gj2d_invert(A, scr, lane);
        unsigned char *th = sm + HT + (warp >> 1) * HT_PAIR;
        if (!(min_piv >= 0x1p-12f * dmax)) {
            if (lane == 0) eslot[24 + warp] = 1;    // FP64 retry after the phase
        } else {
            tc32_put_operator_2d(A, th, warp & 1, eslot + 16 + warp, lane);
        }
    }
}

template <typename TIn, int NS>
__global__ void __launch_bounds__(tc32::THREADS, 2) dbp_tc32_kernel(const FusedParams p) {
    using namespace tc32;
    using GOp = typename GramOp<TIn>::type;
    constexpr bool IN16 = InTraits<TIn>::bytes == 4;
    constexpr int EB = InTraits<TIn>::bytes;
    constexpr int HRAW = IN16 ? 32768 : 0;      // raw H[w] offset in the H region
    extern __shared__ __align__(1024) unsigned char sm[];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wg = warp >> 2, q = warp & 3;
    const int C = p.C, N = p.N, B = p.B, W = p.W, T = p.T;
    const int npairs = C >> 1;
    // this thread's row of a pair's accumulator tile: cluster 2j + cl,
    // component pp of user uu
    const int cl = q >> 1, pp = lane >> 4, uu = 16 * (q & 1) + (lane & 15);
    const int kgrp = 2 * wg + cl;      // consensus partial written by this thread

    uint64_t *bar_ld = reinterpret_cast<uint64_t *>(sm + BARS);
    uint64_t *bar_mma = bar_ld + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar_ld + 2);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);
    int *eslot = reinterpret_cast<int *>(sm + SLOTS);           // eH[8] | eY[8] | eB[8] | retry flags[8]
    float *mslot = reinterpret_cast<float *>(sm + SLOTS + 128); // per-warp maxima

    if (tid == 0) {
        mbar_init(bar_ld, 1);
        mbar_init(bar_mma, 1);
        *abort_flag = 0;
        for (int k = 0; k < 8; ++k) eslot[24 + k] = 0;
        OpParams *op = reinterpret_cast<OpParams *>(sm + PARAMS);
        op->H = p.H;
        op->retries = p.retries;
        op->delta = p.delta;
        op->C = p.C;
        fence_mbar_init();
    }
    if (warp == 0) {
        tc5::tmem_alloc(tslot, TMEM_COLS);
        tc5::tmem_relinquish();
    }
    tc5::fence_before_sync();
    __syncthreads();
    tc5::fence_after_sync();
    const uint32_t tbase = *tslot;
    const uint32_t tq = tbase + ((uint32_t)(32 * q) << 16);     // this warp's lane quadrant
    const uint32_t sbase = tc5::smem_addr(sm);
    grid_dependency_wait();

    uint32_t ph_ld = 0, ph_mma = 0;
    const uint32_t hbytes = (uint32_t)B * 32u * EB;            // H[w]: B rows x U = 32
    const uint32_t ybytes = (uint32_t)N * (uint32_t)B * EB;    // y[w]: N rows x B
    const uint32_t id_in = tc5::idesc(Op16<GOp>::fmt, 128, 64);     // matched filter
    const uint32_t id_gram = tc5::idesc(Op16<GOp>::fmt, 128, 128);  // Gram
    const uint32_t id_op = tc5::idesc(tc5::FMT_F16, 128, 64);       // operator x state
    const float rho = p.f_rho, gam = p.f_gamma;

    auto wait_mma = [&]() {
        if (!mbar_wait_bounded(bar_mma, ph_mma, p.status)) *abort_flag = 1;
        ph_mma ^= 1u;
        tc5::fence_after_sync();
    };
    // Consensus: w = sum_c contrib_c.  Each thread passes the sum of its two
    // rows' contributions (clusters k and k + 4 of partial group k = kgrp);
    // the four partials are added in the fixed order (0 + 1) + (2 + 3), so w
    // = ((c0 + c4) + (c1 + c5)) + ((c2 + c6) + (c3 + c7)) in every thread.
    auto consensus = [&](const float (&part_in)[NS], float (&wsum)[NS]) {
        float *part = reinterpret_cast<float *>(sm + VT);
        float *mine = part + ((kgrp * 2 + pp) * 32 + uu) * PART_LD;
#pragma unroll
        for (int n = 0; n < 16; n += 4) {
            float v[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) v[t] = (n + t < NS) ? part_in[n + t] : 0.f;
            *reinterpret_cast<float4 *>(mine + n) = make_float4(v[0], v[1], v[2], v[3]);
        }
        __syncthreads();
        const float *r0 = part + ((0 * 2 + pp) * 32 + uu) * PART_LD;
        const float *r1 = part + ((1 * 2 + pp) * 32 + uu) * PART_LD;
        const float *r2 = part + ((2 * 2 + pp) * 32 + uu) * PART_LD;
        const float *r3 = part + ((3 * 2 + pp) * 32 + uu) * PART_LD;
#pragma unroll
        for (int n = 0; n < NS; ++n) wsum[n] = (r0[n] + r1[n]) + (r2[n] + r3[n]);
    };
    // (E2) prox of the consensus sum, component pp.
    auto prox = [&](float (&wsum)[NS]) {
#pragma unroll
        for (int n = 0; n < NS; ++n) {
            if (p.reg >= 2) {
                const float v = clip_r(wsum[n] * p.f_invC, p.f_box_r);
                wsum[n] = (p.reg == 2 || pp == 0) ? v : 0.f;
            } else {
                wsum[n] = wsum[n] * p.f_e2_scale;
            }
        }
    };
    // Operator product result of pair j (this thread's row): component pp
    // of B_c^{-1} V_c for the NS symbols, scale removed.
    auto op_read = [&](int j, float us, float (&z)[NS]) {
        float a[16];
        tc5::ld_x16(tq + 64 * j + 32 * cl + 16, a);      // columns of p' = 1
        tc5::ld_wait();
#pragma unroll
        for (int n = 0; n < NS; ++n) z[n] = __shfl_xor_sync(0xffffffffu, a[n], 16);
        tc5::ld_x16(tq + 64 * j + 32 * cl, a);           // columns of p' = 0
        tc5::ld_wait();
#pragma unroll
        for (int n = 0; n < NS; ++n) z[n] = (a[n] + (pp ? z[n] : -z[n])) * us;
    };
    // Write this thread's column (user uu, component pp) of the state tile
    // V_c (B operand: rows 16 p' + n, K = user) for pair j, scaled by 2^ev.
    auto put_state = [&](int j, const float (&v)[NS], float sv) {
        unsigned char *base = sm + VT + j * VT_PAIR;
#pragma unroll
        for (int n = 0; n < 16; ++n) {
            uint32_t hi = 0, lo = 0;
            if (n < NS && n < N) split16(v[n] * sv, hi, lo);
            const int o = off16(32 * cl + 16 * pp + n, uu);
            *reinterpret_cast<uint16_t *>(base + o) = (uint16_t)hi;
            *reinterpret_cast<uint16_t *>(base + VT_LO + o) = (uint16_t)lo;
        }
    };
    // Largest |v| over the CTA (every thread passes its values; 0 if none).
    auto cta_max = [&](float m) {
        m = warp_max(m);
        if (lane == 0) mslot[warp] = m;
        __syncthreads();
        float r = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) r = fmaxf(r, mslot[k]);
        return r;
    };

    for (int w = blockIdx.x; w < W; w += gridDim.x) {
        // ---- bulk copies of H[w] and y[w] ------------------------------------
        if (tid == 0) {
            mbar_arrive_expect_tx(bar_ld, hbytes + ybytes + p.starve_bytes);
            bulk_g2s(sm + HT + HRAW, static_cast<const unsigned char *>(p.H) + (size_t)w * hbytes, hbytes, bar_ld);
            bulk_g2s(sm + VT, static_cast<const unsigned char *>(p.vin) + (size_t)w * ybytes, ybytes, bar_ld);
        }
        if (!mbar_wait_bounded(bar_ld, ph_ld, p.status, p.wait_iters)) *abort_flag = 1;
        ph_ld ^= 1u;

        // ---- operand conversion (warp c: cluster c).  The raw inputs and the
        // tiles share the regions, so each is read whole before any tile is
        // written: H first, then y. -------------------------------------------
        const int kc = lane >> 3, n8 = lane & 7;
        // H: clusters 0-3 then 4-7 (FP32: their raw bytes are exactly their
        // tiles' bytes; 16-bit: the raw H sits in the upper half, where only
        // the tiles of clusters 4-7 go); thread t converts rows s = 16 (t/32 % 2) .. + 15 of user
        // t % 32 of cluster 4 half + t / 64.
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            const int c = 4 * half + (tid >> 6), sh16 = 16 * ((tid >> 5) & 1);
            float2 hv[16];
            float mh = 0.f;
            if (c < C) {
                const TIn *Hc = reinterpret_cast<const TIn *>(sm + HT + HRAW) + (size_t)c * 32 * 32;
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    hv[s] = to_f2(Hc[(sh16 + s) * 32 + lane]);
                    mh = fmaxf(mh, fmaxf(fabsf(hv[s].x), fabsf(hv[s].y)));
                }
            }
            mh = warp_max(mh);
            if (lane == 0) mslot[warp] = mh;
            __syncthreads();        // the raw rows of this half are in registers
            if (*abort_flag) break;
            if (c < C) {
                const int eh = IN16 ? 0 : scale_exp(fmaxf(mslot[warp & ~1], mslot[warp | 1]));
                if (lane == 0 && sh16 == 0) eslot[c] = eh;
                const float sh = exp2i(eh);
                unsigned char *th = sm + HT + (c >> 1) * HT_PAIR;
#pragma unroll
                for (int pc = 0; pc < 2; ++pc) {
                    const int row = 64 * (c & 1) + arow(pc, lane);
#pragma unroll
                    for (int k2 = 0; k2 < 2; ++k2) {
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const float2 a = hv[8 * k2 + 2 * t], b = hv[8 * k2 + 2 * t + 1];
                            const float xa = pc ? a.y : a.x, xb = pc ? b.y : b.x;
                            if constexpr (IN16) {
                                hw[t] = pack2(Op16<GOp>::bits(xa), Op16<GOp>::bits(xb));
                                lw[t] = 0;
                            } else {
                                uint32_t ha, la, hb, lb;
                                split16(xa * sh, ha, la);
                                split16(xb * sh, hb, lb);
                                hw[t] = pack2(ha, hb);
                                lw[t] = pack2(la, lb);
                            }
                        }
                        const int o = off16(row, sh16 + 8 * k2);
                        *reinterpret_cast<uint4 *>(th + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        if (!IN16) *reinterpret_cast<uint4 *>(th + HT_LO + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                }
            }
            __syncthreads();        // the slots are read; the next half's raw rows are intact
        }
        if (*abort_flag) break;
        {
            float2 yv[2][8];    // y[n][c S + 8 kc + t], n = n8, n8 + 8
            float my = 0.f;
            if (warp < C) {
                const TIn *Y = reinterpret_cast<const TIn *>(sm + VT);
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int n = n8 + 8 * r;
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        yv[r][t] = (n < N) ? to_f2(Y[(size_t)n * B + warp * 32 + 8 * kc + t]) : make_float2(0.f, 0.f);
                        my = fmaxf(my, fmaxf(fabsf(yv[r][t].x), fabsf(yv[r][t].y)));
                    }
                }
            }
            __syncthreads();
            if (warp < C) {
                const int ey = IN16 ? 0 : scale_exp(warp_max(my));
                if (lane == 0) eslot[8 + warp] = ey;
                const float sy = exp2i(ey);
                unsigned char *tv = sm + VT + (warp >> 1) * VT_PAIR;
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int n = n8 + 8 * r;
#pragma unroll
                    for (int pc = 0; pc < 2; ++pc) {
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const float2 a = yv[r][2 * t], b = yv[r][2 * t + 1];
                            const float xa = pc ? a.y : a.x, xb = pc ? b.y : b.x;
                            if constexpr (IN16) {
                                hw[t] = pack2(Op16<GOp>::bits(xa), Op16<GOp>::bits(xb));
                                lw[t] = 0;
                            } else {
                                uint32_t ha, la, hb, lb;
                                split16(xa * sy, ha, la);
                                split16(xb * sy, hb, lb);
                                hw[t] = pack2(ha, hb);
                                lw[t] = pack2(la, lb);
                            }
                        }
                        const int o = off16(32 * (warp & 1) + 16 * pc + n, 8 * kc);
                        *reinterpret_cast<uint4 *>(tv + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        if (!IN16) *reinterpret_cast<uint4 *>(tv + VT_LO + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    }
                }
            }
        }
        tc5::fence_smem_to_async();
        __syncthreads();

        // ---- matched filter m_c = H_c^H y_c (every pair, one chain each) ----
        if (tid == 0) {
            tc5::fence_after_sync();
            for (int j = 0; j < npairs; ++j) {
                const uint32_t a = sbase + HT + j * HT_PAIR, b = sbase + VT + j * VT_PAIR;
                mma_k32(tbase + 64 * j, a, a + HT_LO, b, b + VT_LO, id_in, !IN16);
            }
            tc5::commit(bar_mma);
        }
        wait_mma();
        // m_c (component pp of user uu): its largest magnitude over the CTA
        // sets the state scale, then it is read again and written as the
        // state tile of the y_reg product
        auto mf_read = [&](int j, float (&m)[NS]) {
            const int c = 2 * j + cl;
            const float us = exp2i(-(eslot[c] + eslot[8 + c]));
            float a[16];
            tc5::ld_x16(tq + 64 * j + 32 * cl + 16, a);  // columns of p' = 1
            tc5::ld_wait();
#pragma unroll
            for (int n = 0; n < NS; ++n) m[n] = __shfl_xor_sync(0xffffffffu, a[n], 16);
            tc5::ld_x16(tq + 64 * j + 32 * cl, a);       // columns of p' = 0
            tc5::ld_wait();
            // Re m = D00 + D11 (lane p = 0), Im m = D01 - D10 (lane p = 1)
#pragma unroll
            for (int n = 0; n < NS; ++n) m[n] = (pp ? m[n] - a[n] : a[n] + m[n]) * us;
        };
        float mloc = 0.f;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int j = wg + 2 * r;
            if (j < npairs) {
                float m[NS];
                mf_read(j, m);
#pragma unroll
                for (int n = 0; n < NS; ++n) mloc = fmaxf(mloc, fabsf(m[n]));
            }
        }
        int ev = scale_exp(cta_max(mloc));
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int j = wg + 2 * r;
            if (j < npairs) {
                float m[NS];
                mf_read(j, m);
                put_state(j, m, exp2i(ev));
            }
        }
        tc5::fence_smem_to_async();
        tc5::fence_before_sync();
        __syncthreads();

        // ---- Gram G_c = H_c^H H_c + rho I: two rounds of two pairs -----------
        for (int rd = 0; rd < 2 && 2 * rd < npairs; ++rd) {
            if (tid == 0) {
                tc5::fence_after_sync();
                for (int g2 = 0; g2 < 2; ++g2) {
                    const int j = 2 * rd + g2;
                    if (j < npairs) {
                        const uint32_t a = sbase + HT + j * HT_PAIR;
                        mma_k32(tbase + 128 * g2, a, a + HT_LO, a, a + HT_LO, id_gram, !IN16);
                    }
                }
                tc5::commit(bar_mma);
            }
            wait_mma();
            const int j = 2 * rd + wg;
            if (j < npairs) {
                const int c = 2 * j + cl;
                const uint32_t col = tbase + ((uint32_t)(32 * q) << 16) + 128 * wg + 64 * cl;
                // columns 32h' + 16p' + i' hold component p' of user 16h' + i'
                float b1[32], b0[32];
                {
                    float x[16];
                    tc5::ld_x16(col + 16, x);
                    tc5::ld_wait();
#pragma unroll
                    for (int e = 0; e < 16; ++e) b1[e] = x[e];
                    tc5::ld_x16(col + 48, x);
                    tc5::ld_wait();
#pragma unroll
                    for (int e = 0; e < 16; ++e) b1[16 + e] = x[e];
                    tc5::ld_x16(col, x);
                    tc5::ld_wait();
#pragma unroll
                    for (int e = 0; e < 16; ++e) b0[e] = x[e];
                    tc5::ld_x16(col + 32, x);
                    tc5::ld_wait();
#pragma unroll
                    for (int e = 0; e < 16; ++e) b0[16 + e] = x[e];
                }
                const float us = exp2i(-2 * eslot[c]);
                float *plane = reinterpret_cast<float *>(sm + HT + j * HT_PAIR + cl * 8192 + pp * 4096);
#pragma unroll
                for (int ch = 0; ch < 8; ++ch) {
                    float g[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int e = 4 * ch + t;
                        const float recv = __shfl_xor_sync(0xffffffffu, b1[e], 16);
                        // Re G = D00 + D11 (p = 0), Im G = D01 - D10 (p = 1)
                        float v = (pp ? recv - b0[e] : b0[e] + recv) * us;
                        if (pp == 0 && e == uu) v += p.f_delta;
                        g[t] = v;
                    }
                    *reinterpret_cast<float4 *>(plane + uu * 32 + 4 * (ch ^ (uu & 7))) = make_float4(g[0], g[1], g[2], g[3]);
                }
            }
            tc5::fence_before_sync();
            __syncthreads();
        }
        if (*abort_flag) break;

        // ---- B_c^{-1}: Gauss-Jordan per warp, pivot check, FP64 retry --------
        if (tid == 0) reinterpret_cast<OpParams *>(sm + PARAMS)->row0 = (long long)w * B;
        __syncthreads();
        tc32_operator_phase<TIn>();
        if (warp < C && eslot[24 + warp]) {
            // FP64 retry: this cluster's Gram from the inputs in global
            // memory and its inverse, in FP64, written as the operator
            const TIn *Hg = static_cast<const TIn *>(p.H) + ((size_t)w * B + (size_t)warp * 32) * 32;
            __syncwarp();
            tc32_fp64_operator<TIn>(Hg, p.delta, reinterpret_cast<double2 *>(sm + SCR + warp * SCR_WARP),
                                    sm + HT + (warp >> 1) * HT_PAIR, warp & 1, eslot + 16 + warp, lane);
            if (lane == 0) {
                eslot[24 + warp] = 0;
                if (p.retries) atomicAdd(p.retries, 1u);
            }
        }
        tc5::fence_smem_to_async();
        __syncthreads();

        // ---- operator products: y_reg, then one per iteration ----------------
        auto issue_op = [&]() {
            if (tid == 0) {
                tc5::fence_after_sync();
                for (int j = 0; j < npairs; ++j) {
                    const uint32_t a = sbase + HT + j * HT_PAIR, b = sbase + VT + j * VT_PAIR;
                    mma_k32(tbase + 64 * j, a, a + HT_LO, b, b + VT_LO, id_op, true);
                }
                tc5::commit(bar_mma);
            }
        };
        issue_op();
        wait_mma();
        float yreg[2][NS], lam[2][NS], wsum[NS], part[NS];
#pragma unroll
        for (int n = 0; n < NS; ++n) part[n] = 0.f;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int j = wg + 2 * r;
            if (j < npairs) {
                op_read(j, exp2i(-(eslot[16 + 2 * j + cl] + ev)), yreg[r]);
            } else {
#pragma unroll
                for (int n = 0; n < NS; ++n) yreg[r][n] = 0.f;
            }
#pragma unroll
            for (int n = 0; n < NS; ++n) {
                lam[r][n] = 0.f;
                part[n] += yreg[r][n];
            }
        }
        // init: z_c = y_c^reg, lambda_c = 0, consensus and prox
        consensus(part, wsum);
        prox(wsum);
        for (int t = 2; t <= T; ++t) {
            // (E3) lambda_c += gamma (z_c - s) with z_c from the last product
            // (y_reg itself at t = 2); the state is rho (s - lambda_c)
            float mloc2 = 0.f;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int j = wg + 2 * r;
                if (j < npairs) {
                    float z[NS];
                    if (t == 2) {
#pragma unroll
                        for (int n = 0; n < NS; ++n) z[n] = yreg[r][n];
                    } else {
                        op_read(j, exp2i(-(eslot[16 + 2 * j + cl] + ev)), z);
#pragma unroll
                        for (int n = 0; n < NS; ++n) z[n] += yreg[r][n];
                    }
#pragma unroll
                    for (int n = 0; n < NS; ++n) {
                        lam[r][n] = fmaf(gam, z[n] - wsum[n], lam[r][n]);
                        mloc2 = fmaxf(mloc2, fabsf((wsum[n] - lam[r][n]) * rho));
                    }
                }
            }
            ev = scale_exp(cta_max(mloc2));      // also: every consensus read is done
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int j = wg + 2 * r;
                if (j < npairs) {
                    float v[NS];
#pragma unroll
                    for (int n = 0; n < NS; ++n) v[n] = (wsum[n] - lam[r][n]) * rho;
                    put_state(j, v, exp2i(ev));
                }
            }
            tc5::fence_smem_to_async();
            tc5::fence_before_sync();
            __syncthreads();
            issue_op();
            wait_mma();
            // (E1) z_c = y_reg + B_c^{-1} rho (s - lambda_c); w = sum_c (z_c + lambda_c)
#pragma unroll
            for (int n = 0; n < NS; ++n) part[n] = 0.f;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int j = wg + 2 * r;
                if (j < npairs) {
                    float z[NS];
                    op_read(j, exp2i(-(eslot[16 + 2 * j + cl] + ev)), z);
#pragma unroll
                    for (int n = 0; n < NS; ++n) part[n] += (z[n] + yreg[r][n]) + lam[r][n];
                }
            }
            consensus(part, wsum);
            prox(wsum);
        }
        if (*abort_flag) break;

        // ---- outputs: x_hat = s and its labels (partial group kgrp writes the
        // symbols n = kgrp mod 4; lane p = 0 pairs its real part with the
        // imaginary part of lane + 16) ---------------------------------------
        {
            float2 *xo = static_cast<float2 *>(p.out);
#pragma unroll
            for (int n = 0; n < NS; ++n) {
                const float other = __shfl_xor_sync(0xffffffffu, wsum[n], 16);
                if (pp == 0 && (n & 3) == kgrp && n < N && uu < p.U) {
                    const size_t o = ((size_t)w * N + n) * p.U + uu;
                    xo[o] = make_float2(wsum[n], other);
                    if (p.labels)
                        p.labels[o] = qam_label(wsum[n], other, p.f_qam_inv_a, p.qam_L, p.qam_half);
                }
            }
        }
        tc5::fence_smem_to_async();
        tc5::fence_before_sync();
        __syncthreads();        // every shared-memory read of this subcarrier is done
    }
    // a CTA that left early waits (bounded) for copies still in flight
    if (tid == 0 && *abort_flag) mbar_wait_bounded(bar_ld, ph_ld ^ 1u, nullptr, p.wait_iters);
    tc5::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc5::tmem_dealloc(tbase, TMEM_COLS);
}

// Eligible frames: uplink ADMM, U = S = 32, C even and <= 8, N <= 16, FP32 /
// FP16 / BF16 inputs, 16-byte aligned buffers.
inline bool tc32_eligible_shape(int B, int C, int U, int N, int prec) {
    return U == 32 && C >= 2 && C <= 8 && (C & 1) == 0 && B == 32 * C && N >= 1 && N <= 16 &&
           (prec == 0 || prec == 2 || prec == 3);
}

}  // namespace dbp
