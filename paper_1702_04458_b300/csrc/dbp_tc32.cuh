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
constexpr int SLOTS = SCR + 8 * SCR_WARP;   // scale exponents (40 ints) and warp maxima (8 floats)
constexpr int MSLOT = SLOTS + 160;
constexpr int BARS = SLOTS + 256;          // copy and CTA-MMA mbarriers, TMEM slot, abort flag; per-warp mbarriers
constexpr int BAR_OP = BARS + 64;
constexpr int SMEM = BARS + 128;
constexpr int TMEM_COLS = 256;
constexpr int PART_LD = 20;        // floats per consensus partial row (16 used, padded against bank conflicts)

// Byte offset of 16-bit element (row, k) of a K-major operand tile with 32
// contraction elements per row: 8 x 16-byte core matrices, K-direction core
// matrices 128 B apart (LBO), 8-row groups 512 B apart (SBO).
__device__ __forceinline__ int off16(int row, int k) {
    return (row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}
// Byte offset of 16-bit element (n, k) of a B operand tile with 64 rows n
// and 32 contraction elements k stored MN-major: 8 consecutive n in 16
// bytes, the 8 k of a block 16 bytes apart, 8-row blocks of n 128 B apart,
// 8-deep blocks of k 1024 B apart.  The state tiles use it: a thread holds
// one user k for all symbols n and stores them as 16-byte chunks, where the
// K-major layout took one conflicting 2-byte store per symbol.
__device__ __forceinline__ int offmn32(int n, int k) {
    return (n >> 3) * 128 + (k >> 3) * 1024 + (k & 7) * 16 + (n & 7) * 2;
}
constexpr uint32_t TRANSPOSE_B = 1u << 16;      // instruction descriptor: B MN-major
// Row of component p of user u inside a cluster's 64-row tile.
__device__ __forceinline__ int arow(int p, int u) { return 32 * (u >> 4) + 16 * p + (u & 15); }

// Power-of-two exponent e with m 2^e in [2^13, 2^14) (0 for 0 / non-finite).
__device__ __forceinline__ int scale_exp(float m) {
    if (!(m > 0.f) || !(m < 3.0e38f)) return 0;
    const int e = 14 - frexp_exponent(m);
    return e < -100 ? -100 : (e > 100 ? 100 : e);
}
__device__ __forceinline__ float exp2i(int e) { return __int_as_float((127 + e) << 23); }

template <typename T> struct Op16;
// (The conversions go through the packed two-value instructions: one of
// them costs no more than one single-value conversion, which runs at a
// fraction of the rate.)
template <> struct Op16<__half> {
    static constexpr int fmt = tc5::FMT_F16;
    static __device__ __forceinline__ uint16_t bits(float x) { return __half_as_ushort(__low2half(__floats2half2_rn(x, 0.f))); }
    static __device__ __forceinline__ uint32_t bits2(float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    static __device__ __forceinline__ float back(uint16_t b) { return __half2float(__ushort_as_half(b)); }
};
template <> struct Op16<__nv_bfloat16> {
    static constexpr int fmt = tc5::FMT_BF16;
    static __device__ __forceinline__ uint16_t bits(float x) {
        return __bfloat16_as_ushort(__low2bfloat16(__floats2bfloat162_rn(x, 0.f)));
    }
    static __device__ __forceinline__ uint32_t bits2(float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    static __device__ __forceinline__ float back(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }
};
// Operand type of the Gram / matched filter for an input type.
template <typename TIn> struct GramOp { using type = __half; };
template <> struct GramOp<__nv_bfloat162> { using type = __nv_bfloat16; };

// hi / lo FP16 split of x (already scaled), through the packed conversion
// with a zero partner (the low half is fp16(x) as a single conversion gives).
__device__ __forceinline__ void split16(float x, uint32_t &hi, uint32_t &lo) {
    const __half2 h = __floats2half2_rn(x, 0.f);
    const __half2 l = __floats2half2_rn(x - __low2float(h), 0.f);
    hi = *reinterpret_cast<const uint32_t *>(&h) & 0xffffu;
    lo = *reinterpret_cast<const uint32_t *>(&l) & 0xffffu;
}
__device__ __forceinline__ uint32_t pack2(uint32_t a, uint32_t b) { return a | (b << 16); }
// hi / lo words of a and b (already scaled) as f16x2 (a in the low half):
// the values split16 gives for each, with one conversion per pair.
__device__ __forceinline__ void split16x2(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

// D (+)= A B^T over K = 32 (two K steps of 16): A tile of 128 rows at a_hi /
// a_lo, B tile at b_hi / b_lo (shared-memory byte addresses); three products
// with the split, one (hi only) without.  The small terms (lo hi, hi lo) are
// accumulated first and hi hi last: the tensor core's FP32 accumulation
// loses bits of terms added to a larger running sum (measured on sm_103a:
// up to 5.8 units of 2^-24 sum|ab| with hi hi first, 1.8 with it last; an
// FP32 FMA chain over the same 16 terms: 2.9).
// B in K-major (B_MN false) or in the MN-major layout of offmn32 (B_MN true;
// the instruction descriptor then sets transpose B): per K step of 16, two
// 8-deep k blocks 1024 B apart (leading offset), 8-row n blocks 128 B apart
// (stride offset).
template <bool B_MN = false>
__device__ __forceinline__ void mma_k32(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo,
                                        uint32_t id, bool split) {
    auto bd = [](uint32_t b, int ks) {
        return B_MN ? tc5::sdesc(b + ks * 2048, 1024, 128) : tc5::sdesc(b + ks * 256, 128, 512);
    };
    if (split) {
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
            tc5::mma_f16(d, tc5::sdesc(a_lo + ks * 256, 128, 512), bd(b_hi, ks), id, ks > 0 ? 1u : 0u);
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
            tc5::mma_f16(d, tc5::sdesc(a_hi + ks * 256, 128, 512), bd(b_lo, ks), id, 1u);
    }
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
        tc5::mma_f16(d, tc5::sdesc(a_hi + ks * 256, 128, 512), bd(b_hi, ks), id, (split || ks > 0) ? 1u : 0u);
}

__device__ __forceinline__ float warp_max(float v) { return warp_redux_max(v); }

// Load 32 consecutive accumulator columns of this warp's lane quadrant.
__device__ __forceinline__ void ld32(uint32_t taddr, float (&a)[32]) {
    tc5::ld_x32(taddr, a);
    tc5::ld_wait();
}

}  // namespace tc32

// Gauss-Jordan inversion of the 16 x 32 block [A | R] (A HPD: no pivoting,
// every pivot is a Schur complement) into [A^{-1} | A^{-1} R], in registers:
// lane (rg, cg) = (lane / 4, lane % 4) holds rows 2 rg, 2 rg + 1 and columns
// 8 cg .. 8 cg + 7.  Two pivots per round: a lane's two rows are one pivot
// pair.  Round m takes the
// pivot block P = A[K][K] of K = {2m, 2m + 1}: every row i outside K takes
// A[i][j] -= M_i A[K][j] with M_i = A[i][K] P^{-1} (the two scalar steps of
// the pair at once) and A[i][K] = -M_i; the pair's rows are left as they
// are, with A[K][K] = I, and multiplied by P^{-1} after the last round.  The
// exchange (pivot rows and columns through shared memory) happens once per
// pair, so there are half as many rounds.  buf: 112 complex (two pivot
// rows with 80-byte groups, two pivot columns), 16-byte aligned.  Returns
// the smallest real part of the scalar pivots (P00 and its Schur complement
// P11 - P10 P01 / P00, the pivots of the one-pivot-per-step order).
__device__ __forceinline__ float gj_pair_invert(float2 (&A)[2][8], float2 *buf, int lane) {
    constexpr int CB = 8, CBP = 10;
    const int rg = lane >> 2, cg = lane & 3;
    float2 *rowb = buf;                 // [2][4 CBP]: pivot rows, group cg at CBP cg
    float2 *colb = buf + 8 * CBP;       // [2][16]: pivot columns
    float min_piv = 3.0e38f;
    float2 q00 = make_float2(1.f, 0.f), q01 = make_float2(0.f, 0.f), q10 = q01, q11 = q00;   // this pair's P^{-1}
#pragma unroll 1
    for (int blk = 0; blk < 2; ++blk) {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int m = 4 * blk + h, k = 2 * m, kk = 2 * h;
            const bool ownc = (cg == blk), ownr = (rg == m);
            if (ownc) {
                *reinterpret_cast<float4 *>(&colb[2 * rg]) =
                    make_float4(A[0][kk].x, A[0][kk].y, A[1][kk].x, A[1][kk].y);
                *reinterpret_cast<float4 *>(&colb[16 + 2 * rg]) =
                    make_float4(A[0][kk + 1].x, A[0][kk + 1].y, A[1][kk + 1].x, A[1][kk + 1].y);
            }
            if (ownr) {
#pragma unroll
                for (int e = 0; e < 2; ++e)
#pragma unroll
                    for (int c = 0; c < CB; c += 2)
                        *reinterpret_cast<float4 *>(&rowb[4 * CBP * e + CBP * cg + c]) =
                            make_float4(A[e][c].x, A[e][c].y, A[e][c + 1].x, A[e][c + 1].y);
            }
            __syncwarp();
            float2 p00, p10, p01, p11, f0[2], f1[2];
            ld2(&colb[k], p00, p10);                // column k, rows k and k + 1
            ld2(&colb[16 + k], p01, p11);           // column k + 1
            ld2(&colb[2 * rg], f0[0], f0[1]);       // my rows in column k
            ld2(&colb[16 + 2 * rg], f1[0], f1[1]);  // ... and in column k + 1
            // P^{-1} through the two scalar pivots p00 and s = p11 - p10 p01 / p00
            // (never det P, whose square leaves the FP32 range long before
            // the pivots' do): with a = p01 / p00, b = p10 / p00,
            // P^{-1} = [1/p00 + a b / s, -a / s; -b / s, 1 / s]
            const float d0 = rcp_approx(fmaf(p00.x, p00.x, p00.y * p00.y));
            const float2 i0 = make_float2(p00.x * d0, -p00.y * d0);
            const float2 a = cmul(p01, i0), b = cmul(p10, i0);
            float2 sp = p11;
            cmac(sp, make_float2(-p10.x, -p10.y), a);
            const float d1 = rcp_approx(fmaf(sp.x, sp.x, sp.y * sp.y));
            const float2 r11 = make_float2(sp.x * d1, -sp.y * d1);
            const float2 r01 = cmul(make_float2(-a.x, -a.y), r11), r10 = cmul(make_float2(-b.x, -b.y), r11);
            float2 r00 = i0;
            cmac(r00, make_float2(-r01.x, -r01.y), b);
            min_piv = fminf(min_piv, fminf(p00.x, sp.x));
            if (ownr) {
                q00 = r00;
                q01 = r01;
                q10 = r10;
                q11 = r11;
            }
            float2 n0[2], n1[2];            // -M_i (0 on the pair's own rows)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                float2 m0 = cmul(f0[r], r00), m1 = cmul(f0[r], r01);
                cmac(m0, f1[r], r10);
                cmac(m1, f1[r], r11);
                n0[r] = ownr ? make_float2(0.f, 0.f) : make_float2(-m0.x, -m0.y);
                n1[r] = ownr ? make_float2(0.f, 0.f) : make_float2(-m1.x, -m1.y);
            }
#pragma unroll
            for (int c = 0; c < CB; c += 2) {
                float2 a0, a1, b0, b1;
                ld2(&rowb[CBP * cg + c], a0, a1);
                ld2(&rowb[4 * CBP + CBP * cg + c], b0, b1);
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    cmac(A[r][c], n0[r], a0);
                    cmac(A[r][c], n1[r], b0);
                    cmac(A[r][c + 1], n0[r], a1);
                    cmac(A[r][c + 1], n1[r], b1);
                }
            }
            if (ownc) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    A[r][kk] = ownr ? make_float2(r == 0 ? 1.f : 0.f, 0.f) : n0[r];
                    A[r][kk + 1] = ownr ? make_float2(r == 1 ? 1.f : 0.f, 0.f) : n1[r];
                }
            }
            __syncwarp();       // every lane has read the buffers before the next round writes them
        }
    }
    // the pair's rows multiplied by its P^{-1}
#pragma unroll
    for (int c = 0; c < CB; ++c) {
        const float2 a0 = A[0][c], a1 = A[1][c];
        float2 x0 = cmul(q00, a0), x1 = cmul(q10, a0);
        cmac(x0, q01, a1);
        cmac(x1, q11, a1);
        A[0][c] = x0;
        A[1][c] = x1;
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
                split16x2((pc ? a.y : a.x) * sb, (pc ? b.y : b.x) * sb, hw[t], lw[t]);
            }
            const int o = off16(row, 8 * k4);
            *reinterpret_cast<uint4 *>(th + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4 *>(th + HT_LO + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
    }
}

// FP64 recomputation of one cluster's operator (whole warp): the Gram
// H_c^H H_c + delta I from the cluster block in global memory (row u per
// lane), its Gauss-Jordan inverse in FP64 (the steps of gj_invert, in the
// same order), rounded to FP32 and written as the operator tile.  Out of
// line and with rolled loops over a row kept in local memory: it runs only
// when an FP32 pivot was too small, so its code stays a few KB instead of
// the hundreds of KB an unrolled FP64 elimination takes, and its rows do
// not weigh on the kernel's registers.
template <typename TIn>
__device__ __noinline__ void tc32_fp64_operator(const TIn *Hg, double delta, double2 *scr, unsigned char *th, int clw,
                                                int *eslot, int lane) {
    double2 D[32];
#pragma unroll 1
    for (int v = 0; v < 32; ++v) {
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll 1
        for (int s = 0; s < 32; ++s) {
            const float2 hu = to_f2(Hg[s * 32 + lane]), hv = to_f2(Hg[s * 32 + v]);
            cmacc(acc, make_double2(hu.x, hu.y), make_double2(hv.x, hv.y));
        }
        if (v == lane) acc.x += delta;
        D[v] = acc;
    }
    __syncwarp();
#pragma unroll 1
    for (int k = 0; k < 32; ++k) {
        if (lane == k) {
#pragma unroll 1
            for (int j = 0; j < 32; ++j) scr[j] = D[j];
        }
        __syncwarp();
        const double2 inv = crcp(scr[k]);
        const bool me = (lane == k);
        const double2 f = me ? make_double2(-inv.x, -inv.y) : cmul(D[k], inv);
#pragma unroll 1
        for (int j = 0; j < 32; ++j) {
            if (j == k) continue;
            double2 base = me ? make_double2(0.0, 0.0) : D[j];
            cmac(base, make_double2(-f.x, -f.y), scr[j]);
            D[j] = base;
        }
        D[k] = me ? inv : make_double2(-f.x, -f.y);
        __syncwarp();
    }
    float2 R[32];
#pragma unroll
    for (int v = 0; v < 32; ++v) R[v] = make_float2((float)D[v].x, (float)D[v].y);
    tc32_put_operator(R, th, clw, eslot, lane);
}

namespace tc32 {

// ---- blocked inverse (operator phase) ------------------------------------
// Cluster c's own 8 KB while its inverse is formed: chunk 0 and chunk 1 are
// the hi and lo halves of its final operator tile (rows 64 (c & 1) .. + 63 of
// pair c / 2), so no other warp touches them.  The Gram readout leaves
// there the FP32 planes of A11, A12 and A22 and the A12 column tile; the
// operator phase reuses the A11 and A12 planes for K = 16 operand tiles and
// the planes of P = A11^{-1}.
__device__ __forceinline__ int chunk0(int c) { return HT + (c >> 1) * HT_PAIR + (c & 1) * 4096; }
__device__ __forceinline__ int chunk1(int c) { return chunk0(c) + HT_LO; }
constexpr int SLOT0 = 0, SLOT1 = 2048, SLOT_LO = 1024;     // chunk 0: A11 planes, then a tile | A12 column tile
constexpr int PL_A11 = 0;                                   // chunk 0
constexpr int PL_A22 = 0, PL_A12 = 2048, PL_IM = 1024;      // chunk 1: A22 (then S) | A12 (then P)

// Element (i, j) of a 16 x 16 FP32 plane (floats): 16-byte chunks XOR-
// swizzled by row, so a lane per row (4 x 16 B) and a 2 x 4 block per lane
// both read without bank conflicts beyond the minimum.
__device__ __forceinline__ int pl16(int i, int j) { return i * 16 + 4 * ((j >> 2) ^ (i & 3)) + (j & 3); }

// Byte offset of 16-bit element (row, k) of a K = 16 operand tile: 32-byte
// rows as two 16-byte core matrices 128 B apart (LBO), 8-row groups 256 B
// apart (SBO).  A 32-row tile is 1 KB.
__device__ __forceinline__ int offk16(int row, int k) {
    return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Complex product from a real one: D[(p, i), (p', j)] = sum_k comp_p(A'_ik)
// comp_p'(B'_jk) in lane 16 p + i, column 16 p' + j.  Lane (p, i) returns
// component p of row i of A B (PLAIN: Re = D00 - D11, Im = D01 + D10),
// of A^H B with A' = A^T (CONJ_A: Re = D00 + D11, Im = D01 - D10) or of
// A B^H with B' = B (CONJ_B: Re = D00 + D11, Im = D10 - D01), scaled by us.
enum { PLAIN = 0, CONJ_A = 1, CONJ_B = 2 };
template <int MODE>
__device__ __forceinline__ void cprod_read(uint32_t taddr, float us, int pp, float (&out)[16]) {
    float a[32];
    tc5::ld_x32(taddr, a);
    tc5::ld_wait();
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const float own = a[j], recv = __shfl_xor_sync(0xffffffffu, a[16 + j], 16);
        float v;
        if (MODE == PLAIN) v = pp ? own + recv : own - recv;
        else if (MODE == CONJ_A) v = pp ? recv - own : own + recv;
        else v = pp ? own - recv : own + recv;
        out[j] = v * us;
    }
}

// One warp's product D = A B^T over K = 16 from hi / lo tiles: three MMAs
// (lo hi, hi lo, hi hi) into the warp's 32 tensor-memory columns, completion
// on the warp's mbarrier.  `a_win` is the start of a 128-row window whose
// rows 32 m .. 32 m + 31 are the warp's A tile (m = its lane quadrant); the
// other rows are other clusters' bytes, and their products land in lanes no
// other warp reads at these columns.
__device__ __forceinline__ void issue_prod(uint32_t d, uint32_t a_win, uint32_t b_tile, uint64_t *bar) {
    constexpr uint32_t id = tc5::idesc(tc5::FMT_F16, 128, 32);
    tc5::fence_after_sync();
    const uint64_t ah = tc5::sdesc(a_win, 128, 256), al = tc5::sdesc(a_win + SLOT_LO, 128, 256);
    const uint64_t bh = tc5::sdesc(b_tile, 128, 256), bl = tc5::sdesc(b_tile + SLOT_LO, 128, 256);
    tc5::mma_f16(d, al, bh, id, 0u);       // small terms first (see mma_k32)
    tc5::mma_f16(d, ah, bl, id, 1u);
    tc5::mma_f16(d, ah, bh, id, 1u);
    tc5::commit(bar);
}

// hi / lo words of x (already scaled) as one 16-bit store each.
__device__ __forceinline__ void st_split(unsigned char *hi_tile, int off, float x) {
    uint32_t h, l;
    split16(x, h, l);
    *reinterpret_cast<uint16_t *>(hi_tile + off) = (uint16_t)h;
    *reinterpret_cast<uint16_t *>(hi_tile + SLOT_LO + off) = (uint16_t)l;
}
// A tile row from 16 values (K = 0..15): two 16-byte chunks per half.
__device__ __forceinline__ void st_row16(unsigned char *hi_tile, int row, const float (&v)[16], float sc) {
#pragma unroll
    for (int k8 = 0; k8 < 2; ++k8) {
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            split16x2(v[8 * k8 + 2 * t] * sc, v[8 * k8 + 2 * t + 1] * sc, hw[t], lw[t]);
        }
        const int o = offk16(row, 8 * k8);
        *reinterpret_cast<uint4 *>(hi_tile + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(hi_tile + SLOT_LO + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
}
__device__ __forceinline__ float absmax16(const float (&v)[16]) {
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j) m = fmaxf(m, fabsf(v[j]));
    return m;
}
__device__ __forceinline__ float absmax_blk8(const float2 (&M)[2][8]) {
    float m = 0.f;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) m = fmaxf(m, fmaxf(fabsf(M[r][c].x), fabsf(M[r][c].y)));
    return m;
}
// Rows 2 rg, 2 rg + 1, columns j0 .. j0 + 7 of a 16 x 16 complex matrix from
// its planes (re; im 256 floats further), as 2 x 8 block columns, and back.
__device__ __forceinline__ void ld_blk8(const float *re, float2 (&M)[2][8], int rg, int j0) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int i = 2 * rg + r;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const float4 x = *reinterpret_cast<const float4 *>(re + pl16(i, j0 + 4 * t));
            const float4 y = *reinterpret_cast<const float4 *>(re + 256 + pl16(i, j0 + 4 * t));
            M[r][4 * t + 0] = make_float2(x.x, y.x);
            M[r][4 * t + 1] = make_float2(x.y, y.y);
            M[r][4 * t + 2] = make_float2(x.z, y.z);
            M[r][4 * t + 3] = make_float2(x.w, y.w);
        }
    }
}
__device__ __forceinline__ void st_blk8(float *re, const float2 (&M)[2][8], int rg, int j0) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int i = 2 * rg + r;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            *reinterpret_cast<float4 *>(re + pl16(i, j0 + 4 * t)) =
                make_float4(M[r][4 * t].x, M[r][4 * t + 1].x, M[r][4 * t + 2].x, M[r][4 * t + 3].x);
            *reinterpret_cast<float4 *>(re + 256 + pl16(i, j0 + 4 * t)) =
                make_float4(M[r][4 * t].y, M[r][4 * t + 1].y, M[r][4 * t + 2].y, M[r][4 * t + 3].y);
        }
    }
}
// Rows 2 rg, 2 rg + 1 of a 2 x 8 block as the hi / lo chunk (K = k0 .. k0 + 7)
// of tile rows (p, row0 + 2 rg + r), scaled by sc.
__device__ __forceinline__ void st_chunk8(unsigned char *hi_tile, const float2 (&M)[2][8], int rg, int row0, int k0,
                                          float sc) {
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int pc = 0; pc < 2; ++pc) {
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                split16x2((pc ? M[r][2 * t].y : M[r][2 * t].x) * sc, (pc ? M[r][2 * t + 1].y : M[r][2 * t + 1].x) * sc, hw[t], lw[t]);
            }
            const int o = offk16(16 * pc + row0 + 2 * rg + r, k0);
            *reinterpret_cast<uint4 *>(hi_tile + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4 *>(hi_tile + SLOT_LO + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
}
// Component p of row i of a 16 x 16 plane pair (16 floats).
__device__ __forceinline__ void ld_row(const float *re, int pp, int i, float (&v)[16]) {
    const float *pl = re + 256 * pp;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const float4 x = *reinterpret_cast<const float4 *>(pl + pl16(i, 4 * t));
        v[4 * t] = x.x;
        v[4 * t + 1] = x.y;
        v[4 * t + 2] = x.z;
        v[4 * t + 3] = x.w;
    }
}

}  // namespace tc32

// B_c^{-1} of one cluster (whole warp) by the 2 x 2 block inverse with 16 x 16
// blocks of A = G_c + delta I (A21 = A12^H), as two eliminations and two
// tensor-core products:
//   [P | X]   = A11^{-1} [I | A12]      Gauss-Jordan on [A11 | A12]
//   S         = A22 - A12^H X           tensor cores
//   [Q | Y^H] = S^{-1} [I | X^H]        Gauss-Jordan on [S | X^H]
//   Z         = Y X^H                   tensor cores
//   A^{-1}    = [P + Z, -Y; -Y^H, Q].
// X and Y come from eliminations, not from products with the explicit
// inverses P and Q: a product with an explicit inverse of an ill-conditioned
// block leaves a residual A^{-1} A - I that grows with that block's
// condition number, while these eliminations keep it at the level of the
// 32 x 32 one (the operator is applied to vectors close to G_c s, so the
// residual is what reaches the estimate).  The pivots of the two
// eliminations are those of the 32 x 32 one, so the same pivot check
// applies.  The products run on the tensor cores, issued by the warp itself
// (FP16 hi / lo operands scaled by powers of two, FP32 accumulators), so the
// warp never waits for another.  Expects the Gram readout's planes and A12
// column tile (scale exponent e12) in the cluster's chunks.  Writes the
// operator tile (scale at *eslot_b) unless a pivot fails the check (returns
// false, writes nothing) or a wait gives up (timed_out).
__device__ __forceinline__ bool tc32_blocked_operator(int c, int e12, uint32_t sbase, uint32_t tbase,
                                                      uint64_t *bar, uint32_t &ph, const FusedParams &p,
                                                      int *eslot_b, bool &timed_out) {
    using namespace tc32;
    extern __shared__ __align__(1024) unsigned char sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rg = lane >> 2, cg = lane & 3, pp = lane >> 4, ii = lane & 15;
    const bool right = cg >= 2;                 // the lane holds columns 16.. of [A | R]
    const int j8 = 8 * (cg & 1);                // ... starting at column j8 of its 16 x 16 block
    const int m = warp & 3;
    unsigned char *c0 = sm + chunk0(c), *c1 = sm + chunk1(c);
    float *pA11 = reinterpret_cast<float *>(c0 + PL_A11), *pA22 = reinterpret_cast<float *>(c1 + PL_A22);
    float *pA12 = reinterpret_cast<float *>(c1 + PL_A12);      // later the planes of P
    float *pYH = reinterpret_cast<float *>(c0 + SLOT0);         // planes of Y^H (after the X column tile)
    unsigned char *slot0 = c0 + SLOT0, *slot1 = c0 + SLOT1;
    const uint32_t s0 = sbase + (uint32_t)chunk0(c) + SLOT0, s1 = sbase + (uint32_t)chunk0(c) + SLOT1;
    const uint32_t dcol = tbase + 32u * (uint32_t)warp;                      // the warp's columns
    const uint32_t dread = dcol + ((uint32_t)(32 * m) << 16);                // ... in its lane quadrant
    float2 *scr = reinterpret_cast<float2 *>(sm + SCR + warp * SCR_WARP);

    // Issue the product (A window at a_tile - m KB) and wait for it.
    auto run = [&](uint32_t a_tile, uint32_t b_tile) -> bool {
        tc5::fence_smem_to_async();
        tc5::fence_before_sync();
        __syncwarp();
        if (lane == 0) issue_prod(dcol, a_tile - 1024u * (uint32_t)m, b_tile, bar);
        __syncwarp();
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar, ph, p.status));
        ph ^= 1u;
        tc5::fence_after_sync();
        return ok;
    };

    // largest diagonal entry of A (both blocks)
    const float dmax = warp_max((lane < 16 ? pA11 : pA22)[pl16(ii, ii)]);
    // M = [A11 | A12] -> [P | X] (pass 0), then [S | X^H] -> [Q | Y^H]
    // (pass 1): one copy of the elimination's code serves both (a smaller
    // kernel for the instruction caches; measured faster in FP32 and FP16).
    float2 M[2][8];
    ld_blk8(right ? pA12 : pA11, M, rg, j8);
    float mp = 3.0e38f;
    int eX = 0;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        __syncwarp();
        mp = fminf(mp, gj_pair_invert(M, scr, lane));
        if (pass == 1) break;
        // P as FP32 planes (for B11); X as the B operand of A12^H X: rows
        // (p', j) hold comp_p'(X_kj), K = k (a column of X per row: 2-byte
        // stores)
        eX = scale_exp(warp_max(right ? absmax_blk8(M) : 0.f));
        const float sX = exp2i(eX);
        if (!right) {
            st_blk8(pA12, M, rg, j8);
        } else {
            // rows k = 2 rg and 2 rg + 1 of a column are adjacent 16-bit
            // entries: one 32-bit store per pair
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
                const int j = j8 + cc;
#pragma unroll
                for (int pc = 0; pc < 2; ++pc) {
                    uint32_t hw, lw;
                    split16x2((pc ? M[0][cc].y : M[0][cc].x) * sX, (pc ? M[1][cc].y : M[1][cc].x) * sX, hw, lw);
                    const int o = offk16(16 * pc + j, 2 * rg);
                    *reinterpret_cast<uint32_t *>(slot0 + o) = hw;
                    *reinterpret_cast<uint32_t *>(slot0 + SLOT_LO + o) = lw;
                }
            }
        }
        // S = A22 - A12^H X
        if (!run(s1, s0)) { timed_out = true; return false; }
        {
            float sv[16], a22[16];
            cprod_read<CONJ_A>(dread, exp2i(-(e12 + eX)), pp, sv);
            ld_row(pA22, pp, ii, a22);
#pragma unroll
            for (int t = 0; t < 4; ++t)
                *reinterpret_cast<float4 *>(pA22 + 256 * pp + pl16(ii, 4 * t)) =
                    make_float4(a22[4 * t] - sv[4 * t], a22[4 * t + 1] - sv[4 * t + 1],
                                a22[4 * t + 2] - sv[4 * t + 2], a22[4 * t + 3] - sv[4 * t + 3]);
        }
        // X as the B operand of Y X^H (rows (p, i) hold comp_p(X_ik), K = k),
        // where the A12 tile was
        if (right) st_chunk8(slot1, M, rg, 0, j8, sX);
        __syncwarp();
        // [S | X^H]: S from its planes; X^H_ki = conj(X_ik) from the X column
        // tile (row k, K = i: the same rounded X the product above used)
        if (!right) {
            ld_blk8(pA22, M, rg, j8);
        } else {
            const float us = exp2i(-eX);
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                float v[2][8];
#pragma unroll
                for (int pc = 0; pc < 2; ++pc) {
                    const int o = offk16(16 * pc + 2 * rg + r, j8);
                    const uint4 h = *reinterpret_cast<const uint4 *>(slot0 + o);
                    const uint4 l = *reinterpret_cast<const uint4 *>(slot0 + SLOT_LO + o);
                    const uint32_t hw[4] = {h.x, h.y, h.z, h.w}, lw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const float2 hf = __half22float2(*reinterpret_cast<const __half2 *>(&hw[t]));
                        const float2 lf = __half22float2(*reinterpret_cast<const __half2 *>(&lw[t]));
                        v[pc][2 * t] = (hf.x + lf.x) * us;
                        v[pc][2 * t + 1] = (hf.y + lf.y) * us;
                    }
                }
#pragma unroll
                for (int cc = 0; cc < 8; ++cc) M[r][cc] = make_float2(v[0][cc], -v[1][cc]);
            }
        }
    }
    float2 (&N2)[2][8] = M;                                     // [Q | Y^H]

    // Y^H through FP32 planes, so that lane (p, i) holds row i of Y
    if (right) st_blk8(pYH, N2, rg, j8);
    __syncwarp();
    float yv[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const float h = pYH[256 * pp + pl16(k, ii)];
        yv[k] = pp ? -h : h;                                    // comp_p(Y_ik) = comp_p(conj(Y^H_ki))
    }
    __syncwarp();
    const int eY = scale_exp(warp_max(absmax16(yv)));
    st_row16(slot0, 16 * pp + ii, yv, exp2i(eY));
    // Z = Y X^H;  B11 = P + Z
    if (!run(s0, s1)) { timed_out = true; return false; }
    float bv[16];
    {
        float pv[16];
        cprod_read<CONJ_B>(dread, exp2i(-(eY + eX)), pp, bv);
        ld_row(pA12, pp, ii, pv);
#pragma unroll
        for (int j = 0; j < 16; ++j) bv[j] += pv[j];
    }
    if (!(mp >= 0x1p-12f * dmax)) return false;                // FP64 retry

    // The operator tile: rows 64 (c & 1) + arow(p, u), K = v (two 16-byte
    // chunks per 8 columns), one scale for the whole inverse.
    const int eB = scale_exp(warp_max(fmaxf(fmaxf(absmax16(bv), absmax16(yv)), absmax_blk8(N2))));
    if (lane == 0) *eslot_b = eB;
    const float sB = exp2i(eB);
    __syncwarp();        // every lane has read the planes the tile overwrites
    unsigned char *th = sm + HT + (c >> 1) * HT_PAIR;
    const int rbase = 64 * (c & 1);
    // rows u = i < 16: [B11 | -Y] (component pp)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
#pragma unroll
        for (int k8 = 0; k8 < 2; ++k8) {
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const float xa = half ? -yv[8 * k8 + 2 * t] : bv[8 * k8 + 2 * t];
                const float xb = half ? -yv[8 * k8 + 2 * t + 1] : bv[8 * k8 + 2 * t + 1];
                split16x2(xa * sB, xb * sB, hw[t], lw[t]);
            }
            const int o = off16(rbase + arow(pp, ii), 16 * half + 8 * k8);
            *reinterpret_cast<uint4 *>(th + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4 *>(th + HT_LO + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
    }
    // rows u = 16 + k: [-Y^H | Q] from the second elimination's blocks
    {
        const float sg = right ? -sB : sB;
        const int k0 = right ? j8 : 16 + j8;
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int pc = 0; pc < 2; ++pc) {
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    split16x2((pc ? N2[r][2 * t].y : N2[r][2 * t].x) * sg, (pc ? N2[r][2 * t + 1].y : N2[r][2 * t + 1].x) * sg, hw[t], lw[t]);
                }
                const int o = off16(rbase + arow(pc, 16 + 2 * rg + r), k0);
                *reinterpret_cast<uint4 *>(th + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4 *>(th + HT_LO + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
    }
    return true;
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
    // eH[8] | eY[8] | eB[8] | retry flags[8] | e12[8]
    int *eslot = reinterpret_cast<int *>(sm + SLOTS);
    float *mslot = reinterpret_cast<float *>(sm + MSLOT);      // per-warp maxima
    uint64_t *bar_op = reinterpret_cast<uint64_t *>(sm + BAR_OP) + warp;   // this warp's products

    if (tid == 0) {
        mbar_init(bar_ld, 1);
        mbar_init(bar_mma, 1);
        for (int k = 0; k < 8; ++k) mbar_init(reinterpret_cast<uint64_t *>(sm + BAR_OP) + k, 1);
        *abort_flag = 0;
        for (int k = 0; k < 8; ++k) eslot[24 + k] = 0;
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

    uint32_t ph_ld = 0, ph_mma = 0, ph_op = 0;
    const uint32_t hbytes = (uint32_t)B * 32u * EB;            // H[w]: B rows x U = 32
    const uint32_t ybytes = (uint32_t)N * (uint32_t)B * EB;    // y[w]: N rows x B
    // staged y rows 16 bytes apart beyond their length where they fit the
    // region: the conversion's lanes read 8 rows at one column, which with
    // 2 KB rows all fall in one bank
    const uint32_t yrow = (uint32_t)B * EB;
    const uint32_t ypitch = ((uint32_t)N * (yrow + 16u) <= (uint32_t)(SCR - VT)) ? yrow + 16u : yrow;
    const uint32_t id_in = tc5::idesc(Op16<GOp>::fmt, 128, 64);     // matched filter
    const uint32_t id_gram = tc5::idesc(Op16<GOp>::fmt, 128, 128);  // Gram
    const uint32_t id_op = tc5::idesc(tc5::FMT_F16, 128, 64) | TRANSPOSE_B;   // operator x state (MN-major)
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
    // V_c (B operand, MN-major: rows n' = 32 cl + 16 p' + n, K = user) for
    // pair j, scaled by 2^ev, as one 16-byte chunk per 8 symbols and half.
    auto put_state = [&](int j, const float (&v)[NS], float sv) {
        unsigned char *base = sm + VT + j * VT_PAIR;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int n = 8 * h + 2 * t;
                float xa = 0.f, xb = 0.f;        // (0 splits into 0 and 0)
                if (n < NS && n < N) xa = v[n] * sv;
                if (n + 1 < NS && n + 1 < N) xb = v[n + 1] * sv;
                split16x2(xa, xb, hw[t], lw[t]);
            }
            const int o = offmn32(32 * cl + 16 * pp + 8 * h, uu);
            *reinterpret_cast<uint4 *>(base + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4 *>(base + VT_LO + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
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
            const unsigned char *ysrc = static_cast<const unsigned char *>(p.vin) + (size_t)w * ybytes;
            if (ypitch == yrow) {
                bulk_g2s(sm + VT, ysrc, ybytes, bar_ld);
            } else {
                for (int n = 0; n < N; ++n) bulk_g2s(sm + VT + n * ypitch, ysrc + (size_t)n * yrow, yrow, bar_ld);
            }
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
            // 16-bit inputs go into the tiles as they are (their exponent is
            // 0): the raw (re, im) words, rearranged by byte permutes
            float2 hv[16];
            uint32_t hr[16];
            float mh = 0.f;
            if (c < C) {
                const TIn *Hc = reinterpret_cast<const TIn *>(sm + HT + HRAW) + (size_t)c * 32 * 32;
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    if constexpr (IN16) {
                        hr[s] = *reinterpret_cast<const uint32_t *>(&Hc[(sh16 + s) * 32 + lane]);
                    } else {
                        hv[s] = to_f2(Hc[(sh16 + s) * 32 + lane]);
                        mh = fmaxf(mh, fmaxf(fabsf(hv[s].x), fabsf(hv[s].y)));
                    }
                }
            }
            if constexpr (!IN16) {
                mh = warp_max(mh);
                if (lane == 0) mslot[warp] = mh;
            }
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
                            if constexpr (IN16) {
                                // low halves (re) or high halves (im) of two words
                                hw[t] = __byte_perm(hr[8 * k2 + 2 * t], hr[8 * k2 + 2 * t + 1], pc ? 0x7632 : 0x5410);
                                lw[t] = 0;
                            } else {
                                const float2 a = hv[8 * k2 + 2 * t], b = hv[8 * k2 + 2 * t + 1];
                                split16x2((pc ? a.y : a.x) * sh, (pc ? b.y : b.x) * sh, hw[t], lw[t]);
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
            uint32_t yr[2][8];  // ... as raw words (16-bit inputs)
            float my = 0.f;
            if (warp < C) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int n = n8 + 8 * r;
                    const TIn *Y = reinterpret_cast<const TIn *>(sm + VT + n * ypitch) + warp * 32 + 8 * kc;
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        if constexpr (IN16) {
                            yr[r][t] = (n < N) ? *reinterpret_cast<const uint32_t *>(&Y[t]) : 0u;
                        } else {
                            yv[r][t] = (n < N) ? to_f2(Y[t]) : make_float2(0.f, 0.f);
                            my = fmaxf(my, fmaxf(fabsf(yv[r][t].x), fabsf(yv[r][t].y)));
                        }
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
                            if constexpr (IN16) {
                                hw[t] = __byte_perm(yr[r][2 * t], yr[r][2 * t + 1], pc ? 0x7632 : 0x5410);
                                lw[t] = 0;
                            } else {
                                const float2 a = yv[r][2 * t], b = yv[r][2 * t + 1];
                                split16x2((pc ? a.y : a.x) * sy, (pc ? b.y : b.x) * sy, hw[t], lw[t]);
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
            float a1[16], a[16];
            tc5::ld_x16(tq + 64 * j + 32 * cl + 16, a1);  // columns of p' = 1
            tc5::ld_x16(tq + 64 * j + 32 * cl, a);        // columns of p' = 0
            tc5::ld_wait();
#pragma unroll
            for (int n = 0; n < NS; ++n) m[n] = __shfl_xor_sync(0xffffffffu, a1[n], 16);
            // Re m = D00 + D11 (lane p = 0), Im m = D01 - D10 (lane p = 1)
#pragma unroll
            for (int n = 0; n < NS; ++n) m[n] = (pp ? m[n] - a[n] : a[n] + m[n]) * us;
        };
        float mloc = 0.f;
#pragma unroll 1
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
#pragma unroll 1
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
        // (This loop, and the pair loops of the matched-filter readout, stay
        // rolled: the kernel is bound by instruction fetch, and unrolled they
        // doubled their code; measured 670 against 739 us per FP32 frame.)
#pragma unroll 1
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
                    // the four loads in flight together, one wait
                    float x0[16], x1[16], x2[16], x3[16];
                    tc5::ld_x16(col + 16, x0);
                    tc5::ld_x16(col + 48, x1);
                    tc5::ld_x16(col, x2);
                    tc5::ld_x16(col + 32, x3);
                    tc5::ld_wait();
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        b1[e] = x0[e];
                        b1[16 + e] = x1[e];
                        b0[e] = x2[e];
                        b0[16 + e] = x3[e];
                    }
                }
                const float us = exp2i(-2 * eslot[c]);
                float g[32];
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    const float recv = __shfl_xor_sync(0xffffffffu, b1[e], 16);
                    // Re G = D00 + D11 (p = 0), Im G = D01 - D10 (p = 1)
                    float v = (pp ? recv - b0[e] : b0[e] + recv) * us;
                    if (pp == 0 && e == uu) v += p.f_delta;
                    g[e] = v;
                }
                // The blocks of A = G_c + rho I the blocked inverse needs, in
                // the cluster's own chunks: A11, A12 and A22 as FP32 planes,
                // A12 also as the column tile (rows (p', j) hold
                // comp_p'(A12_kj), K = k).
                const int i16 = uu & 15;
                float *plA = reinterpret_cast<float *>(uu < 16 ? sm + chunk0(c) + PL_A11 + pp * PL_IM
                                                               : sm + chunk1(c) + PL_A22 + pp * PL_IM);
                const int eA = uu < 16 ? 0 : 16;
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    *reinterpret_cast<float4 *>(plA + pl16(i16, 4 * t)) =
                        make_float4(g[eA + 4 * t], g[eA + 4 * t + 1], g[eA + 4 * t + 2], g[eA + 4 * t + 3]);
                if (uu < 16) {      // warp-uniform: q even holds rows 0..15
                    float *pl12 = reinterpret_cast<float *>(sm + chunk1(c) + PL_A12 + pp * PL_IM);
                    float m12 = 0.f;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        *reinterpret_cast<float4 *>(pl12 + pl16(i16, 4 * t)) =
                            make_float4(g[16 + 4 * t], g[17 + 4 * t], g[18 + 4 * t], g[19 + 4 * t]);
                        m12 = fmaxf(m12, fmaxf(fmaxf(fabsf(g[16 + 4 * t]), fabsf(g[17 + 4 * t])),
                                               fmaxf(fabsf(g[18 + 4 * t]), fabsf(g[19 + 4 * t]))));
                    }
                    const int e12 = scale_exp(warp_max(m12));
                    if (lane == 0) eslot[32 + c] = e12;
                    const float s12 = exp2i(e12);
                    unsigned char *t12 = sm + chunk0(c) + SLOT1;
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) st_split(t12, offk16(16 * pp + jj, i16), g[16 + jj] * s12);
                }
            }
            tc5::fence_smem_to_async();
            tc5::fence_before_sync();
            __syncthreads();
        }
        if (*abort_flag) break;

        // ---- B_c^{-1}: blocked inverse per warp, pivot check, FP64 retry -----
        if (warp < C) {
            bool timed_out = false;
            if (!tc32_blocked_operator(warp, eslot[32 + warp], sbase, tbase, bar_op, ph_op, p, eslot + 16 + warp,
                                       timed_out)) {
                if (timed_out) *abort_flag = 1;
                else if (lane == 0) eslot[24 + warp] = 1;
            }
            __syncwarp();
        }
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
        tc5::fence_before_sync();
        __syncthreads();
        if (*abort_flag) break;

        // ---- operator products: y_reg, then one per iteration ----------------
        auto issue_op = [&]() {
            if (tid == 0) {
                tc5::fence_after_sync();
                for (int j = 0; j < npairs; ++j) {
                    const uint32_t a = sbase + HT + j * HT_PAIR, b = sbase + VT + j * VT_PAIR;
                    mma_k32<true>(tbase + 64 * j, a, a + HT_LO, b, b + VT_LO, id_op, true);
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
            for (int j = 0; j < (NS + 3) / 4; ++j) {
                // kgrp is the same across the warp: pick wsum[4j + kgrp]
                float v = wsum[4 * j];
#pragma unroll
                for (int k = 1; k < 4; ++k)
                    if (4 * j + k < NS && kgrp == k) v = wsum[4 * j + k];
                const float other = __shfl_xor_sync(0xffffffffu, v, 16);
                const int n = 4 * j + kgrp;
                if (pp == 0 && n < N && uu < p.U) {
                    const size_t o = ((size_t)w * N + n) * p.U + uu;
                    xo[o] = make_float2(v, other);
                    if (p.labels)
                        p.labels[o] = qam_label(v, other, p.f_qam_inv_a, p.qam_L, p.qam_half);
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
