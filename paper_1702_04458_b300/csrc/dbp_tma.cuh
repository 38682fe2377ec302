// dbp_tma.cuh -- persistent, bulk-copy-fed fused kernel for the common shapes
// (U a power of two, an even cluster size S <= 64, all C warps of a
// subcarrier in one CTA), for FP32 inputs and for FP16 / BF16 inputs.
//
// Same per-(subcarrier, cluster) warp mapping and the same FP32 arithmetic
// as dbp_fused_kernel, with these structural changes:
//  * staging: each warp copies its cluster block H_c and its N receive rows
//    y_c[n] into shared memory with bulk asynchronous copies (cp.async.bulk,
//    completion on an mbarrier), double-buffered: the CTA is persistent and
//    the copies of the next subcarrier are in flight while the current one
//    computes;
//  * FP16 / BF16 inputs: the two contractions with the channel, the Gram
//    H_c^H H_c and the matched filter H_c^H y_c, run on the tensor cores
//    (mma.sync m16n8k16, FP32 accumulation; every product of two 16-bit
//    inputs is exact in FP32).  The complex product is embedded in a real
//    one with real/imaginary parts interleaved along the contraction, so
//    that every A and B fragment is one 32-bit shared-memory load of a
//    stored complex value (or its 90-degree rotation);
//  * every Gauss-Jordan pivot is checked: a pivot below 2^-12 of the
//    largest diagonal entry means FP32 has lost at least 12 bits, and that
//    cluster's Gram and inverse are recomputed in FP64 (counted on the
//    device, read back with dbp_fp64_retries);
//  * consensus in two phases: every warp publishes w_c, each warp then sums
//    a 1/C slice of the entries over all C clusters (in cluster order) and
//    publishes the sums, and every warp reads back its own entries -- the
//    fusion node's gather/sum/broadcast, spread over the C processing
//    elements;
//  * the equaliser outputs and labels are written by all C warps (each warp
//    a share of the symbols), since every warp holds the same consensus.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dbp_fused.cuh"

namespace dbp {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while the previous kernel of its stream is still
// running; grid_dependency_wait() blocks until that kernel has completed and
// its memory is visible (a no-op for an ordinary launch), so every global
// access of the kernels comes after it and only the set-up overlaps.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" :::); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for one mbarrier phase: after `limit` polls (default 2^23,
// ~0.5 s) the wait gives up, raises bit 0 of *status and the kernel carries
// on with whatever the buffer holds (the host reports DBP_ERR_TIMEOUT), so
// no wait can hang.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *status, int limit = 0) {
    const int lim = limit > 0 ? limit : (1 << 23);
    for (int i = 0; i < lim; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i >= 32) __nanosleep(64);
    }
    if (status) atomicOr(status, 1);
    return false;
}

// ---------------------------------------------------------------------------
// Input element types.
// ---------------------------------------------------------------------------
template <typename TIn> struct InTraits;
template <> struct InTraits<float2> { static constexpr int bytes = 8; static constexpr bool mma = false; };
template <> struct InTraits<__half2> { static constexpr int bytes = 4; static constexpr bool mma = true; };
template <> struct InTraits<__nv_bfloat162> { static constexpr int bytes = 4; static constexpr bool mma = true; };

__device__ __forceinline__ float2 to_f2(float2 v) { return v; }
__device__ __forceinline__ float2 to_f2(__half2 v) { return __half22float2(v); }
__device__ __forceinline__ float2 to_f2(__nv_bfloat162 v) { return __bfloat1622float2(v); }

// ---------------------------------------------------------------------------
// Tensor-core helpers for 16-bit inputs.
// ---------------------------------------------------------------------------
template <typename TIn>
__device__ __forceinline__ void mma_k16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                        uint32_t b0, uint32_t b1);
template <>
__device__ __forceinline__ void mma_k16<__half2>(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                                 uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
template <>
__device__ __forceinline__ void mma_k16<__nv_bfloat162>(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                                        uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// FP32 accuracy from TF32 tensor cores (the U = 8 tensor-core kernel and the
// FP32 Gram / matched filter here): every operand x is split into two TF32
// values x_hi + x_lo (truncated, |x - x_hi - x_lo| < 2^-20 |x|) and a product
// is accumulated as a_lo b_hi + a_hi b_lo + a_hi b_hi in FP32 (the a_lo b_lo
// term, < 2^-20 relative, is dropped): three mma.sync.m16n8k8.tf32 per
// product.
__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
// x = hi + lo + r with hi, lo TF32 values: hi keeps the 10 leading mantissa
// bits of x (truncation), lo those of the exact remainder x - hi, and
// |r| < 2^-20 |x|.
__device__ __forceinline__ void split3(float x, uint32_t &hi, uint32_t &lo) {
    hi = __float_as_uint(x) & 0xffffe000u;
    lo = __float_as_uint(x - __uint_as_float(hi)) & 0xffffe000u;
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

// A fragment of H_c^H for one k-step of the complex embedding (complex rows
// s0..s0+3 of H_c, row pitch hp): lane (g, t) takes H[s0 + t/2][user] and
// H[s0 + 2 + t/2][user], component t & 1 for the real rows and the matching
// component of the rotation (-Im, Re) for the imaginary rows.
__device__ __forceinline__ void hh_frag_p(const float2 *Hs, int hp, int s0, int user, int t, float (&a)[4]) {
    const float2 h0 = Hs[(s0 + (t >> 1)) * hp + user];
    const float2 h1 = Hs[(s0 + 2 + (t >> 1)) * hp + user];
    const bool odd = t & 1;
    a[0] = odd ? h0.y : h0.x;
    a[1] = odd ? h0.x : -h0.y;
    a[2] = odd ? h1.y : h1.x;
    a[3] = odd ? h1.x : -h1.y;
}

// (re, im) -> (-im, re) for a packed pair of 16-bit values (sign bit 15 of
// the low half; the same layout for FP16 and BF16).
__device__ __forceinline__ uint32_t rot16(uint32_t h) { return __byte_perm(h, 0, 0x1032) ^ 0x8000u; }

// Complex C = H_c^H B on the tensor cores.  With k' = 2s + a (a = re, im),
//   Re C[u][n] = sum_k' Are[u][k'] B'[k'][n],  Im C[u][n] = sum_k' Aim[u][k'] B'[k'][n],
//   Are[u][2s:2s+2] = H[s][u] (as stored),  Aim[u][2s:2s+2] = rot(H[s][u]),
//   B'[2s:2s+2][n] = B[s][n] (as stored).
// An m16 tile stacks the real rows of 8 users over their imaginary rows, so
// the D fragment gives each lane whole complex results: lane (g, t) gets
// C[8mt+g][8nt+2t] = (d0, d2) and C[8mt+g][8nt+2t+1] = (d1, d3).
// Gram: B = H_c.  The D fragments go through the row buffer G[16][UT+2]
// (float2), 16 matrix rows per pass, and lane (u, g) picks up row u into R.
template <int UT, typename TIn>
__device__ __forceinline__ void gram_mma(const uint32_t *Hs, int hp, int h_rows, float2 *G, int lane, int u,
                                         float2 (&R)[UT]) {
    constexpr int MT = (UT >= 8) ? UT / 8 : 1;
    constexpr int LD = UT + 2;
    constexpr int PASSES = (UT > 16) ? UT / 16 : 1;
    constexpr int MPP = MT / PASSES;   // m-tiles per pass
    const int g = lane >> 2, t = lane & 3;
    float acc[MT][MT][4];
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < MT; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    for (int s0 = 0; s0 < h_rows; s0 += 8) {
        uint32_t h0[MT], h1[MT];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            const int uu = 8 * mt + g;
            h0[mt] = (uu < UT) ? Hs[(s0 + t) * hp + uu] : 0u;
            h1[mt] = (uu < UT) ? Hs[(s0 + t + 4) * hp + uu] : 0u;
        }
        // only the blocks on and above the diagonal (the Gram is Hermitian)
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            const uint32_t r0 = rot16(h0[mt]), r1 = rot16(h1[mt]);
#pragma unroll
            for (int nt = mt; nt < MT; ++nt) mma_k16<TIn>(acc[mt][nt], h0[mt], r0, h1[mt], r1, h0[nt], h1[nt]);
        }
    }
#pragma unroll
    for (int pass = 0; pass < PASSES; ++pass) {
#pragma unroll
        for (int m = 0; m < MPP; ++m) {
            const int mt = pass * MPP + m;
            const int row = 8 * m + g;          // row within this pass
#pragma unroll
            for (int nt = 0; nt < MT; ++nt) {
                const int v = 8 * nt + 2 * t;
                if (nt >= mt) {
                    if (8 * mt + g < UT && v < UT)
                        *reinterpret_cast<float4 *>(&G[row * LD + v]) =
                            make_float4(acc[mt][nt][0], acc[mt][nt][2], acc[mt][nt][1], acc[mt][nt][3]);
                } else {
                    // block (mt, nt) = conjugate transpose of block (nt, mt): this
                    // lane holds G[8 nt + g][8 mt + 2t + q]
#pragma unroll
                    for (int q = 0; q < 2; ++q)
                        if (8 * mt + 2 * t + q < UT && 8 * nt + g < UT)
                            G[(8 * m + 2 * t + q) * LD + 8 * nt + g] =
                                make_float2(acc[nt][mt][q], -acc[nt][mt][2 + q]);
                }
            }
        }
        __syncwarp();
        if (u / 16 == pass) {
#pragma unroll
            for (int v = 0; v < UT; v += 2) ld2(&G[(u - 16 * pass) * LD + v], R[v], R[v + 1]);
        }
        __syncwarp();
    }
}

// Matched filter: B[s][n] = y_c[n][s] (receive rows staged as Ys[n][yp]);
// results stored symbol-major into M[n][UT+2] (float2), all N symbols.
template <int UT, typename TIn>
__device__ __forceinline__ void mf_mma(const uint32_t *Hs, int hp, int h_rows, const uint32_t *Ys, int yp,
                                       int n_tiles, float2 *M, int lane) {
    constexpr int MT = (UT >= 8) ? UT / 8 : 1;
    constexpr int LD = UT + 2;
    const int g = lane >> 2, t = lane & 3;
    for (int nb = 0; nb < n_tiles; nb += 2) {
        float acc[MT][2][4];
#pragma unroll
        for (int i = 0; i < MT; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
        const bool two = (nb + 1 < n_tiles);
        for (int s0 = 0; s0 < h_rows; s0 += 8) {
            uint32_t b0[2], b1[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int n = 8 * (nb + q) + g;
                b0[q] = (q == 0 || two) ? Ys[n * yp + s0 + t] : 0u;
                b1[q] = (q == 0 || two) ? Ys[n * yp + s0 + t + 4] : 0u;
            }
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                const int uu = 8 * mt + g;
                const uint32_t h0 = (uu < UT) ? Hs[(s0 + t) * hp + uu] : 0u;
                const uint32_t h1 = (uu < UT) ? Hs[(s0 + t + 4) * hp + uu] : 0u;
                const uint32_t r0 = rot16(h0), r1 = rot16(h1);
                mma_k16<TIn>(acc[mt][0], h0, r0, h1, r1, b0[0], b1[0]);
                if (two) mma_k16<TIn>(acc[mt][1], h0, r0, h1, r1, b0[1], b1[1]);
            }
        }
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            const int uu = 8 * mt + g;
            if (uu >= UT) continue;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (q == 1 && !two) continue;
                const int n = 8 * (nb + q) + 2 * t;
                M[n * LD + uu] = make_float2(acc[mt][q][0], acc[mt][q][2]);
                M[(n + 1) * LD + uu] = make_float2(acc[mt][q][1], acc[mt][q][3]);
            }
        }
    }
}

// FP32 inputs at U = 32: the Gram and the matched filter run on the tensor
// cores (three TF32 products per k-step) instead of the CUDA cores.
template <int UT, typename TIn> struct FP32Mma {
    static constexpr bool value = (UT == 32) && !InTraits<TIn>::mma;
};

// The same two products from FP32 inputs, on the tensor cores with three
// TF32 products per k-step (dbp_mma8.cuh's embedding: A_re[u][2s:2s+2] =
// H[s][u] as stored, A_im = (-Im, Re) of it, B'[2s:2s+2][n] = B[s][n] as
// stored; m16n8k8, four complex rows per k-step).  Output paths as gram_mma
// and mf_mma.
// Accumulates the Gram's blocks on and above the diagonal (the Gram is
// Hermitian) over rows 0 .. h_rows - 1 of Hs (pitch hp; h_rows a multiple
// of 4) into acc, which the caller zeroes; calls may continue one sum over
// several row blocks.
template <int UT>
__device__ __forceinline__ void gram_mma3_acc(const float2 *Hs, int hp, int h_rows, int lane,
                                              float (&acc)[UT / 8][UT / 8][4]) {
    constexpr int MT = UT / 8;
    const int g = lane >> 2, t = lane & 3;
    for (int s0 = 0; s0 < h_rows; s0 += 4) {
        uint32_t ah[MT][4], al[MT][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            float a[4];
            hh_frag_p(Hs, hp, s0, 8 * mt + g, t, a);
#pragma unroll
            for (int i = 0; i < 4; ++i) split3(a[i], ah[mt][i], al[mt][i]);
        }
        // the B fragment of H_c for n-tile nt holds the values a[0], a[2] of
        // m-tile nt
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = mt; nt < MT; ++nt)
                mma3(acc[mt][nt], ah[mt], al[mt], ah[nt][0], ah[nt][2], al[nt][0], al[nt][2]);
    }
}

// Writes the Gram accumulated by gram_mma3_acc through the row buffer G
// (16 rows of pitch UT + 2) and returns row u in R (lane u); the blocks
// below the diagonal are the conjugate transposes of those above it.
template <int UT>
__device__ __forceinline__ void gram_mma3_rows(const float (&acc)[UT / 8][UT / 8][4], float2 *G, int lane, int u,
                                               float2 (&R)[UT]) {
    constexpr int MT = UT / 8;
    constexpr int LD = UT + 2;
    constexpr int PASSES = (UT > 16) ? UT / 16 : 1;
    constexpr int MPP = MT / PASSES;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int pass = 0; pass < PASSES; ++pass) {
#pragma unroll
        for (int m = 0; m < MPP; ++m) {
            const int mt = pass * MPP + m;
            const int row = 8 * m + g;
#pragma unroll
            for (int nt = 0; nt < MT; ++nt) {
                if (nt >= mt) {
                    *reinterpret_cast<float4 *>(&G[row * LD + 8 * nt + 2 * t]) =
                        make_float4(acc[mt][nt][0], acc[mt][nt][2], acc[mt][nt][1], acc[mt][nt][3]);
                } else {
                    // block (mt, nt) = conjugate transpose of block (nt, mt): this
                    // lane holds G[8 nt + g][8 mt + 2t + q]
#pragma unroll
                    for (int q = 0; q < 2; ++q)
                        G[(8 * m + 2 * t + q) * LD + 8 * nt + g] = make_float2(acc[nt][mt][q], -acc[nt][mt][2 + q]);
                }
            }
        }
        __syncwarp();
        if (u / 16 == pass) {
#pragma unroll
            for (int v = 0; v < UT; v += 2) ld2(&G[(u - 16 * pass) * LD + v], R[v], R[v + 1]);
        }
        __syncwarp();
    }
}

template <int UT>
__device__ __forceinline__ void gram_mma3(const float2 *Hs, int hp, int h_rows, float2 *G, int lane, int u,
                                          float2 (&R)[UT]) {
    constexpr int MT = UT / 8;
    float acc[MT][MT][4];
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < MT; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    gram_mma3_acc<UT>(Hs, hp, h_rows, lane, acc);
    gram_mma3_rows<UT>(acc, G, lane, u, R);
}

template <int UT>
__device__ __forceinline__ void mf_mma3(const float2 *Hs, int hp, int h_rows, const float2 *Ys, int yp, int n_tiles,
                                        float2 *M, int lane) {
    constexpr int MT = UT / 8;
    constexpr int LD = UT + 2;
    const int g = lane >> 2, t = lane & 3;
    const float *Yf = reinterpret_cast<const float *>(Ys);
    for (int nb = 0; nb < n_tiles; nb += 2) {
        const bool two = (nb + 1 < n_tiles);
        float acc[MT][2][4];
#pragma unroll
        for (int i = 0; i < MT; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
        for (int s0 = 0; s0 < h_rows; s0 += 4) {
            uint32_t bh0[2], bl0[2], bh1[2], bl1[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                // B'[k' = t][n] and B'[t + 4][n]: component t & 1 of y[n][s0 + t/2], y[n][s0 + 2 + t/2]
                const float *yr = Yf + ((8 * (nb + q) + g) * yp + s0 + (t >> 1)) * 2 + (t & 1);
                const float b0 = (q == 0 || two) ? yr[0] : 0.f;
                const float b1 = (q == 0 || two) ? yr[4] : 0.f;
                split3(b0, bh0[q], bl0[q]);
                split3(b1, bh1[q], bl1[q]);
            }
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                float a[4];
                hh_frag_p(Hs, hp, s0, 8 * mt + g, t, a);
                uint32_t ah[4], al[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) split3(a[i], ah[i], al[i]);
                mma3(acc[mt][0], ah, al, bh0[0], bh1[0], bl0[0], bl1[0]);
                if (two) mma3(acc[mt][1], ah, al, bh0[1], bh1[1], bl0[1], bl1[1]);
            }
        }
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            const int uu = 8 * mt + g;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (q == 1 && !two) continue;
                const int n = 8 * (nb + q) + 2 * t;
                M[n * LD + uu] = make_float2(acc[mt][q][0], acc[mt][q][2]);
                M[(n + 1) * LD + uu] = make_float2(acc[mt][q][1], acc[mt][q][3]);
            }
        }
    }
}

// Gauss-Jordan inversion as in gj_invert with one uniform update for every
// lane.  The pivot lane does not normalise its row in the step: it keeps
// row k multiplied by its pivot p_k (only the pivot column is set, to p_k
// times the new entry 1/p_k, i.e. 1), which the later steps preserve since
// they update a row linearly; after the last step every lane divides its row
// by its own pivot.  Every lane's step is then R[j] -= f P[j] with f = 0 on
// the pivot lane, and nothing cancels (normalising in the step as
// R[j] - (1 - 1/p) P[j] loses log2(p) bits of the pivot row to the rounding
// of 1 - 1/p, all of them once p > 2^24).  FP32 reciprocal via rcp_approx.
// Returns the smallest pivot's real part (all pivots are real and positive
// for a Hermitian positive definite matrix).
//
// Every row is kept rotated so that step k's pivot column sits in R[0]: at
// the start of step k, R[j] holds column (k + j) mod UT.  The step writes the
// updated column k + j + 1 into R[j] and the new column k into R[UT - 1],
// which is the rotation for step k + 1; after UT steps the columns are back
// in order.  Every step is then the same code with fixed register indices,
// so the step loop stays rolled (a fully unrolled UT = 32 elimination is
// several thousand instructions and thrashes the instruction cache).
// Pivot-row load for the elimination: an ordered shared-memory load, so that
// the compiler does not hoist the whole row ahead of the multiply-adds (which
// would keep a second row in registers).
__device__ __forceinline__ void ld2_ordered(const float2 *p, float2 &a, float2 &b) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"((unsigned)__cvta_generic_to_shared(p)));
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
}

template <int UT>
__device__ __forceinline__ float gj_invert_f(float2 (&R)[UT], float2 *scratch, int u, int lane) {
    float min_piv = 3.0e38f;
    float2 my_inv = make_float2(1.f, 0.f);   // 1 / (this lane's pivot)
#pragma unroll 1
    for (int k = 0; k < UT; ++k) {
        if (lane == k) {
#pragma unroll
            for (int j = 0; j < UT; j += 2)
                *reinterpret_cast<float4 *>(&scratch[j]) = make_float4(R[j].x, R[j].y, R[j + 1].x, R[j + 1].y);
        }
        __syncwarp();
        const float2 pk = scratch[0];
        min_piv = fminf(min_piv, pk.x);
        const float d = rcp_approx(fmaf(pk.x, pk.x, pk.y * pk.y));
        const float2 inv = make_float2(pk.x * d, -pk.y * d);
        const bool me = (u == k);
        float2 f;
        if (me) {
            f = make_float2(0.f, 0.f);
            my_inv = inv;
        } else {
            f = make_float2(R[0].x * inv.x - R[0].y * inv.y, R[0].x * inv.y + R[0].y * inv.x);
        }
        const float2 nf = make_float2(-f.x, -f.y);
#pragma unroll
        for (int j = 0; j < UT; j += 2) {
            float2 a, b;
            ld2(&scratch[j], a, b);
            if (j > 0) {
                cmac(R[j], nf, a);
                R[j - 1] = R[j];
            }
            cmac(R[j + 1], nf, b);
            R[j] = R[j + 1];
        }
        R[UT - 1] = me ? make_float2(1.f, 0.f) : nf;
        __syncwarp();
    }
#pragma unroll
    for (int j = 0; j < UT; ++j)
        R[j] = make_float2(R[j].x * my_inv.x - R[j].y * my_inv.y, R[j].x * my_inv.y + R[j].y * my_inv.x);
    return min_piv;
}

// The per-cluster operator from the staged block H_c (row pitch hp, h_rows
// rows with zero padding past S), row u per lane (every lane group g holds a
// copy): B_c^{-1} for Alg. 1 (B_c = H_c^H H_c + delta I) and Alg. 3 (B_c =
// conj(H_c^H H_c) + delta I), G_c = H_c^H H_c for Alg. 2.  The Gram runs on
// the tensor cores for 16-bit inputs.  An FP32 pivot below 2^-12 of the
// largest diagonal entry recomputes this cluster's Gram and inverse in FP64
// (counted in *retries).  Shared by the fused kernel and the operator kernel
// (dbp_factor.cuh), so both give the same bits.
template <int UT, typename TIn, int ALG>
__device__ __forceinline__ void cluster_operator(const TIn *Hs, int hp, int h_rows, int S, float2 *Gm, float2 *Vb,
                                                 int lane, int u, int g, float f_delta, double delta, bool valid,
                                                 unsigned int *retries, float2 (&R)[UT]) {
    using C2 = float2;
    constexpr bool MMA = InTraits<TIn>::mma;
    constexpr bool MMA3 = FP32Mma<UT, TIn>::value;
    // ---- Gram (+ diagonal loading) ----
    if constexpr (MMA) {
        gram_mma<UT, TIn>(reinterpret_cast<const uint32_t *>(Hs), hp, h_rows, Gm, lane, u, R);
    } else if constexpr (MMA3) {
        gram_mma3<UT>(reinterpret_cast<const float2 *>(Hs), hp, h_rows, Gm, lane, u, R);
        if (ALG == ALG_ADMM_DL) {
#pragma unroll
            for (int v = 0; v < UT; ++v) R[v].y = -R[v].y;       // conj(H_c^H H_c)
        }
    } else {
#pragma unroll
        for (int v = 0; v < UT; ++v) R[v] = make_float2(0.f, 0.f);
        for (int r = g; r < S; r += Tile<UT>::G) {
            const C2 hu = to_f2(Hs[r * hp + u]);
#pragma unroll
            for (int v = 0; v < UT; v += 2) {
                C2 a, bb;
                ld2(reinterpret_cast<const C2 *>(&Hs[r * hp + v]), a, bb);
                if (ALG == ALG_ADMM_DL) {
                    cmacc(R[v], a, hu);
                    cmacc(R[v + 1], bb, hu);
                } else {
                    cmacc(R[v], hu, a);
                    cmacc(R[v + 1], hu, bb);
                }
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
    }
    float dmax = 0.f;
#pragma unroll
    for (int v = 0; v < UT; ++v)
        if (v == u) {
            R[v].x += f_delta;
            dmax = R[v].x;
        }
    if (ALG == ALG_ADMM_UL || ALG == ALG_ADMM_DL) {
        dmax = warp_redux_max(dmax);
        const float min_piv = gj_invert_f<UT>(R, Vb, u, lane);
        if (valid && !(min_piv >= 0x1p-12f * dmax)) {
            // FP64 retry: recompute this cluster's Gram and inverse in FP64.
            double2 D[UT];
#pragma unroll
            for (int v = 0; v < UT; ++v) D[v] = make_double2(0.0, 0.0);
            for (int r = 0; r < S; ++r) {
                const float2 hu = to_f2(Hs[r * hp + u]);
                const double2 hd = make_double2(hu.x, hu.y);
#pragma unroll
                for (int v = 0; v < UT; ++v) {
                    const float2 hv = to_f2(Hs[r * hp + v]);
                    const double2 vd = make_double2(hv.x, hv.y);
                    if (ALG == ALG_ADMM_DL) cmacc(D[v], vd, hd);
                    else cmacc(D[v], hd, vd);
                }
            }
#pragma unroll
            for (int v = 0; v < UT; ++v)
                if (v == u) D[v].x += delta;
            __syncwarp();
            gj_invert<UT>(D, reinterpret_cast<double2 *>(Vb), u, lane);
#pragma unroll
            for (int v = 0; v < UT; ++v) R[v] = make_float2((float)D[v].x, (float)D[v].y);
            if (lane == 0 && retries) atomicAdd(retries, 1u);
        }
    }
}

template <int UT> struct TmaCfg {
    using K = Tile<UT>;
    static constexpr int E = K::NCH * UT;   // consensus entries per subcarrier chunk
};

// Per-CTA shared memory after the warps' regions (host computes the same):
//   contrib[2][nwarps][E] | wsum[2][P][E]  (float2)  |  mbarriers[nwarps][2]
template <int UT> __host__ __device__ constexpr size_t tma_cta_bytes(int nwarps, int P) {
    return (2 * (size_t)nwarps * TmaCfg<UT>::E + 2 * (size_t)P * TmaCfg<UT>::E) * sizeof(float2) +
           (size_t)nwarps * 2 * sizeof(uint64_t);
}

template <int UT, int ALG, typename TIn>
__global__ void __launch_bounds__(Bounds<float, UT>::threads) dbp_tma_kernel(const FusedParams p) {
    using C2 = float2;
    using K = Tile<UT>;
    constexpr int E = TmaCfg<UT>::E;
    constexpr int EB = InTraits<TIn>::bytes;
    constexpr bool MMA = InTraits<TIn>::mma;
    constexpr bool MMA3 = FP32Mma<UT, TIn>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int C = p.C, P = p.P, S = p.S, N = p.N, B = p.B, W = p.W;
    const int pl = warp / C, c = warp - pl * C;
    const int u = lane % UT, g = lane / UT;
    const int hp = p.hp, yp = p.yp;

    unsigned char *wb = smem_raw + (size_t)warp * p.warp_bytes;
    C2 *Gm = reinterpret_cast<C2 *>(wb + p.off_g);            // Gram / matched-filter results
    C2 *Vb = reinterpret_cast<C2 *>(wb + p.off_v);
    C2 *contrib = reinterpret_cast<C2 *>(smem_raw + (size_t)nwarps * p.warp_bytes);   // [2][nwarps][E]
    C2 *wsum = contrib + 2 * (size_t)nwarps * E;                                        // [2][P][E]
    uint64_t *bars = reinterpret_cast<uint64_t *>(wsum + 2 * (size_t)P * E) + 2 * warp;

    // Zero this warp's region (rows and symbols that no copy fills stay
    // finite), then set up its two mbarriers.
    for (int i = lane * 16; i < p.warp_bytes; i += 32 * 16)
        *reinterpret_cast<float4 *>(wb + i) = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    fence_proxy_async();

    const TIn *Hg = reinterpret_cast<const TIn *>(p.H);
    const TIn *Vg = reinterpret_cast<const TIn *>(p.vin);

    // Copies of subcarrier w's cluster block (and receive rows) into buffer b.
    auto issue = [&](int w, int b) {
        const bool dense = (hp == UT);
        const uint32_t hbytes = (uint32_t)(S * UT * EB);
        const uint32_t ybytes = (uint32_t)(S * EB);
        const uint32_t total = hbytes + ((ALG == ALG_ADMM_DL) ? 0u : (uint32_t)N * ybytes);
        fence_proxy_async();
        if (lane == 0) mbar_arrive_expect_tx(&bars[b], total + p.starve_bytes);
        __syncwarp();
        const TIn *src = Hg + ((size_t)w * B + (size_t)c * S) * UT;
        unsigned char *hdst = wb + (b ? p.off_h1 : 0);
        if (dense) {
            if (lane == 0) bulk_g2s(hdst, src, hbytes, &bars[b]);
        } else {
            for (int s = lane; s < S; s += 32)
                bulk_g2s(hdst + (size_t)s * hp * EB, src + (size_t)s * UT, (uint32_t)(UT * EB), &bars[b]);
        }
        if (ALG != ALG_ADMM_DL) {
            unsigned char *ydst = wb + (b ? p.off_y1 : p.off_y0);
            for (int n = lane; n < N; n += 32)
                bulk_g2s(ydst + (size_t)n * yp * EB, Vg + ((size_t)w * N + n) * B + (size_t)c * S, ybytes, &bars[b]);
        }
    };

    grid_dependency_wait();
    grid_dependents_launch();
    uint32_t parity = 0u;   // bit b: phase parity of buffer b's mbarrier
    int tile = blockIdx.x;
    if (tile < p.tiles && tile * P + pl < W) issue(tile * P + pl, 0);

    int buf = 0;   // consensus double buffer
    const bool dbl = (p.single_buf == 0);
    for (int it = 0; tile < p.tiles; ++it, tile += gridDim.x) {
        const int b = dbl ? (it & 1) : 0;
        const int w = tile * P + pl;
        const bool valid = (w < W);
        const int ntile = tile + gridDim.x;
        const bool has_next = ntile < p.tiles && ntile * P + pl < W;
        if (dbl && has_next) issue(ntile * P + pl, b ^ 1);
        if (valid) {
            mbar_wait_bounded(&bars[b], (parity >> b) & 1u, p.status, p.wait_iters);
            parity ^= (1u << b);
        }
        const TIn *Hs = reinterpret_cast<const TIn *>(wb + (b ? p.off_h1 : 0));
        const TIn *Ys = reinterpret_cast<const TIn *>(wb + (b ? p.off_y1 : p.off_y0));

        // ---- Per-cluster operator: row u per lane ----
        C2 R[UT];
        C2 *frow = (p.factor != nullptr && valid)
                       ? p.factor + (((size_t)w * C + c) * UT + u) * UT : nullptr;
        if (p.factor_mode == 2) {
            // resident operator of this coherence block
            if (frow != nullptr) {
#pragma unroll
                for (int v = 0; v < UT; v += 2) {
                    const float4 q = *reinterpret_cast<const float4 *>(&frow[v]);
                    R[v] = make_float2(q.x, q.y);
                    R[v + 1] = make_float2(q.z, q.w);
                }
            } else {
#pragma unroll
                for (int v = 0; v < UT; ++v) R[v] = make_float2(0.f, 0.f);
            }
        } else {
        cluster_operator<UT, TIn, ALG>(Hs, hp, p.h_rows, S, Gm, Vb, lane, u, g, p.f_delta, p.delta, valid,
                                       p.retries, R);
        if (p.factor_mode == 1 && frow != nullptr && g == 0) {
#pragma unroll
            for (int v = 0; v < UT; v += 2)
                *reinterpret_cast<float4 *>(&frow[v]) = make_float4(R[v].x, R[v].y, R[v + 1].x, R[v + 1].y);
        }
        }   // operator computed

        if constexpr (MMA) {
            if (ALG != ALG_ADMM_DL) {
                mf_mma<UT, TIn>(reinterpret_cast<const uint32_t *>(Hs), hp, p.h_rows,
                                reinterpret_cast<const uint32_t *>(Ys), yp, (N + 7) / 8, Gm, lane);
                __syncwarp();
                // one staging buffer: H_c and y_c are no longer read
                if (!dbl && has_next) issue(ntile * P + pl, 0);
            }
        } else if constexpr (MMA3) {
            if (ALG != ALG_ADMM_DL) {
                mf_mma3<UT>(reinterpret_cast<const float2 *>(Hs), hp, p.h_rows, reinterpret_cast<const float2 *>(Ys),
                            yp, (N + 7) / 8, Gm, lane);
                __syncwarp();
                if (!dbl && has_next) issue(ntile * P + pl, 0);
            }
        }

        for (int n0 = 0; n0 < N; n0 += K::NCH) {
            C2 s_[K::NN];
            C2 acc[K::NN];

            // Two-phase consensus over the C clusters of this subcarrier.
            auto consensus = [&](const C2 (&val)[K::NN], C2 (&sum)[K::NN]) {
                C2 *mine = contrib + ((size_t)buf * nwarps + warp) * E;
#pragma unroll
                for (int j = 0; j < K::NN; ++j) mine[(g + K::G * j) * UT + u] = val[j];
                __syncthreads();
                const C2 *grp = contrib + ((size_t)buf * nwarps + pl * C) * E;
                C2 *ws = wsum + ((size_t)buf * P + pl) * E;
                const int per = (E + C - 1) / C;
                for (int e = c * per + lane; e < min(E, (c + 1) * per); e += 32) {
                    C2 a = make_float2(0.f, 0.f);
                    for (int cc = 0; cc < C; ++cc) {
                        const C2 tv = grp[(size_t)cc * E + e];
                        a.x += tv.x;
                        a.y += tv.y;
                    }
                    ws[e] = a;
                }
                __syncthreads();
#pragma unroll
                for (int j = 0; j < K::NN; ++j) sum[j] = ws[(g + K::G * j) * UT + u];
                buf ^= 1;
            };

            if (ALG == ALG_ADMM_UL || ALG == ALG_CG_UL) {
                // Matched filter m_c = H_c^H y_c.
                if constexpr (MMA || MMA3) {
#pragma unroll
                    for (int j = 0; j < K::NN; ++j) acc[j] = Gm[(n0 + g + K::G * j) * (UT + 2) + u];
                } else {
#pragma unroll
                    for (int j = 0; j < K::NN; ++j) acc[j] = make_float2(0.f, 0.f);
                    for (int r = 0; r < S; r += 2) {
                        const C2 h0 = to_f2(Hs[r * hp + u]);
                        const C2 h1 = to_f2(Hs[(r + 1) * hp + u]);
#pragma unroll
                        for (int j = 0; j < K::NN; ++j) {
                            C2 a, bb;
                            ld2(reinterpret_cast<const C2 *>(&Ys[(size_t)(n0 + g + K::G * j) * yp + r]), a, bb);
                            cmacc(acc[j], h0, a);
                            cmacc(acc[j], h1, bb);
                        }
                    }
                    // one staging buffer: the last chunk's matched filter was
                    // the last read of H_c and y_c
                    if (!dbl && n0 + K::NCH >= N) {
                        __syncwarp();
                        if (has_next) issue(ntile * P + pl, 0);
                    }
                }
            }

            if (ALG == ALG_ADMM_UL) {
                C2 yreg[K::NN], lam[K::NN], z[K::NN];
                put_vec<UT>(Vb, u, g, acc);
                __syncwarp();
                matvec<UT>(R, Vb, g, yreg);
                __syncwarp();
#pragma unroll
                for (int j = 0; j < K::NN; ++j) {
                    lam[j] = make_float2(0.f, 0.f);
                    z[j] = yreg[j];
                }
                auto prox = [&](C2 (&sum)[K::NN]) {
#pragma unroll
                    for (int j = 0; j < K::NN; ++j) {
                        if (p.reg >= 2) {   // (E2-BOX); BPSK: the real segment [-r, r]
                            const float r = p.f_box_r, ic = p.f_invC;
                            s_[j].x = clip_r(sum[j].x * ic, r);
                            s_[j].y = (p.reg == 2) ? clip_r(sum[j].y * ic, r) : 0.f;
                        } else {
                            s_[j] = cscale(sum[j], p.f_e2_scale);
                        }
                    }
                };
                consensus(z, acc);
                prox(acc);
                const float gam = p.f_gamma, rho = p.f_rho;
                for (int t = 2; t <= p.T; ++t) {
                    C2 d[K::NN];
#pragma unroll
                    for (int j = 0; j < K::NN; ++j) {
                        lam[j].x = fmaf(gam, z[j].x - s_[j].x, lam[j].x);
                        lam[j].y = fmaf(gam, z[j].y - s_[j].y, lam[j].y);
                        d[j] = cscale(csub(s_[j], lam[j]), rho);
                    }
                    put_vec<UT>(Vb, u, g, d);
                    __syncwarp();
                    matvec<UT>(R, Vb, g, z);
                    __syncwarp();
                    C2 wv[K::NN];
#pragma unroll
                    for (int j = 0; j < K::NN; ++j) {
                        z[j] = cadd(z[j], yreg[j]);
                        wv[j] = cadd(z[j], lam[j]);
                    }
                    consensus(wv, acc);
                    prox(acc);
                }
            } else if (ALG == ALG_CG_UL) {
                C2 r[K::NN], pv[K::NN], x[K::NN];
                float rr[K::NN];
                bool live[K::NN];
                consensus(acc, r);
#pragma unroll
                for (int j = 0; j < K::NN; ++j) {
                    pv[j] = r[j];
                    x[j] = make_float2(0.f, 0.f);
                    rr[j] = group_sum<UT>(r[j].x * r[j].x + r[j].y * r[j].y);
                    live[j] = true;
                }
                const float rcg = p.f_rho_cg;
                for (int t = 1; t <= p.T; ++t) {
                    C2 wc[K::NN], e[K::NN];
                    put_vec<UT>(Vb, u, g, pv);
                    __syncwarp();
                    matvec<UT>(R, Vb, g, wc);
                    __syncwarp();
                    consensus(wc, e);
#pragma unroll
                    for (int j = 0; j < K::NN; ++j) {
                        e[j].x = fmaf(rcg, pv[j].x, e[j].x);
                        e[j].y = fmaf(rcg, pv[j].y, e[j].y);
                        const float pe = group_sum<UT>(pv[j].x * e[j].x + pv[j].y * e[j].y);
                        const bool go = live[j] && rr[j] != 0.f && pe != 0.f;
                        const float alpha = go ? __fdiv_rn(rr[j], pe) : 0.f;
                        x[j].x = fmaf(alpha, pv[j].x, x[j].x);
                        x[j].y = fmaf(alpha, pv[j].y, x[j].y);
                        r[j].x = fmaf(-alpha, e[j].x, r[j].x);
                        r[j].y = fmaf(-alpha, e[j].y, r[j].y);
                        const float rn = group_sum<UT>(r[j].x * r[j].x + r[j].y * r[j].y);
                        const float beta = go ? __fdiv_rn(rn, rr[j]) : 0.f;
                        if (go) {
                            pv[j].x = fmaf(beta, pv[j].x, r[j].x);
                            pv[j].y = fmaf(beta, pv[j].y, r[j].y);
                            rr[j] = rn;
                        }
                        live[j] = go;
                    }
                }
#pragma unroll
                for (int j = 0; j < K::NN; ++j) s_[j] = x[j];
            } else {  // ALG_ADMM_DL (FP32 inputs only)
                C2 sv[K::NN], z[K::NN], lam[K::NN], v[K::NN], m[K::NN];
                const float kap = p.f_kappa, gam = p.f_gamma, ic = p.f_invC;
                const C2 *Sg = reinterpret_cast<const C2 *>(p.vin);
#pragma unroll
                for (int j = 0; j < K::NN; ++j) {
                    const int n = n0 + g + K::G * j;
                    sv[j] = (valid && n < N) ? Sg[((size_t)w * N + n) * UT + u] : make_float2(0.f, 0.f);
                    z[j] = cscale(sv[j], kap);
                    lam[j] = make_float2(0.f, 0.f);
                    v[j] = z[j];
                }
                const float ir = p.f_inv_rho;
                for (int t = 2; t <= p.T; ++t) {
                    put_vec<UT>(Vb, u, g, v);
                    __syncwarp();
                    matvec<UT>(R, Vb, g, m);
                    __syncwarp();
                    // m_c = H_c x_c = v_c - rho^{-1} B_c^{-1} v_c
#pragma unroll
                    for (int j = 0; j < K::NN; ++j) {
                        m[j].x = fmaf(-ir, m[j].x, v[j].x);
                        m[j].y = fmaf(-ir, m[j].y, v[j].y);
                    }
                    C2 wc[K::NN], ws[K::NN];
#pragma unroll
                    for (int j = 0; j < K::NN; ++j) wc[j] = csub(m[j], lam[j]);
                    consensus(wc, ws);
                    if (p.f_eps > 0.f) {
                        // Lemma 2: s - w scaled by max{0, 1 - eps / ||s - w||}
#pragma unroll
                        for (int j = 0; j < K::NN; ++j) {
                            const C2 dl = csub(sv[j], ws[j]);
                            const float nrm = sqrtf(group_sum<UT>(dl.x * dl.x + dl.y * dl.y));
                            const float k = (nrm > 0.f) ? fmaxf(0.f, 1.f - p.f_eps / nrm) : 0.f;
                            ws[j] = csub(sv[j], cscale(dl, k));
                        }
                    }
#pragma unroll
                    for (int j = 0; j < K::NN; ++j) {
                        z[j].x = fmaf(sv[j].x - ws[j].x, ic, wc[j].x);
                        z[j].y = fmaf(sv[j].y - ws[j].y, ic, wc[j].y);
                        lam[j].x = fmaf(-gam, m[j].x - z[j].x, lam[j].x);
                        lam[j].y = fmaf(-gam, m[j].y - z[j].y, lam[j].y);
                        v[j] = cadd(z[j], lam[j]);
                    }
                }
                put_vec<UT>(Vb, u, g, v);
                __syncwarp();
                matvec<UT>(R, Vb, g, m);          // B_c^{-1} v_c
                __syncwarp();
                put_vec<UT>(Vb, u, g, m);
                __syncwarp();
                C2 *xo = reinterpret_cast<C2 *>(p.out);
                const C2 *Hc = reinterpret_cast<const C2 *>(p.H) + ((size_t)(valid ? w : 0) * B + (size_t)c * S) * UT;
                float energy = 0.f;
                for (int r0 = 0; r0 < S; r0 += 32) {
                    const int sr = r0 + lane;
                    C2 h[UT];
                    if (valid && sr < S) {
#pragma unroll
                        for (int k = 0; k < UT; k += 2) {
                            const float4 q = *reinterpret_cast<const float4 *>(&Hc[(size_t)sr * UT + k]);
                            h[k] = make_float2(q.x, q.y);
                            h[k + 1] = make_float2(q.z, q.w);
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < UT; ++k) h[k] = make_float2(0.f, 0.f);
                    }
                    for (int nl = 0; nl < K::NCH; ++nl) {
                        const int n = n0 + nl;
                        if (n >= N) break;
                        C2 a = make_float2(0.f, 0.f);
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

            // Uplink outputs: warp c writes the symbol slots j with j % C == c.
            if (ALG != ALG_ADMM_DL && valid) {
                C2 *xo = reinterpret_cast<C2 *>(p.out);
#pragma unroll
                for (int j = 0; j < K::NN; ++j) {
                    const int n = n0 + g + K::G * j;
                    if ((j % C) == c && n < N) {
                        const size_t o = ((size_t)w * N + n) * UT + u;
                        xo[o] = s_[j];
                        if (p.labels != nullptr)
                            p.labels[o] = qam_label<float>(s_[j].x, s_[j].y, p.f_qam_inv_a, p.qam_L, p.qam_half);
                    }
                }
            }
        }
    }
}

}  // namespace dbp
