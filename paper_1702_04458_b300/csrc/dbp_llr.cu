// dbp_llr.cu -- soft outputs of the uplink detectors: max-log LLRs of every
// label bit from the detector's estimate x_hat and the bias / noise
// statistics of the linear (MMSE or ZF) estimate.
//
// For A = (G + delta I)^{-1} with the subcarrier's Gram G = H^H H (the sum of
// the cluster Grams, Sec. III-C), the estimate behaves as
// x_u = mu_u s_u + e_u with
//   MMSE (delta = N0/Es): mu_u = 1 - delta A_uu, E|e_u|^2 = Es mu_u (1 - mu_u)
//   ZF   (delta = 0):     mu_u = 1,              E|e_u|^2 = N0 A_uu,
// and the max-log LLR of label bit j is
//   L_j = (min_{s: bit_j = 1} |x - mu s|^2 - min_{s: bit_j = 0} |x - mu s|^2) / E|e|^2,
// positive when the bit is more likely 0.  For a square Gray QAM alphabet
// |x - mu s|^2 separates into the two axes, and each axis's bits depend on
// its PAM level only, so every bit takes a minimum over L = sqrt(M) levels.
//
// One CTA of four warps per subcarrier.  The CTA stages the B rows of H_w
// into shared memory with asynchronous copies (every load of a chunk issued
// before the first wait, so a subcarrier costs one memory round trip per
// chunk, not one per row) and splits the Gram's rows over its warps (on the
// tensor cores at 8 and 32 users, on the CUDA cores otherwise); the warps'
// partial Grams are summed through shared memory, one warp inverts the Gram
// in registers (Gauss-Jordan, HPD, no pivoting) for A_uu, and the CTA's
// threads then run over the (symbol, user) entries of the subcarrier.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "dbp.h"
#include "dbp_fused.cuh"
#include "dbp_mma8.cuh"
#include "dbp_internal.h"

namespace dbp {

struct LlrParams {
    const float2 *H;     // [W][B][U]
    const float2 *x;     // [W][N][U]
    float *llr;          // [W][N][U][m]
    int W, N, B, U;
    int half;            // bits per axis (selects the kernel's template argument)
    int llr_align;       // largest power of two (up to 16) dividing the llr address
    int zf;              // 1: ZF statistics, 0: MMSE
    float delta, N0, Es;
    float a;             // PAM half-spacing: levels (2k - L + 1) a
};

constexpr int kLlrThreads = 128;

// Rows of H_w staged per chunk (pitch UT, padded columns zero).  The buffer
// also holds the three other warps' partial Grams after the last chunk.
template <int UT> struct LlrCfg {
    static constexpr int kChunkBytes = UT == 32 ? 24576 : 8192;
    static constexpr int kRows = kChunkBytes / (UT * 8);
    static_assert((kLlrThreads / 32 - 1) * UT * UT * 8 <= kChunkBytes, "partial Grams fit the staging buffer");
};

__device__ __forceinline__ void llr_cp16(void *dst, const void *src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void llr_cp8(void *dst, const void *src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void llr_cp_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Bias and inverse noise variance of user u from A_uu = ((G + delta I)^{-1})_uu.
__device__ __forceinline__ void llr_stats_store(const LlrParams &p, float Auu, int u, float *mus, float *inv_nus) {
    float mu, nu2;
    if (p.zf) {
        mu = 1.f;
        nu2 = p.N0 * Auu;
    } else {
        mu = 1.f - p.delta * Auu;
        nu2 = p.Es * mu * (1.f - mu);
    }
    mus[u] = mu;
    inv_nus[u] = 1.f / nu2;
}

// Gauss-Jordan inversion of a 32 x 32 HPD matrix shared by the CTA's four
// warps by columns: warp w, lane u holds entries (u, 8 w .. 8 w + 7) in A.
// Step k publishes row k (lane k of every warp, its 8 entries) and column k
// (warp k / 8) in one of two buffers of buf (2 x 64 complex, 16-byte
// aligned) and every thread updates its 8 entries; one CTA barrier per step.
// No pivoting (every pivot is a Schur complement of an HPD matrix).  The
// pivot row of a step is left as it is (its column-k entry set to 1) and
// divided by its pivot after the last step, as in gj_split.
__device__ __forceinline__ void gj_cols32(float2 (&A)[8], int u, int w, float2 *buf) {
    float2 myinv = make_float2(1.f, 0.f);     // 1 / the pivot of row u's own step
#pragma unroll 1
    for (int wk = 0; wk < 4; ++wk) {
#pragma unroll
        for (int ik = 0; ik < 8; ++ik) {
            const int k = 8 * wk + ik;
            float2 *b = buf + (ik & 1) * 64;   // [0, 32): row k; [32, 64): column k
            if (u == k) {
#pragma unroll
                for (int i = 0; i < 8; i += 2)
                    *reinterpret_cast<float4 *>(&b[8 * w + i]) = make_float4(A[i].x, A[i].y, A[i + 1].x, A[i + 1].y);
            }
            if (w == wk) b[32 + u] = A[ik];
            __syncthreads();
            const float2 piv = b[32 + k];
            const float2 f = b[32 + u];
            float2 rk[8];
#pragma unroll
            for (int i = 0; i < 8; i += 2) ld2(&b[8 * w + i], rk[i], rk[i + 1]);
            const float dd = rcp_approx(fmaf(piv.x, piv.x, piv.y * piv.y));
            const float2 inv = make_float2(piv.x * dd, -piv.y * dd);
            const bool me = (u == k);
            const float2 fi = cmul(f, inv);                  // f_u / p
            const float2 nm = me ? make_float2(0.f, 0.f) : make_float2(-fi.x, -fi.y);
            if (me) myinv = inv;
#pragma unroll
            for (int i = 0; i < 8; ++i) cmac(A[i], nm, rk[i]);
            if (w == wk) A[ik] = me ? make_float2(1.f, 0.f) : make_float2(-fi.x, -fi.y);
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) A[i] = cmul(A[i], myinv);
}

template <int UT, int HALF>
__global__ void __launch_bounds__(kLlrThreads, UT == 32 ? 5 : 1) dbp_llr_kernel(const LlrParams p) {
    using Cfg = LlrCfg<UT>;
    constexpr int NW = kLlrThreads / 32;   // warps per CTA
    constexpr int G = kLlrThreads / UT;    // row groups per CTA
    __shared__ __align__(16) float2 Hs[Cfg::kRows * UT];
    __shared__ __align__(16) float2 scratch[UT];
    __shared__ float mus[UT], inv_nus[UT];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int u = tid % UT, g = tid / UT;
    const int w = blockIdx.x;
    const int U = p.U, B = p.B, NU = p.N * U;
    const float2 *xw = p.x + (size_t)w * NU;

    // this thread's first estimate entry, in flight while the Gram is formed
    float2 x0 = make_float2(0.f, 0.f);
    if (tid < NU) x0 = __ldg(&xw[tid]);
    if (U != UT) {   // padded columns stay zero through every chunk
        for (int i = tid; i < Cfg::kRows * UT; i += kLlrThreads) Hs[i] = make_float2(0.f, 0.f);
        __syncthreads();
    }

    // G = H^H H.  UT = 8: 3xTF32 m16n8k8 products (FP32 accuracy) over
    // k-steps of 4 rows, lane (gq, t) of each warp accumulating entries
    // (gq, 2t), (gq, 2t + 1) of its k-steps.  UT = 32: the same products for
    // the blocks on and above the diagonal, each warp summing a quarter of
    // every staged chunk (gram_mma3_acc), then row u per lane.  Otherwise
    // thread (u, g) sums row u over its rows on the CUDA cores.  Padded users
    // give zero rows.
    constexpr bool kTc = (UT == 8);
    constexpr bool kTc32 = (UT == 32);
    constexpr int kGbuf = kTc32 ? NW * 16 * (UT + 2) : 2;   // gram_mma3_rows' row buffers
    __shared__ __align__(16) float2 gbuf[kGbuf];
    __shared__ __align__(16) float2 gjbuf[kTc32 ? 128 : 2];   // gj_cols32's two buffers
    const int gq = lane >> 2, t = lane & 3;
    float gacc[4] = {0.f, 0.f, 0.f, 0.f};
    constexpr int kMT = kTc32 ? UT / 8 : 1;
    float acc32[kMT][kMT][4];
#pragma unroll
    for (int i = 0; i < kMT; ++i)
#pragma unroll
        for (int j = 0; j < kMT; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc32[i][j][e] = 0.f;
    float2 R[UT];
#pragma unroll
    for (int v = 0; v < UT; ++v) R[v] = make_float2(0.f, 0.f);
    const float2 *Hw = p.H + (size_t)w * B * U;
    const bool vec = (U == UT) && ((reinterpret_cast<uintptr_t>(Hw) & 15) == 0);
    for (int s0 = 0; s0 < B; s0 += Cfg::kRows) {
        const int rows = min(Cfg::kRows, B - s0);
        if (s0 > 0) __syncthreads();   // the previous chunk's reads are done
        const float2 *src = Hw + (size_t)s0 * U;
        if (vec) {                      // contiguous rows, U even: 16-byte pieces
            for (int i = tid; i < rows * UT / 2; i += kLlrThreads) llr_cp16(&Hs[2 * i], src + 2 * i);
        } else {
            for (int i = tid; i < rows * U; i += kLlrThreads) {
                const int r = i / U;
                llr_cp8(&Hs[r * UT + (i - r * U)], src + i);
            }
        }
        const int rows4 = (rows + 3) & ~3;
        if (kTc || kTc32) {   // a k-step reads four rows: the ones past B are zero
            for (int i = rows * UT + tid; i < rows4 * UT; i += kLlrThreads) Hs[i] = make_float2(0.f, 0.f);
        }
        llr_cp_wait();
        __syncthreads();
        if constexpr (kTc32) {
            constexpr int kWarpRows = Cfg::kRows / NW;   // a multiple of 4
            const int r0 = warp * kWarpRows, r1 = min(r0 + kWarpRows, rows4);
            if (r1 > r0) gram_mma3_acc<UT>(Hs + r0 * UT, UT, r1 - r0, lane, acc32);
        } else if constexpr (kTc) {
            for (int ks = warp; 4 * ks < rows4; ks += NW) {
                float a[4];
                hh_frag(Hs, 4 * ks, gq, t, a);
                uint32_t ah[4], al[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) split3(a[i], ah[i], al[i]);
                mma3(gacc, ah, al, ah[0], ah[2], al[0], al[2]);   // B operand = H: the same values
            }
        } else {
            for (int s = g; s < rows; s += G) {
                const float2 hu = Hs[s * UT + u];
#pragma unroll
                for (int v = 0; v < UT; v += 2) {
                    const float4 q = *reinterpret_cast<const float4 *>(&Hs[s * UT + v]);
                    cmacc(R[v], hu, make_float2(q.x, q.y));
                    cmacc(R[v + 1], hu, make_float2(q.z, q.w));
                }
            }
        }
    }
    if constexpr (kTc32) gram_mma3_rows<UT>(acc32, &gbuf[warp * 16 * (UT + 2)], lane, u, R);
    if constexpr (!kTc) {
#pragma unroll
        for (int msk = UT; msk < 32; msk <<= 1) {   // the warp's row groups
#pragma unroll
            for (int v = 0; v < UT; ++v) {
                R[v].x += shfl_x(R[v].x, msk);
                R[v].y += shfl_x(R[v].y, msk);
            }
        }
    }
    __syncthreads();   // every read of the staged rows is done: the buffer takes the partial Grams
    if constexpr (kTc) {
        float *part = reinterpret_cast<float *>(Hs);   // part[((k 4) + i) 32 + lane]: warp k + 1's gacc[i]
        if (warp > 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) part[((warp - 1) * 4 + i) * 32 + lane] = gacc[i];
        }
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int k = 0; k < NW - 1; ++k) {
#pragma unroll
                for (int i = 0; i < 4; ++i) gacc[i] += part[(k * 4 + i) * 32 + lane];
            }
            float2 e0 = make_float2(gacc[0], gacc[2]), e1 = make_float2(gacc[1], gacc[3]);
            const float dl = (gq < U) ? p.delta : 1.f;   // padded users: identity rows
            if (2 * t == gq) e0.x += dl;
            if (2 * t + 1 == gq) e1.x += dl;
            gj8<float2, float>(e0, e1, gq, t);
            if (gq < U && (gq >> 1) == t) llr_stats_store(p, (gq & 1) ? e1.x : e0.x, gq, mus, inv_nus);
        }
    } else if constexpr (kTc32) {
        // part[(k UT + v) UT + u]: warp k + 1's entry (u, v) in the staging
        // buffer; warp 0's in the Gram row buffers, free after the epilogue
        float2 *part = Hs;
        if (warp > 0) {
#pragma unroll
            for (int v = 0; v < UT; ++v) part[((warp - 1) * UT + v) * UT + u] = R[v];
        } else {
#pragma unroll
            for (int v = 0; v < UT; ++v) gbuf[v * UT + u] = R[v];
        }
        __syncthreads();
        float2 A[8];   // entries (u, 8 warp + i) of G + delta I
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int v = 8 * warp + i;
            float2 a = gbuf[v * UT + u];
#pragma unroll
            for (int k = 0; k < NW - 1; ++k) {
                const float2 q = part[(k * UT + v) * UT + u];
                a.x += q.x;
                a.y += q.y;
            }
            if (v == u) a.x += (u < U) ? p.delta : 1.f;   // padded users: identity rows
            A[i] = a;
        }
        gj_cols32(A, u, warp, gjbuf);
        // A_uu sits in warp u / 8 at index u % 8 (fixed register indices)
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (8 * warp + i == u && u < U) llr_stats_store(p, A[i].x, u, mus, inv_nus);
    } else {
        float2 *part = Hs;  // part[(k UT + v) UT + u]: warp k + 1's entry (u, v)
        if (warp > 0 && lane < UT) {
#pragma unroll
            for (int v = 0; v < UT; ++v) part[((warp - 1) * UT + v) * UT + u] = R[v];
        }
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int k = 0; k < NW - 1; ++k) {
#pragma unroll
                for (int v = 0; v < UT; ++v) {
                    const float2 q = part[(k * UT + v) * UT + u];
                    R[v].x += q.x;
                    R[v].y += q.y;
                }
            }
#pragma unroll
            for (int v = 0; v < UT; ++v)
                if (v == u) R[v].x += (u < U) ? p.delta : 1.f;   // padded users: identity rows
            gj_invert<UT>(R, scratch, u, lane);
            float Auu = 0.f;
#pragma unroll
            for (int v = 0; v < UT; ++v)
                if (v == u) Auu = R[v].x;
            if (lane < UT) llr_stats_store(p, Auu, u, mus, inv_nus);
        }
    }
    __syncthreads();

    // LLRs of the (symbol, user) entries of this subcarrier: per axis the
    // minima of |v - mu l a|^2 over the PAM levels l = 2k - L + 1 whose Gray
    // label has bit j = 0 / 1.
    constexpr int L = 1 << HALF;
    for (int e = tid; e < NU; e += kLlrThreads) {
        const float2 xv = (e == tid) ? x0 : __ldg(&xw[e]);
        const int uu = e % U;
        const float mua = mus[uu] * p.a;
        const float inv_nu2 = inv_nus[uu];
        float out[2 * HALF];
#pragma unroll
        for (int axis = 0; axis < 2; ++axis) {
            const float v = axis ? xv.y : xv.x;
            float mn0[HALF], mn1[HALF];
#pragma unroll
            for (int j = 0; j < HALF; ++j) mn0[j] = mn1[j] = INFINITY;
#pragma unroll
            for (int k = 0; k < L; ++k) {
                const float d = v - (float)(2 * k - L + 1) * mua;
                const float d2 = d * d;
                const int gray = k ^ (k >> 1);
#pragma unroll
                for (int j = 0; j < HALF; ++j) {
                    if ((gray >> (HALF - 1 - j)) & 1) mn1[j] = fminf(mn1[j], d2);
                    else mn0[j] = fminf(mn0[j], d2);
                }
            }
#pragma unroll
            for (int j = 0; j < HALF; ++j) out[axis * HALF + j] = (mn1[j] - mn0[j]) * inv_nu2;
        }
        float *dst = p.llr + ((size_t)w * NU + e) * (2 * HALF);
        if (p.llr_align >= 16 && (HALF % 2) == 0) {
#pragma unroll
            for (int j = 0; j < 2 * HALF; j += 4)
                *reinterpret_cast<float4 *>(dst + j) = make_float4(out[j], out[j + 1], out[j + 2], out[j + 3]);
        } else if (p.llr_align >= 8) {
#pragma unroll
            for (int j = 0; j < 2 * HALF; j += 2) *reinterpret_cast<float2 *>(dst + j) = make_float2(out[j], out[j + 1]);
        } else {
#pragma unroll
            for (int j = 0; j < 2 * HALF; ++j) dst[j] = out[j];
        }
    }
}

template <int UT>
cudaError_t launch_llr(const LlrParams &p, cudaStream_t st) {
    switch (p.half) {
    case 1: dbp_llr_kernel<UT, 1><<<p.W, kLlrThreads, 0, st>>>(p); break;
    case 2: dbp_llr_kernel<UT, 2><<<p.W, kLlrThreads, 0, st>>>(p); break;
    case 3: dbp_llr_kernel<UT, 3><<<p.W, kLlrThreads, 0, st>>>(p); break;
    default: dbp_llr_kernel<UT, 4><<<p.W, kLlrThreads, 0, st>>>(p); break;
    }
    return cudaGetLastError();
}

}  // namespace dbp
extern "C" {

dbp_status dbp_uplink_llr(dbp_handle_t h, const dbp_frame_desc *d, const void *H, const void *x_hat, float *llr,
                          void *stream) {
    if (!h) return DBP_ERR_INVALID_ARG;
    std::string err;
    dbp_status v = dbp_validate_internal(h, d, DBP_KIND_UPLINK_ADMM, &err);
    if (v != DBP_OK) {
        h->err = err;
        return v;
    }
    if (d->qam_order == 0) {
        h->err = "dbp_uplink_llr needs the QAM order (qam_order > 0)";
        return DBP_ERR_INVALID_ARG;
    }
    if (d->regularizer != DBP_REG_MMSE && d->regularizer != DBP_REG_ZF) {
        h->err = "soft outputs are defined for the MMSE and ZF estimates";
        return DBP_ERR_INVALID_ARG;
    }
    if (d->precision != DBP_FP32) {
        h->err = "dbp_uplink_llr takes FP32 (complex64) H and x_hat";
        return DBP_ERR_UNSUPPORTED;
    }
    if (!(d->N0 > 0.0) || !(d->Es > 0.0)) {
        h->err = "soft outputs need N0 > 0 and Es > 0";
        return DBP_ERR_INVALID_ARG;
    }
    if (d->regularizer == DBP_REG_ZF && d->U > d->B) {
        h->err = "ZF statistics need U <= B";
        return DBP_ERR_INVALID_ARG;
    }
    if ((long long)d->W * d->N == 0) return DBP_OK;
    if (!H || !x_hat || !llr) {
        h->err = "NULL data pointer";
        return DBP_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) {
        h->err = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
        return DBP_ERR_CUDA;
    }
    dbp::LlrParams p{};
    p.H = static_cast<const float2 *>(H);
    p.x = static_cast<const float2 *>(x_hat);
    p.llr = llr;
    p.llr_align = 4;
    while (p.llr_align < 16 && (reinterpret_cast<uintptr_t>(llr) % (2 * p.llr_align)) == 0) p.llr_align *= 2;
    p.W = d->W;
    p.N = d->N;
    p.B = d->B;
    p.U = d->U;
    int m = 0;
    while ((1 << m) < d->qam_order) ++m;
    p.half = m / 2;
    p.zf = (d->regularizer == DBP_REG_ZF);
    p.delta = p.zf ? 0.f : (float)(d->N0 / d->Es);
    p.N0 = (float)d->N0;
    p.Es = (float)d->Es;
    p.a = (float)(std::sqrt(3.0 / (2.0 * (d->qam_order - 1))) * std::sqrt(d->Es));
    const int UT = dbp_padded_users(d->U);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (UT) {
    case 4: e = dbp::launch_llr<4>(p, st); break;
    case 8: e = dbp::launch_llr<8>(p, st); break;
    case 16: e = dbp::launch_llr<16>(p, st); break;
    default: e = dbp::launch_llr<32>(p, st); break;
    }
    if (e != cudaSuccess) {
        h->err = std::string("soft-output launch: ") + cudaGetErrorString(e);
        return DBP_ERR_CUDA;
    }
    return DBP_OK;
}

}  // extern "C"
