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
// One warp per subcarrier: lane (u, g) accumulates row u of G over the rows
// s = g, g + G, ... of H, the groups are summed by shuffles, the Gram is
// inverted in registers (Gauss-Jordan, HPD, no pivoting) for A_uu, and the
// lanes then run over the (symbol, user) entries of the subcarrier.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "dbp.h"
#include "dbp_fused.cuh"
#include "dbp_internal.h"

namespace dbp {

struct LlrParams {
    const float2 *H;     // [W][B][U]
    const float2 *x;     // [W][N][U]
    float *llr;          // [W][N][U][m]
    int W, N, B, U;
    int L, m, half;      // PAM levels per axis, bits per symbol, bits per axis
    int zf;              // 1: ZF statistics, 0: MMSE
    float delta, N0, Es;
    float a;             // PAM half-spacing: levels (2k - L + 1) a
};

constexpr int kLlrWarps = 8;

template <int UT>
__global__ void __launch_bounds__(32 * kLlrWarps) dbp_llr_kernel(const LlrParams p) {
    constexpr int G = 32 / UT;
    __shared__ __align__(16) float2 scratch[kLlrWarps][UT];
    __shared__ float mus[kLlrWarps][UT], nus[kLlrWarps][UT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u = lane % UT, g = lane / UT;
    const int w = blockIdx.x * kLlrWarps + warp;
    if (w >= p.W) return;                       // whole warp: no block-level sync below
    const int U = p.U, B = p.B;

    // Row u of G = H^H H (zero for padded users)
    float2 R[UT];
#pragma unroll
    for (int v = 0; v < UT; ++v) R[v] = make_float2(0.f, 0.f);
    if (u < U) {
        const float2 *Hw = p.H + (size_t)w * B * U;
        for (int s = g; s < B; s += G) {
            const float2 hu = __ldg(&Hw[(size_t)s * U + u]);
#pragma unroll
            for (int v = 0; v < UT; ++v)
                if (v < U) cmacc(R[v], hu, __ldg(&Hw[(size_t)s * U + v]));
        }
    }
#pragma unroll
    for (int msk = UT; msk < 32; msk <<= 1) {
#pragma unroll
        for (int v = 0; v < UT; ++v) {
            R[v].x += shfl_x(R[v].x, msk);
            R[v].y += shfl_x(R[v].y, msk);
        }
    }
#pragma unroll
    for (int v = 0; v < UT; ++v)
        if (v == u) R[v].x += (u < U) ? p.delta : 1.f;   // padded users: identity rows
    gj_invert<UT>(R, &scratch[warp][0], u, lane);
    float Auu = 0.f;
#pragma unroll
    for (int v = 0; v < UT; ++v)
        if (v == u) Auu = R[v].x;
    if (g == 0) {
        float mu, nu2;
        if (p.zf) {
            mu = 1.f;
            nu2 = p.N0 * Auu;
        } else {
            mu = 1.f - p.delta * Auu;
            nu2 = p.Es * mu * (1.f - mu);
        }
        mus[warp][u] = mu;
        nus[warp][u] = nu2;
    }
    __syncwarp();

    // LLRs of the (symbol, user) entries of this subcarrier
    for (int e = lane; e < p.N * U; e += 32) {
        const int n = e / U, uu = e - n * U;
        const float2 xv = p.x[((size_t)w * p.N + n) * U + uu];
        const float mu = mus[warp][uu];
        const float inv_nu2 = 1.f / nus[warp][uu];
        float *out = p.llr + (((size_t)w * p.N + n) * U + uu) * p.m;
#pragma unroll
        for (int axis = 0; axis < 2; ++axis) {
            const float v = axis ? xv.y : xv.x;
            float mn0[4], mn1[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) mn0[j] = mn1[j] = INFINITY;
            for (int k = 0; k < p.L; ++k) {
                const float d = v - mu * (float)(2 * k - p.L + 1) * p.a;
                const float d2 = d * d;
                const int gray = k ^ (k >> 1);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (j < p.half) {
                        if ((gray >> (p.half - 1 - j)) & 1) mn1[j] = fminf(mn1[j], d2);
                        else mn0[j] = fminf(mn0[j], d2);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (j < p.half) out[axis * p.half + j] = (mn1[j] - mn0[j]) * inv_nu2;
        }
    }
}

template <int UT>
cudaError_t launch_llr(const LlrParams &p, cudaStream_t st) {
    const int blocks = (p.W + kLlrWarps - 1) / kLlrWarps;
    dbp_llr_kernel<UT><<<blocks, 32 * kLlrWarps, 0, st>>>(p);
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
    p.W = d->W;
    p.N = d->N;
    p.B = d->B;
    p.U = d->U;
    int L = 1;
    while (L * L < d->qam_order) ++L;
    int m = 0;
    while ((1 << m) < d->qam_order) ++m;
    p.L = L;
    p.m = m;
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
