// dbp_factor.cuh -- the per-cluster operator B_c^{-1} of Alg. 1 (uplink
// ADMM) and Alg. 3 (downlink ADMM) as a kernel of its own.
//
// B_c depends on H_c only (Sec. III-B, IV-B: the preprocessing of each
// cluster), so it can be formed before the iterations run.  This kernel does
// exactly that for every (subcarrier, cluster) and stores row u of B_c^{-1}
// at factor[((w C + c) U + u) U + v], the layout the fused kernels load with
// factor_mode 2 (the resident operator of a coherence block).  It has no
// consensus and no CTA barrier, so its warps are independent: small CTAs,
// many warps per SM, the Gauss-Jordan latency hidden by the other warps.
// The fused kernels at U = 32 (bulk-copy kernel) and U = 16 downlink
// (tensor-core kernel) hold one CTA per SM; there the inverse, a long chain
// of dependent steps, is what the SM waits on.
//
// Same arithmetic as the fused kernels: the operator is computed by the same
// device functions (cluster_operator, tcdl_operator) on the same staged
// layout, so the results are bit-identical with and without this kernel.
#pragma once

#include "dbp_tcdl.cuh"
#include "dbp_tma.cuh"

namespace dbp {

struct FactorParams {
    const void *H;            // [W][B][U] complex (16-bit inputs: (re, im) pairs)
    float2 *factor;           // [W][C][UT][UT]
    int W, B, C, S;
    int hp, h_rows;           // staged row pitch (elements) and rows (zero past S)
    int warp_bytes;           // shared memory per warp
    int off_g, off_v;         // Gram row buffer and scratch, byte offsets in the warp's region
    float f_delta;            // diagonal loading in FP32 (rho for Alg. 1, 1/rho for Alg. 3)
    double delta;             // the same in FP64 (the FP64 retry)
    unsigned int *retries;    // FP64 retries (device counter) or null
};

constexpr int kFactorWarps = 4;   // warps per CTA

// Copy the S rows of one cluster block (row_bytes each, contiguous in global
// memory) into shared memory with row pitch pitch_bytes, 16 bytes per lane
// and step.  row_bytes and pitch_bytes are multiples of 16.
__device__ __forceinline__ void stage_block(unsigned char *dst, const unsigned char *src, int S, int row_bytes,
                                            int pitch_bytes, int lane) {
    const int cpr = row_bytes >> 4;
    for (int q = lane; q < S * cpr; q += 32) {
        const int r = q / cpr, j = q - r * cpr;
        *reinterpret_cast<uint4 *>(dst + (size_t)r * pitch_bytes + j * 16) =
            __ldg(reinterpret_cast<const uint4 *>(src + (size_t)r * row_bytes + j * 16));
    }
}

// Operator of the persistent bulk-copy kernel: one warp per (subcarrier,
// cluster) task, row u per lane (lane group 0 stores).
template <int UT, typename TIn, int ALG>
__global__ void __launch_bounds__(kFactorWarps * 32) dbp_factor_kernel(const FactorParams p) {
    constexpr int EB = InTraits<TIn>::bytes;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u = lane % UT, g = lane / UT;
    unsigned char *wb = smem_raw + (size_t)warp * p.warp_bytes;
    const TIn *Hs = reinterpret_cast<const TIn *>(wb);
    float2 *Gm = reinterpret_cast<float2 *>(wb + p.off_g);
    float2 *Vb = reinterpret_cast<float2 *>(wb + p.off_v);
    // zero once: rows past S (16-bit inputs pad to a multiple of 8) stay zero
    for (int i = lane * 16; i < p.warp_bytes; i += 32 * 16)
        *reinterpret_cast<float4 *>(wb + i) = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
    grid_dependency_wait();
    grid_dependents_launch();
    const unsigned char *Hg = static_cast<const unsigned char *>(p.H);
    const long long tasks = (long long)p.W * p.C;
    for (long long task = (long long)blockIdx.x * kFactorWarps + warp; task < tasks;
         task += (long long)gridDim.x * kFactorWarps) {
        const int w = (int)(task / p.C), c = (int)(task - (long long)w * p.C);
        __syncwarp();   // the previous task's reads of the staging buffer are done
        stage_block(wb, Hg + ((size_t)w * p.B + (size_t)c * p.S) * UT * EB, p.S, UT * EB, p.hp * EB, lane);
        __syncwarp();
        float2 R[UT];
        cluster_operator<UT, TIn, ALG>(Hs, p.hp, p.h_rows, p.S, Gm, Vb, lane, u, g, p.f_delta, p.delta, true,
                                       p.retries, R);
        if (g == 0) {
            float2 *frow = p.factor + ((size_t)task * UT + u) * UT;
#pragma unroll
            for (int v = 0; v < UT; v += 2)
                *reinterpret_cast<float4 *>(&frow[v]) = make_float4(R[v].x, R[v].y, R[v + 1].x, R[v + 1].y);
        }
    }
}

// Operator of the U = 16 tensor-core downlink kernel: lane (ur, gc) stores
// entries (ur, 8 gc .. 8 gc + 7).  Per warp: H_c [S][16], B_c [16][QP],
// scratch for the FP64 retry (16 double2).
template <int UT>
__global__ void __launch_bounds__(kFactorWarps * 32) dbp_factor_tcdl_kernel(const FactorParams p) {
    static_assert(UT == TcDl::U, "the downlink tensor-core operator is for 16 users");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ur = lane & 15, gc = lane >> 4;
    unsigned char *wb = smem_raw + (size_t)warp * p.warp_bytes;
    const float2 *Hs = reinterpret_cast<const float2 *>(wb);
    float2 *Qs = reinterpret_cast<float2 *>(wb + p.off_g);
    float2 *Vb = reinterpret_cast<float2 *>(wb + p.off_v);
    grid_dependency_wait();
    grid_dependents_launch();
    const unsigned char *Hg = static_cast<const unsigned char *>(p.H);
    const long long tasks = (long long)p.W * p.C;
    for (long long task = (long long)blockIdx.x * kFactorWarps + warp; task < tasks;
         task += (long long)gridDim.x * kFactorWarps) {
        const int w = (int)(task / p.C), c = (int)(task - (long long)w * p.C);
        __syncwarp();
        stage_block(wb, Hg + ((size_t)w * p.B + (size_t)c * p.S) * UT * 8, p.S, UT * 8, UT * 8, lane);
        __syncwarp();
        float2 A[8];
        tcdl_operator(Hs, p.S, tcdl_h_scale(Hs, p.S, lane), Qs, Vb, lane, p.f_delta, p.delta, true, p.retries, A);
        float2 *frow = p.factor + ((size_t)task * UT + ur) * UT + 8 * gc;
#pragma unroll
        for (int i = 0; i < 8; i += 2)
            *reinterpret_cast<float4 *>(&frow[i]) = make_float4(A[i].x, A[i].y, A[i + 1].x, A[i + 1].y);
    }
}

}  // namespace dbp
