// dbp_launch.cuh -- launch of the fused kernels for one algorithm: the
// thread-block shape chosen on the host, and the template dispatch over
// precision, padded user count UT and CTA / thread-block-cluster mapping.
#pragma once

#include <cuda_runtime.h>

#include "dbp.h"
#include "dbp_fused.cuh"

namespace dbp {

// Launch shape: CTA mapping (P whole subcarriers per CTA) when all C warps of
// a subcarrier fit in one CTA, else thread-block clusters of CL CTAs.
struct Shape {
    bool clu;
    int P, CPB, CL, nwarps;
    long long grid;
    size_t smem;
};


template <typename T, int UT, int ALG, bool CLU>
cudaError_t launch_one(const FusedParams &p, const Shape &s, cudaStream_t st) {
    auto kern = dbp::dbp_fused_kernel<T, UT, ALG, CLU>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
    if (e != cudaSuccess) return e;
    if (!CLU) {
        kern<<<(unsigned)s.grid, s.nwarps * 32, s.smem, st>>>(p);
        return cudaGetLastError();
    }
    if (s.CL > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)s.grid, 1, 1);
    cfg.blockDim = dim3(s.nwarps * 32, 1, 1);
    cfg.dynamicSmemBytes = s.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = s.CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p);
}

template <typename T, int ALG, bool CLU>
cudaError_t launch_ut(int UT, const FusedParams &p, const Shape &s, cudaStream_t st) {
    switch (UT) {
    case 4: return launch_one<T, 4, ALG, CLU>(p, s, st);
    case 8: return launch_one<T, 8, ALG, CLU>(p, s, st);
    case 16: return launch_one<T, 16, ALG, CLU>(p, s, st);
    default:
        if constexpr (sizeof(T) == 4) return launch_one<T, 32, ALG, CLU>(p, s, st);
        else return cudaErrorInvalidValue;  // FP64 supports U <= 16
    }
}

template <int ALG>
cudaError_t launch_alg(int prec, int UT, const FusedParams &p, const Shape &s, cudaStream_t st) {
    if (prec == DBP_FP32)
        return s.clu ? launch_ut<float, ALG, true>(UT, p, s, st) : launch_ut<float, ALG, false>(UT, p, s, st);
    return s.clu ? launch_ut<double, ALG, true>(UT, p, s, st) : launch_ut<double, ALG, false>(UT, p, s, st);
}


}  // namespace dbp

// One translation unit per algorithm instantiates its kernels.
cudaError_t dbp_launch_admm_ul(int prec, int UT, const dbp::FusedParams &p, const dbp::Shape &s, cudaStream_t st);
cudaError_t dbp_launch_cg_ul(int prec, int UT, const dbp::FusedParams &p, const dbp::Shape &s, cudaStream_t st);
cudaError_t dbp_launch_admm_dl(int prec, int UT, const dbp::FusedParams &p, const dbp::Shape &s, cudaStream_t st);
