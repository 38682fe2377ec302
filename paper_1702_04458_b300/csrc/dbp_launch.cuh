// dbp_launch.cuh -- launch of the fused kernels for one algorithm: the
// thread-block shape chosen on the host, and the template dispatch over
// precision, padded user count UT and CTA / thread-block-cluster mapping.
#pragma once

#include <cuda_runtime.h>

#include "dbp.h"
#include "dbp_fused.cuh"
#include "dbp_tma.cuh"
#include "dbp_mma8.cuh"
#include "dbp_cg.cuh"
#include "dbp_admm.cuh"
#include "dbp_tc8.cuh"
#include "dbp_tcdl.cuh"
#include "dbp_tc32.cuh"

// Host-side caches (dbp_api.cu): the dynamic shared-memory limit of a kernel
// is raised once per device and size, and the resident-CTA count of a
// (kernel, threads, shared memory) shape is queried once, so that a launch
// costs no driver attribute or occupancy call after the first.
cudaError_t dbp_prepare_kernel(const void *kern, size_t smem);
int dbp_occupancy_cached(const void *kern, int threads, size_t smem);

namespace dbp {

// Persistent kernels are launched with programmatic stream serialisation:
// their set-up (shared-memory zeroing, mbarrier initialisation) may overlap
// the end of the previous kernel in the stream, and they wait for it in
// grid_dependency_wait() before their first global access.
template <typename K, typename... Args>
cudaError_t launch_pdl(K kern, unsigned grid, unsigned block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(block, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Launch shape: CTA mapping (P whole subcarriers per CTA) when all C warps of
// a subcarrier fit in one CTA, else thread-block clusters of CL CTAs.
struct Shape {
    bool clu;
    bool tma;              // persistent bulk-copy kernel
    bool tc8 = false;      // U = 8 tensor-core uplink kernel
    bool tcdl = false;     // U = 16 tensor-core downlink kernel
    bool tc32 = false;     // U = S = 32 tcgen05 uplink ADMM kernel
    bool single = false;   // bulk-copy kernel with one staging buffer (uplink)
    bool bcast = false;    // consensus step once per symbol, result broadcast
    int P, CPB, CL, nwarps;
    long long grid;
    size_t smem;
    // bulk-copy kernel only: tiles, staging pitches and the per-warp layout
    int tiles = 0, hp = 0, yp = 0, h_rows = 0, y_rows = 0, ms_rows = 0;
    int off_h1 = 0, off_y0 = 0, off_y1 = 0, off_g = 0, off_v = 0, warp_bytes = 0;
};


template <typename T, int UT, int ALG, bool CLU>
cudaError_t launch_one(const FusedParams &p, const Shape &s, cudaStream_t st) {
    auto kern = dbp::dbp_fused_kernel<T, UT, ALG, CLU>;
    cudaError_t e = dbp_prepare_kernel(reinterpret_cast<const void *>(kern), s.smem);
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

template <int UT, int ALG, typename TIn>
cudaError_t launch_tma_one(const FusedParams &p, const Shape &s, cudaStream_t st) {
    auto kern = dbp::dbp_tma_kernel<UT, ALG, TIn>;
    cudaError_t e = dbp_prepare_kernel(reinterpret_cast<const void *>(kern), s.smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, (unsigned)s.grid, (unsigned)s.nwarps * 32, s.smem, st, p);
}

// Resident CTAs per SM of the persistent kernel at this shape.
template <int UT, int ALG, typename TIn>
int tma_occupancy_one(int threads, size_t smem) {
    auto kern = dbp::dbp_tma_kernel<UT, ALG, TIn>;
    return dbp_occupancy_cached(reinterpret_cast<const void *>(kern), threads, smem);
}

template <int ALG, typename TIn>
int tma_occupancy_ut(int UT, int threads, size_t smem) {
    switch (UT) {
    case 4: return tma_occupancy_one<4, ALG, TIn>(threads, smem);
    case 8: return tma_occupancy_one<8, ALG, TIn>(threads, smem);
    case 16: return tma_occupancy_one<16, ALG, TIn>(threads, smem);
    default: return tma_occupancy_one<32, ALG, TIn>(threads, smem);
    }
}

template <int ALG, typename TIn>
cudaError_t launch_tma_ut(int UT, const FusedParams &p, const Shape &s, cudaStream_t st) {
    switch (UT) {
    case 4: return launch_tma_one<4, ALG, TIn>(p, s, st);
    case 8: return launch_tma_one<8, ALG, TIn>(p, s, st);
    case 16: return launch_tma_one<16, ALG, TIn>(p, s, st);
    default: return launch_tma_one<32, ALG, TIn>(p, s, st);
    }
}

// Input storage precision -> kernel instance (16-bit inputs: uplink only).
template <int ALG>
int tma_occupancy(int prec, int UT, int threads, size_t smem) {
    if (prec == DBP_FP32) return tma_occupancy_ut<ALG, float2>(UT, threads, smem);
    if constexpr (ALG != ALG_ADMM_DL) {
        if (prec == DBP_FP16) return tma_occupancy_ut<ALG, __half2>(UT, threads, smem);
        if (prec == DBP_BF16) return tma_occupancy_ut<ALG, __nv_bfloat162>(UT, threads, smem);
    }
    return 0;
}

template <int ALG>
cudaError_t launch_tma(int prec, int UT, const FusedParams &p, const Shape &s, cudaStream_t st) {
    if (prec == DBP_FP32) return launch_tma_ut<ALG, float2>(UT, p, s, st);
    if constexpr (ALG != ALG_ADMM_DL) {
        if (prec == DBP_FP16) return launch_tma_ut<ALG, __half2>(UT, p, s, st);
        if (prec == DBP_BF16) return launch_tma_ut<ALG, __nv_bfloat162>(UT, p, s, st);
    }
    return cudaErrorInvalidValue;
}

template <int ALG>
int tc8_occupancy(int threads, size_t smem) {
    if constexpr (ALG == ALG_ADMM_DL) {
        return 0;
    } else {
        auto kern = dbp::dbp_tc8_kernel<ALG>;
        return dbp_occupancy_cached(reinterpret_cast<const void *>(kern), threads, smem);
    }
}

template <int ALG>
cudaError_t launch_tc8(const FusedParams &p, const Shape &s, cudaStream_t st) {
    if constexpr (ALG == ALG_ADMM_DL) {
        return cudaErrorInvalidValue;
    } else {
        auto kern = dbp::dbp_tc8_kernel<ALG>;
        cudaError_t e = dbp_prepare_kernel(reinterpret_cast<const void *>(kern), s.smem);
        if (e != cudaSuccess) return e;
                return launch_pdl(kern, (unsigned)s.grid, (unsigned)s.nwarps * 32, s.smem, st, p);
    }
}

template <int UT>
int cg_occupancy_one(int threads, size_t smem) {
    auto kern = dbp::dbp_cg_kernel<UT>;
    return dbp_occupancy_cached(reinterpret_cast<const void *>(kern), threads, smem);
}

template <int UT>
cudaError_t launch_cg_one(const FusedParams &p, const Shape &s, cudaStream_t st) {
    auto kern = dbp::dbp_cg_kernel<UT>;
    cudaError_t e = dbp_prepare_kernel(reinterpret_cast<const void *>(kern), s.smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, (unsigned)s.grid, (unsigned)s.nwarps * 32, s.smem, st, p);
}

template <int UT>
int admm_occupancy_one(int threads, size_t smem) {
    auto kern = dbp::dbp_admm_kernel<UT>;
    return dbp_occupancy_cached(reinterpret_cast<const void *>(kern), threads, smem);
}

template <int UT>
cudaError_t launch_admm_one(const FusedParams &p, const Shape &s, cudaStream_t st) {
    auto kern = dbp::dbp_admm_kernel<UT>;
    cudaError_t e = dbp_prepare_kernel(reinterpret_cast<const void *>(kern), s.smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, (unsigned)s.grid, (unsigned)s.nwarps * 32, s.smem, st, p);
}

// (a template so that only the unit that calls it compiles the kernel)
template <int = 0>
int tcdl_occupancy(int threads, size_t smem) {
    return dbp_occupancy_cached(reinterpret_cast<const void *>(dbp::dbp_tcdl_kernel<16>), threads, smem);
}

// (a template so that only the unit that calls it compiles the kernel)
template <int = 0>
cudaError_t launch_tcdl(const FusedParams &p, const Shape &s, cudaStream_t st) {
    cudaError_t e = dbp_prepare_kernel(reinterpret_cast<const void *>(dbp::dbp_tcdl_kernel<16>), s.smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(dbp::dbp_tcdl_kernel<16>, (unsigned)s.grid, (unsigned)s.nwarps * 32, s.smem, st, p);
}

template <typename TIn, int NS>
cudaError_t launch_tc32_one(const FusedParams &p, const Shape &s, cudaStream_t st) {
    auto kern = dbp::dbp_tc32_kernel<TIn, NS>;
    cudaError_t e = dbp_prepare_kernel(reinterpret_cast<const void *>(kern), s.smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, (unsigned)s.grid, (unsigned)tc32::THREADS, s.smem, st, p);
}

// The tcgen05 kernel keeps NS symbol slots in registers: 14 (the LTE slot)
// or 16 (any N <= 16).
template <typename TIn>
cudaError_t launch_tc32_n(const FusedParams &p, const Shape &s, cudaStream_t st) {
    return p.N == 14 ? launch_tc32_one<TIn, 14>(p, s, st) : launch_tc32_one<TIn, 16>(p, s, st);
}

// (a template so that only the unit that calls it compiles the kernel)
template <int = 0>
cudaError_t launch_tc32(int prec, const FusedParams &p, const Shape &s, cudaStream_t st) {
    switch (prec) {
    case DBP_FP32: return launch_tc32_n<float2>(p, s, st);
    case DBP_FP16: return launch_tc32_n<__half2>(p, s, st);
    case DBP_BF16: return launch_tc32_n<__nv_bfloat162>(p, s, st);
    default: return cudaErrorInvalidValue;
    }
}

// Resident CTAs per SM of the tcgen05 kernel: from the device's shared
// memory and register file directly (the kernel is built for two: 128
// registers per thread, 104 KB of shared memory, 256 tensor-memory columns).
template <typename TIn, int NS>
int tc32_occupancy_one() {
    cudaFuncSetAttribute(dbp::dbp_tc32_kernel<TIn, NS>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (dbp_prepare_kernel(reinterpret_cast<const void *>(dbp::dbp_tc32_kernel<TIn, NS>), tc32::SMEM) != cudaSuccess)
        return 1;
    int dev = 0, smem_sm = 0, smem_block_reserved = 0, regs_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_block_reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, dbp::dbp_tc32_kernel<TIn, NS>) != cudaSuccess) return 1;
    const int by_smem = smem_sm / (tc32::SMEM + smem_block_reserved);
    const int by_regs = regs_sm / (fa.numRegs * tc32::THREADS);
    int occ = by_smem < by_regs ? by_smem : by_regs;
    if (occ > 2) occ = 2;        // 2 x 256 tensor-memory columns
    return occ < 1 ? 1 : occ;
}

template <int ALG>
cudaError_t launch_alg(int prec, int UT, const FusedParams &p, const Shape &s, cudaStream_t st) {
    if constexpr (ALG == ALG_ADMM_DL) {
        if (s.tcdl) return launch_tcdl(p, s, st);
    }
    if constexpr (ALG == ALG_CG_UL) {
        if (s.bcast) {
            switch (UT) {
            case 4: return launch_cg_one<4>(p, s, st);
            case 8: return launch_cg_one<8>(p, s, st);
            case 16: return launch_cg_one<16>(p, s, st);
            default: return cudaErrorInvalidValue;
            }
        }
    }
    if constexpr (ALG == ALG_ADMM_UL) {
        if (s.tc32) return launch_tc32(prec, p, s, st);
        if (s.bcast) {
            switch (UT) {
            case 4: return launch_admm_one<4>(p, s, st);
            case 8: return launch_admm_one<8>(p, s, st);
            case 16: return launch_admm_one<16>(p, s, st);
            default: return cudaErrorInvalidValue;
            }
        }
    }
    if (s.tc8) return launch_tc8<ALG>(p, s, st);
    if (s.tma) return launch_tma<ALG>(prec, UT, p, s, st);
    if (prec != DBP_FP32 && prec != DBP_FP64) return cudaErrorInvalidValue;
    if (prec == DBP_FP32)
        return s.clu ? launch_ut<float, ALG, true>(UT, p, s, st) : launch_ut<float, ALG, false>(UT, p, s, st);
    return s.clu ? launch_ut<double, ALG, true>(UT, p, s, st) : launch_ut<double, ALG, false>(UT, p, s, st);
}


}  // namespace dbp

// One translation unit per algorithm instantiates its kernels.
cudaError_t dbp_launch_admm_ul(int prec, int UT, const dbp::FusedParams &p, const dbp::Shape &s, cudaStream_t st);
cudaError_t dbp_launch_cg_ul(int prec, int UT, const dbp::FusedParams &p, const dbp::Shape &s, cudaStream_t st);
cudaError_t dbp_launch_admm_dl(int prec, int UT, const dbp::FusedParams &p, const dbp::Shape &s, cudaStream_t st);
int dbp_tma_occupancy_admm_ul(int prec, int UT, int threads, size_t smem);
int dbp_tma_occupancy_cg_ul(int prec, int UT, int threads, size_t smem);
int dbp_tma_occupancy_admm_dl(int prec, int UT, int threads, size_t smem);
int dbp_tc8_occupancy_admm_ul(int threads, size_t smem);
int dbp_tc8_occupancy_cg_ul(int threads, size_t smem);
int dbp_cg_occupancy(int UT, int threads, size_t smem);
int dbp_bcast_admm_occupancy(int UT, int threads, size_t smem);
int dbp_tcdl_occupancy(int threads, size_t smem);
int dbp_tc32_occupancy(int prec, int N);

// The per-cluster operator kernels (dbp_factor.cu): B_c^{-1} of every
// (subcarrier, cluster) of the frame into p.factor, for the bulk-copy kernel's
// layout (tcdl = false; 16-bit or FP32 inputs, U in {16, 32}) or the U = 16
// tensor-core downlink kernel's (tcdl = true).  Returns cudaErrorInvalidValue
// for a combination that has no instance.
namespace dbp { struct FactorParams; }
cudaError_t dbp_launch_factor(int prec, int UT, bool downlink, bool tcdl, const dbp::FactorParams &p, size_t smem,
                              int num_sms, cudaStream_t st);
