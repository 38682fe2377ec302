// dbp_factor.cu -- launches of the per-cluster operator kernels
// (dbp_factor.cuh): persistent grids of 4-warp CTAs, as many per SM as
// registers and shared memory allow, launched with programmatic stream
// serialisation like the fused kernels.
#include "dbp_launch.cuh"
#include "dbp_factor.cuh"

namespace {

template <typename K>
cudaError_t launch_factor_kernel(K kern, const dbp::FactorParams &p, size_t smem, int num_sms, cudaStream_t st) {
    cudaError_t e = dbp_prepare_kernel(reinterpret_cast<const void *>(kern), smem);
    if (e != cudaSuccess) return e;
    const int threads = dbp::kFactorWarps * 32;
    int occ = dbp_occupancy_cached(reinterpret_cast<const void *>(kern), threads, smem);
    if (occ < 1) occ = 1;
    const long long tasks = (long long)p.W * p.C;
    const long long need = (tasks + dbp::kFactorWarps - 1) / dbp::kFactorWarps;
    const long long slots = (long long)num_sms * occ;
    const unsigned grid = (unsigned)(need < slots ? need : slots);
    if (grid == 0) return cudaSuccess;
    return dbp::launch_pdl(kern, grid, (unsigned)threads, smem, st, p);
}

template <typename TIn>
cudaError_t launch_tma_operator(int UT, bool downlink, const dbp::FactorParams &p, size_t smem, int num_sms,
                                cudaStream_t st) {
    if (downlink) {
        if constexpr (sizeof(TIn) == 8) {
            if (UT == 16) return launch_factor_kernel(dbp::dbp_factor_kernel<16, TIn, dbp::ALG_ADMM_DL>, p, smem, num_sms, st);
            if (UT == 32) return launch_factor_kernel(dbp::dbp_factor_kernel<32, TIn, dbp::ALG_ADMM_DL>, p, smem, num_sms, st);
        }
        return cudaErrorInvalidValue;
    }
    if (UT == 16) return launch_factor_kernel(dbp::dbp_factor_kernel<16, TIn, dbp::ALG_ADMM_UL>, p, smem, num_sms, st);
    if (UT == 32) return launch_factor_kernel(dbp::dbp_factor_kernel<32, TIn, dbp::ALG_ADMM_UL>, p, smem, num_sms, st);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t dbp_launch_factor(int prec, int UT, bool downlink, bool tcdl, const dbp::FactorParams &p, size_t smem,
                              int num_sms, cudaStream_t st) {
    if (tcdl) {
        if (prec != DBP_FP32 || UT != 16 || !downlink) return cudaErrorInvalidValue;
        return launch_factor_kernel(dbp::dbp_factor_tcdl_kernel<16>, p, smem, num_sms, st);
    }
    switch (prec) {
    case DBP_FP32: return launch_tma_operator<float2>(UT, downlink, p, smem, num_sms, st);
    case DBP_FP16: return launch_tma_operator<__half2>(UT, downlink, p, smem, num_sms, st);
    case DBP_BF16: return launch_tma_operator<__nv_bfloat162>(UT, downlink, p, smem, num_sms, st);
    default: return cudaErrorInvalidValue;
    }
}
