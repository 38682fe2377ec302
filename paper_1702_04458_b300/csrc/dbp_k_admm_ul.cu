// dbp_k_admm_ul.cu -- instantiates the fused kernels of one algorithm.
#include "dbp_launch.cuh"

cudaError_t dbp_launch_admm_ul(int prec, int UT, const dbp::FusedParams &p, const dbp::Shape &s, cudaStream_t st) {
    return dbp::launch_alg<dbp::ALG_ADMM_UL>(prec, UT, p, s, st);
}

int dbp_tma_occupancy_admm_ul(int prec, int UT, int threads, size_t smem) {
    return dbp::tma_occupancy<dbp::ALG_ADMM_UL>(prec, UT, threads, smem);
}

int dbp_tc8_occupancy_admm_ul(int threads, size_t smem) { return dbp::tc8_occupancy<dbp::ALG_ADMM_UL>(threads, smem); }

int dbp_bcast_admm_occupancy(int UT, int threads, size_t smem) {
    switch (UT) {
    case 4: return dbp::admm_occupancy_one<4>(threads, smem);
    case 8: return dbp::admm_occupancy_one<8>(threads, smem);
    case 16: return dbp::admm_occupancy_one<16>(threads, smem);
    default: return 0;
    }
}

int dbp_tc32_occupancy(int prec, int N) {
    const bool n14 = (N == 14);
    switch (prec) {
    case DBP_FP32: return n14 ? dbp::tc32_occupancy_one<float2, 14>() : dbp::tc32_occupancy_one<float2, 16>();
    case DBP_FP16: return n14 ? dbp::tc32_occupancy_one<__half2, 14>() : dbp::tc32_occupancy_one<__half2, 16>();
    case DBP_BF16:
        return n14 ? dbp::tc32_occupancy_one<__nv_bfloat162, 14>() : dbp::tc32_occupancy_one<__nv_bfloat162, 16>();
    default: return 0;
    }
}
