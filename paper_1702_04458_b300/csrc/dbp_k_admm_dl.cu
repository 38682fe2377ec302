// dbp_k_admm_dl.cu -- instantiates the fused kernels of one algorithm.
#include "dbp_launch.cuh"

cudaError_t dbp_launch_admm_dl(int prec, int UT, const dbp::FusedParams &p, const dbp::Shape &s, cudaStream_t st) {
    return dbp::launch_alg<dbp::ALG_ADMM_DL>(prec, UT, p, s, st);
}

int dbp_tma_occupancy_admm_dl(int prec, int UT, int threads, size_t smem) {
    return dbp::tma_occupancy<dbp::ALG_ADMM_DL>(prec, UT, threads, smem);
}

int dbp_tcdl_occupancy(int threads, size_t smem) { return dbp::tcdl_occupancy(threads, smem); }
