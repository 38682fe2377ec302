// dbp_k_cg_ul.cu -- instantiates the fused kernels of one algorithm.
#include "dbp_launch.cuh"

cudaError_t dbp_launch_cg_ul(int prec, int UT, const dbp::FusedParams &p, const dbp::Shape &s, cudaStream_t st) {
    return dbp::launch_alg<dbp::ALG_CG_UL>(prec, UT, p, s, st);
}

int dbp_tma_occupancy_cg_ul(int prec, int UT, int threads, size_t smem) {
    return dbp::tma_occupancy<dbp::ALG_CG_UL>(prec, UT, threads, smem);
}

int dbp_tc8_occupancy_cg_ul(int threads, size_t smem) { return dbp::tc8_occupancy<dbp::ALG_CG_UL>(threads, smem); }

int dbp_cg_occupancy(int UT, int threads, size_t smem) {
    switch (UT) {
    case 4: return dbp::cg_occupancy_one<4>(threads, smem);
    case 8: return dbp::cg_occupancy_one<8>(threads, smem);
    case 16: return dbp::cg_occupancy_one<16>(threads, smem);
    default: return 0;
    }
}
