// dbp_static.cu -- downlink beamforming with power normalisation for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: processes whose device memory is
// fully reserved by another allocator or pool, and embedded / real-time
// front ends that must not allocate once they are running.
// dbp_downlink_admm with DBP_FLAG_NORMALIZE allocates a small device
// accumulator on first use; this variant needs no allocation at all:
// its scratch (one partial energy per subcarrier) lives in a file-scope
// device array of fixed size that every GPU which loads the library keeps
// until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "dbp.h"
#include "dbp_fused.cuh"
#include "dbp_internal.h"

namespace {

// Scratch: per-subcarrier sums of |x|^2, then the frame total and beta.
static __device__ __align__(256) double g_dl_energy[DBP_STATIC_MAX_SUBCARRIERS + 2];

constexpr int kMaxDevices = 128;
std::mutex g_setup_mu;
double *g_scratch[kMaxDevices] = {};   // device address of g_dl_energy per device

// Per-device set-up: with `device` current, translate the symbol into a
// device address.  In host code g_dl_energy names a host-side stand-in, not
// device memory, so kernels must be given this address instead.  The
// address is kept for the life of the process: after cudaDeviceReset the
// device's context (and this array) is new, so the entry point must not be
// used after a reset.
dbp_status scratch_for(int device, double **out) {
    if (device < 0 || device >= kMaxDevices) return DBP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (g_scratch[device] == nullptr) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_dl_energy);
        if (e != cudaSuccess || p == nullptr) return DBP_ERR_CUDA;
        g_scratch[device] = static_cast<double *>(p);
    }
    *out = g_scratch[device];
    return DBP_OK;
}

// One block per subcarrier (grid-stride): fixed-order tree sum of |x|^2 over
// the subcarrier's N*B entries, written to partial[w].
template <typename C2>
__global__ void energy_per_subcarrier(const C2 *x, int W, size_t per_w, double *partial) {
    __shared__ double red[256];
    for (int w = blockIdx.x; w < W; w += gridDim.x) {
        const C2 *xw = x + (size_t)w * per_w;
        double acc = 0.0;
        for (size_t i = threadIdx.x; i < per_w; i += blockDim.x)
            acc += (double)xw[i].x * xw[i].x + (double)xw[i].y * xw[i].y;
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int st = blockDim.x / 2; st > 0; st >>= 1) {
            if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[w] = red[0];
        __syncthreads();
    }
}

// Single block: frame total in a fixed order and beta = sqrt(count / total).
__global__ void energy_total(double *scratch, int W, double count, double *beta_out) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int w = threadIdx.x; w < W; w += blockDim.x) acc += scratch[w];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double total = red[0];
        const double beta = total > 0.0 ? sqrt(count / total) : 0.0;
        scratch[DBP_STATIC_MAX_SUBCARRIERS] = total;
        scratch[DBP_STATIC_MAX_SUBCARRIERS + 1] = beta;
        if (beta_out) *beta_out = beta;
    }
}

template <typename C2, typename T>
__global__ void scale_by_beta(C2 *x, size_t n, const double *scratch) {
    const T b = (T)scratch[DBP_STATIC_MAX_SUBCARRIERS + 1];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        x[i].x *= b;
        x[i].y *= b;
    }
}

}  // namespace

namespace {
dbp_status fail_static(dbp_context *h, dbp_status st, const std::string &msg) {
    h->err = "dbp_downlink_admm_static: " + msg;
    return st;
}
}  // namespace

extern "C" dbp_status dbp_downlink_admm_static(dbp_handle_t h, const dbp_frame_desc *d, const void *H,
                                               const void *s, void *x, double *beta_out, void *stream) {
    if (!h) return DBP_ERR_INVALID_ARG;
    if (!d) return fail_static(h, DBP_ERR_INVALID_ARG, "descriptor is NULL");
    if (d->W < 0 || d->N < 0 || d->B <= 0) return fail_static(h, DBP_ERR_INVALID_ARG, "bad shape");
    if (d->W > DBP_STATIC_MAX_SUBCARRIERS)
        return fail_static(h, DBP_ERR_UNSUPPORTED,
                           "W = " + std::to_string(d->W) + " exceeds the fixed scratch of " +
                               std::to_string(DBP_STATIC_MAX_SUBCARRIERS) + " subcarriers");

    // The precoder itself: the fused kernel of dbp_downlink_admm, without its
    // allocating normalisation.  It also makes the handle's device current.
    dbp_frame_desc dd = *d;
    dd.flags &= ~DBP_FLAG_NORMALIZE;
    DbpExec ex;
    ex.no_workspace = true;     // no operator buffer either
    dbp_status st = dbp_run_internal(h, &dd, DBP_K_ADMM_DL, H, s, x, nullptr, nullptr, (cudaStream_t)stream, &ex,
                                     nullptr, nullptr);
    if (st != DBP_OK) return st;
    if (!(d->flags & DBP_FLAG_NORMALIZE) || (long long)d->W * d->N == 0) return DBP_OK;

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return fail_static(h, DBP_ERR_CUDA, "cudaGetDevice failed");
    double *scratch = nullptr;
    st = scratch_for(device, &scratch);
    if (st != DBP_OK) return fail_static(h, st, "no device address for the scratch array");

    // An error left by earlier, unrelated work is reported as such, not as
    // one of these launches (and is not cleared).
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess)
        return fail_static(h, DBP_ERR_CUDA, std::string("a CUDA error from earlier work is pending: ") +
                                                cudaGetErrorString(pending));
    cudaStream_t cs = (cudaStream_t)stream;
    const size_t per_w = (size_t)d->N * d->B;
    const size_t n = per_w * d->W;
    const double count = (double)n;
    const int blocks = d->W < 4096 ? d->W : 4096;
    const size_t sb = (n + 4 * 256 - 1) / (4 * 256);         // about four elements per thread
    const int sblocks = (int)(sb < 1184 ? (sb < 1 ? 1 : sb) : 1184);
    const char *what = "energy_per_subcarrier";
    cudaError_t e;
    if (d->precision == DBP_FP32) {
        energy_per_subcarrier<float2><<<blocks, 256, 0, cs>>>((const float2 *)x, d->W, per_w, scratch);
        if ((e = cudaGetLastError()) == cudaSuccess) {
            what = "energy_total";
            energy_total<<<1, 256, 0, cs>>>(scratch, d->W, count, beta_out);
        }
        if (e == cudaSuccess && (e = cudaGetLastError()) == cudaSuccess) {
            what = "scale_by_beta";
            scale_by_beta<float2, float><<<sblocks, 256, 0, cs>>>((float2 *)x, n, scratch);
            e = cudaGetLastError();
        }
    } else {
        energy_per_subcarrier<double2><<<blocks, 256, 0, cs>>>((const double2 *)x, d->W, per_w, scratch);
        if ((e = cudaGetLastError()) == cudaSuccess) {
            what = "energy_total";
            energy_total<<<1, 256, 0, cs>>>(scratch, d->W, count, beta_out);
        }
        if (e == cudaSuccess && (e = cudaGetLastError()) == cudaSuccess) {
            what = "scale_by_beta";
            scale_by_beta<double2, double><<<sblocks, 256, 0, cs>>>((double2 *)x, n, scratch);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess)
        return fail_static(h, DBP_ERR_CUDA, std::string(what) + " launch: " + cudaGetErrorString(e));
    return DBP_OK;
}
