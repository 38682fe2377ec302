// dbp_internal.h -- host-side definitions shared by the library's
// translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "dbp.h"

struct dbp_server;

struct dbp_context {
    int device = 0;
    uint64_t budget = 0;                 // cap on library-owned device memory (0: none)
    uint64_t used = 0;                   // library-owned device memory in use
    int num_sms = 0;
    size_t smem_optin = 0;
    std::string err;
    dbp_tuning tuning{};
    uint32_t test_faults = 0;            // dbp_set_test_faults
    double *energy = nullptr;            // downlink power accumulator
    int *status = nullptr;               // device status word of the kernels
    void *dev[4] = {nullptr, nullptr, nullptr, nullptr};   // host-variant buffers
    size_t dev_cap[4] = {0, 0, 0, 0};
    // host variants in chunks: streams for the input copies, the kernels and
    // the output copies, and their events (start, inputs and kernel of each
    // chunk, end)
    static constexpr int kPipeMax = 8;
    cudaStream_t pipe[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t pipe_ev[2 * kPipeMax + 2] = {};
    dbp_server *server = nullptr;        // request loop (dbp_server_start)
    // autotuned launch choices per frame shape (kind, B, C, U, N, precision)
    std::mutex tune_mu;
    std::map<std::tuple<int, int, int, int, int, int>, dbp_tuning> tuned;
    // stream-ordered pool of the per-call operator buffers (dbp_factor.cuh)
    std::mutex pool_mu;
    cudaMemPool_t factor_pool = nullptr;
};

inline std::tuple<int, int, int, int, int, int> dbp_tune_key(const dbp_frame_desc *d, int kind) {
    return std::make_tuple(kind, d->B, d->C, d->U, d->N, d->precision);
}


enum DbpKind { DBP_K_ADMM_UL = 0, DBP_K_CG_UL = 1, DBP_K_ADMM_DL = 2 };

// Per-call resources supplied by the request loop instead of the handle's.
struct DbpExec {
    double *energy = nullptr;      // downlink power accumulator (one double)
    float2 *factor = nullptr;      // resident operator [W][C][UT][UT]
    int factor_mode = 0;           // 0 none, 1 compute and store, 2 load
    bool no_workspace = false;     // allocate nothing (no separate operator kernel)
};

// Validate and enqueue one frame on `st` (errors go to *err when non-null).
// *factor_used reports whether the kernel that ran can store / load the
// resident operator (the persistent bulk-copy kernel).
dbp_status dbp_run_internal(dbp_context *h, const dbp_frame_desc *d, int kind, const void *H, const void *vin,
                            void *out, uint8_t *labels, double *beta_out, cudaStream_t st, const DbpExec *ex,
                            bool *factor_used, std::string *err);
dbp_status dbp_validate_internal(dbp_context *h, const dbp_frame_desc *d, int kind, std::string *err);
dbp_status dbp_plan_internal(dbp_context *h, const dbp_frame_desc *d, int kind, const void *H, const void *vin,
                             const void *out, dbp_tuning *chosen);
// Whether a call with tuning t would run the separate operator kernel
// (DBP_PREFACTOR_ON on a shape where it is available).
bool dbp_prefactor_applies(dbp_context *h, const dbp_frame_desc *d, int kind, const dbp_tuning &t, const void *H,
                           const void *vin, const void *out);
size_t dbp_in_elem_bytes(int prec);
size_t dbp_out_elem_bytes(int prec);
int dbp_padded_users(int U);
void dbp_server_destroy(dbp_server *s);
