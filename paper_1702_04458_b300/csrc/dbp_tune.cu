// dbp_tune.cu -- autotuner: time the launch choices that accept a frame and
// remember the fastest per frame shape on the handle.
//
// The candidates are every kernel path (tensor-core, broadcast, persistent
// bulk-copy, generic) with 4, 8 and 16 warps per CTA, the tensor-core and
// bulk-copy paths with and without the separate operator kernel, and for the
// generic kernel also thread-block clusters of 2, 4, 8 and 16 CTAs.  A
// candidate that does not accept the shape is skipped, and so is an
// operator-kernel candidate where that kernel does not apply.  Each is run
// twice untimed and then `reps` times between two CUDA events on the
// caller's stream.
#include <cuda_runtime.h>

#include <cstdio>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "dbp.h"
#include "dbp_internal.h"

namespace {

std::vector<dbp_tuning> candidates(int C) {
    std::vector<dbp_tuning> out;
    const int paths[] = {DBP_PATH_TC5, DBP_PATH_MMA, DBP_PATH_BCAST, DBP_PATH_TMA, DBP_PATH_GENERIC};
    const int wpcs[] = {0, 4, 16};
    for (int k : paths)
        for (int w : wpcs) {
            if (k == DBP_PATH_TC5 && w != 0) continue;   // one CTA shape
            out.push_back(dbp_tuning{DBP_MAP_CTA, 0, w, k, DBP_PREFACTOR_OFF});
            if (k == DBP_PATH_MMA || k == DBP_PATH_TMA)
                out.push_back(dbp_tuning{DBP_MAP_CTA, 0, w, k, DBP_PREFACTOR_ON});
        }
    for (int cl = 2; cl <= 16; cl *= 2)
        if (C % cl == 0) out.push_back(dbp_tuning{DBP_MAP_CLUSTER, cl, 0, DBP_PATH_GENERIC, DBP_PREFACTOR_OFF});
    return out;
}

bool valid_tuning(const dbp_tuning &t) {
    return t.mapping >= DBP_MAP_AUTO && t.mapping <= DBP_MAP_CLUSTER && t.cluster_size >= 0 &&
           t.cluster_size <= 16 && t.warps_per_cta >= 0 && t.warps_per_cta <= 32 &&
           t.kernel >= DBP_PATH_AUTO && t.kernel <= DBP_PATH_TC5 && t.prefactor >= DBP_PREFACTOR_AUTO &&
           t.prefactor <= DBP_PREFACTOR_ON;
}

}  // namespace

extern "C" {

dbp_status dbp_autotune(dbp_handle_t h, int32_t kind, const dbp_frame_desc *d, const void *H, const void *in,
                        void *out, uint8_t *labels, void *stream, int32_t reps, dbp_tuning *best) {
    if (!h) return DBP_ERR_INVALID_ARG;
    if (kind < DBP_KIND_UPLINK_ADMM || kind > DBP_KIND_DOWNLINK_ADMM) {
        h->err = "dbp_autotune: unknown kind";
        return DBP_ERR_INVALID_ARG;
    }
    std::string err;
    dbp_status v = dbp_validate_internal(h, d, kind, &err);
    if (v != DBP_OK) {
        h->err = err;
        return v;
    }
    if (reps == 0) reps = 10;
    if (reps < 1 || reps > 10000) {
        h->err = "dbp_autotune: reps must be in 1..10000";
        return DBP_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) {
        h->err = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
        return DBP_ERR_CUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        h->err = "dbp_autotune: cudaEventCreate failed";
        return DBP_ERR_CUDA;
    }
    dbp_tuning saved;
    {
        std::lock_guard<std::mutex> lk(h->tune_mu);
        saved = h->tuning;
    }
    dbp_tuning chosen{};
    float best_ms = -1.f;
    dbp_status st_out = DBP_OK;
    for (const dbp_tuning &t : candidates(d->C)) {
        // an operator-kernel candidate where that kernel does not apply is
        // the same launch as its DBP_PREFACTOR_OFF twin
        if (t.prefactor == DBP_PREFACTOR_ON && !dbp_prefactor_applies(h, d, kind, t, H, in, out)) continue;
        {
            std::lock_guard<std::mutex> lk(h->tune_mu);
            h->tuning = t;
        }
        std::string e2;
        dbp_status r = DBP_OK;
        for (int i = 0; i < 2 && r == DBP_OK; ++i)
            r = dbp_run_internal(h, d, kind, H, in, out, labels, nullptr, st, nullptr, nullptr, &e2);
        if (r == DBP_ERR_UNSUPPORTED || r == DBP_ERR_INVALID_ARG) continue;   // not for this shape
        if (r != DBP_OK) {
            st_out = r;
            h->err = e2;
            break;
        }
        cudaEventRecord(e0, st);
        for (int i = 0; i < reps && r == DBP_OK; ++i)
            r = dbp_run_internal(h, d, kind, H, in, out, labels, nullptr, st, nullptr, nullptr, &e2);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || r != DBP_OK) {
            st_out = (r != DBP_OK) ? r : DBP_ERR_CUDA;
            h->err = (r != DBP_OK) ? e2 : std::string("dbp_autotune: event synchronisation failed");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best_ms < 0.f || ms < best_ms) {
            best_ms = ms;
            chosen = t;
        }
    }
    {
        std::lock_guard<std::mutex> lk(h->tune_mu);
        h->tuning = saved;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st_out != DBP_OK) return st_out;
    if (best_ms < 0.f) {
        h->err = "dbp_autotune: no launch choice accepts this frame";
        return DBP_ERR_UNSUPPORTED;
    }
    {
        std::lock_guard<std::mutex> lk(h->tune_mu);
        h->tuned[dbp_tune_key(d, kind)] = chosen;
    }
    if (best) *best = chosen;
    return DBP_OK;
}

dbp_status dbp_autotune_clear(dbp_handle_t h) {
    if (!h) return DBP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(h->tune_mu);
    h->tuned.clear();
    return DBP_OK;
}

dbp_status dbp_autotune_save(dbp_handle_t h, const char *path) {
    if (!h) return DBP_ERR_INVALID_ARG;
    if (!path) {
        h->err = "dbp_autotune_save: NULL path";
        return DBP_ERR_INVALID_ARG;
    }
    std::ofstream f(path);
    if (!f) {
        h->err = std::string("dbp_autotune_save: cannot write ") + path;
        return DBP_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(h->tune_mu);
    for (const auto &kv : h->tuned) {
        const auto &k = kv.first;
        const dbp_tuning &t = kv.second;
        f << std::get<0>(k) << ' ' << std::get<1>(k) << ' ' << std::get<2>(k) << ' ' << std::get<3>(k) << ' '
          << std::get<4>(k) << ' ' << std::get<5>(k) << ' ' << t.mapping << ' ' << t.cluster_size << ' '
          << t.warps_per_cta << ' ' << t.kernel << ' ' << t.prefactor << '\n';
    }
    return f ? DBP_OK : DBP_ERR_INVALID_ARG;
}

dbp_status dbp_autotune_load(dbp_handle_t h, const char *path) {
    if (!h) return DBP_ERR_INVALID_ARG;
    if (!path) {
        h->err = "dbp_autotune_load: NULL path";
        return DBP_ERR_INVALID_ARG;
    }
    std::ifstream f(path);
    if (!f) {
        h->err = std::string("dbp_autotune_load: cannot read ") + path;
        return DBP_ERR_INVALID_ARG;
    }
    std::vector<std::pair<std::tuple<int, int, int, int, int, int>, dbp_tuning>> rows;
    std::string line;
    int lineno = 0;
    while (std::getline(f, line)) {
        ++lineno;
        if (line.find_first_not_of(" \t\r") == std::string::npos) continue;
        std::istringstream is(line);
        int kind, B, C, U, N, prec;
        dbp_tuning t{};
        std::string extra;
        if (!(is >> kind >> B >> C >> U >> N >> prec >> t.mapping >> t.cluster_size >> t.warps_per_cta >> t.kernel >>
              t.prefactor) ||
            (is >> extra) || kind < 0 || kind > 2 || !valid_tuning(t)) {
            h->err = std::string("dbp_autotune_load: malformed line ") + std::to_string(lineno) + " of " + path;
            return DBP_ERR_INVALID_ARG;
        }
        rows.push_back({std::make_tuple(kind, B, C, U, N, prec), t});
    }
    std::lock_guard<std::mutex> lk(h->tune_mu);
    for (const auto &r : rows) h->tuned[r.first] = r.second;
    return DBP_OK;
}

}  // extern "C"
