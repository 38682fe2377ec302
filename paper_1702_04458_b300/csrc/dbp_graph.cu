// dbp_graph.cu -- a batch of frames of mixed kinds and shapes captured into
// one CUDA graph and run by a single launch (the batching pattern: many
// small per-frame launches become one graph launch, with the frames on
// independent branches so that different shapes overlap on the device).
#include <cuda_runtime.h>

#include <cstdio>
#include <string>
#include <vector>

#include "dbp.h"
#include "dbp_internal.h"

struct dbp_graph {
    dbp_context *h = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double *energy = nullptr;      // one downlink power accumulator per item
};

namespace {

dbp_status graph_fail(dbp_context *h, dbp_status st, const std::string &msg) {
    h->err = msg;
    return st;
}

void release(dbp_graph *g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->energy) cudaFree(g->energy);
    delete g;
}

}  // namespace

extern "C" {

dbp_status dbp_graph_create(dbp_handle_t h, const dbp_graph_item *items, int32_t n, int32_t branches,
                            dbp_graph_t *out) {
    if (!h) return DBP_ERR_INVALID_ARG;
    if (!out || n < 1 || (n > 0 && !items))
        return graph_fail(h, DBP_ERR_INVALID_ARG, "dbp_graph_create needs n >= 1 items and an output handle");
    *out = nullptr;
    if (branches == 0) branches = 4;
    if (branches < 1 || branches > 16)
        return graph_fail(h, DBP_ERR_INVALID_ARG, "branches must be in 1..16");
    for (int i = 0; i < n; ++i) {
        std::string err;
        const dbp_graph_item &it = items[i];
        if (it.kind < DBP_KIND_UPLINK_ADMM || it.kind > DBP_KIND_DOWNLINK_ADMM)
            return graph_fail(h, DBP_ERR_INVALID_ARG, "item " + std::to_string(i) + ": unknown kind");
        dbp_status v = dbp_validate_internal(h, &it.desc, it.kind, &err);
        if (v != DBP_OK) return graph_fail(h, v, "item " + std::to_string(i) + ": " + err);
    }
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return graph_fail(h, DBP_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));

    dbp_graph *g = new dbp_graph;
    g->h = h;
    e = cudaMalloc(&g->energy, sizeof(double) * (size_t)n);
    if (e != cudaSuccess) {
        release(g);
        return graph_fail(h, DBP_ERR_NOMEM, std::string("cudaMalloc(graph scratch): ") + cudaGetErrorString(e));
    }

    // origin stream, fork into the branch streams, capture, join
    std::vector<cudaStream_t> br((size_t)branches, nullptr);
    cudaStream_t origin = nullptr;
    std::vector<cudaEvent_t> ev((size_t)branches + 1, nullptr);
    auto cleanup_streams = [&]() {
        for (auto &s : br)
            if (s) cudaStreamDestroy(s);
        if (origin) cudaStreamDestroy(origin);
        for (auto &x : ev)
            if (x) cudaEventDestroy(x);
    };
    e = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
    for (int b = 0; b < branches && e == cudaSuccess; ++b) e = cudaStreamCreateWithFlags(&br[b], cudaStreamNonBlocking);
    for (size_t k = 0; k < ev.size() && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cleanup_streams();
        release(g);
        return graph_fail(h, DBP_ERR_CUDA, std::string("graph streams: ") + cudaGetErrorString(e));
    }

    dbp_status st = DBP_OK;
    std::string err;
    e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        cudaEventRecord(ev[0], origin);
        for (int b = 0; b < branches; ++b) cudaStreamWaitEvent(br[b], ev[0], 0);
        for (int i = 0; i < n && st == DBP_OK; ++i) {
            const dbp_graph_item &it = items[i];
            DbpExec ex;
            ex.energy = g->energy + i;
            st = dbp_run_internal(h, &it.desc, it.kind, it.H, it.in, it.out, it.labels, it.beta_out,
                                  br[(size_t)(i % branches)], &ex, nullptr, &err);
            if (st != DBP_OK) err = "item " + std::to_string(i) + ": " + err;
        }
        for (int b = 0; b < branches; ++b) {
            cudaEventRecord(ev[(size_t)b + 1], br[b]);
            cudaStreamWaitEvent(origin, ev[(size_t)b + 1], 0);
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(origin, &graph);
        g->graph = graph;
        if (st == DBP_OK && ee != cudaSuccess) {
            st = DBP_ERR_CUDA;
            err = std::string("stream capture: ") + cudaGetErrorString(ee);
        }
    } else {
        st = DBP_ERR_CUDA;
        err = std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e);
    }
    cleanup_streams();
    if (st == DBP_OK) {
        e = cudaGraphInstantiate(&g->exec, g->graph, 0);
        if (e != cudaSuccess) {
            st = DBP_ERR_CUDA;
            err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
        }
    }
    if (st != DBP_OK) {
        release(g);
        return graph_fail(h, st, err);
    }
    *out = g;
    return DBP_OK;
}

dbp_status dbp_graph_launch(dbp_graph_t g, void *stream) {
    if (!g || !g->exec) return DBP_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(g->h->device);
    if (e == cudaSuccess) e = cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return graph_fail(g->h, DBP_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
    return DBP_OK;
}

dbp_status dbp_graph_destroy(dbp_graph_t g) {
    if (!g) return DBP_ERR_INVALID_ARG;
    cudaSetDevice(g->h->device);
    cudaDeviceSynchronize();
    release(g);
    return DBP_OK;
}

}  // extern "C"
