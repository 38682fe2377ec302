// dbp_serve.cu -- request loop of libdbp.so: frames with host buffers are
// admitted as stream slots and device memory free up, run concurrently, and
// share resident channels (device copy of H plus per-cluster operators) per
// coherence block.  Host code only; every frame runs through the same fused
// kernels as the synchronous entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dbp.h"
#include "dbp_internal.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t kAlign = 256;
constexpr double kBypassLimitUs = 20000.0;   // head-of-line frame may be passed for 20 ms

size_t align_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over one device allocation (offsets, coalescing frees).
class Arena {
  public:
    bool init(size_t bytes) {
        if (cudaMalloc(&base_, bytes) != cudaSuccess) {
            base_ = nullptr;
            return false;
        }
        size_ = bytes;
        free_.clear();
        free_[0] = bytes;
        return true;
    }
    void destroy() {
        if (base_) cudaFree(base_);
        base_ = nullptr;
        free_.clear();
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = align_up(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align_up(bytes ? bytes : 1);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    char *at(size_t off) const { return base_ + off; }
    size_t size() const { return size_; }

  private:
    char *base_ = nullptr;
    size_t size_ = 0;
    std::map<size_t, size_t> free_;
};

struct Factor {
    int kind;
    double rho;
    size_t off = 0, bytes = 0;
    bool valid = false;      // stored by a completed frame
    bool pending = false;    // a frame in flight is storing it
};

struct Resident {
    uint64_t key = 0, epoch = 0;
    int B = 0, U = 0, W = 0, C = 0, prec = 0;
    size_t h_off = 0, h_bytes = 0;
    cudaEvent_t uploaded = nullptr;   // H copy complete
    bool upload_recorded = false;
    int users = 0;                    // frames in flight using it
    uint64_t last_use = 0;
    std::vector<Factor> factors;
};

struct Job {
    uint64_t ticket = 0;
    dbp_request req{};
    int phase = 0;                    // 0 queued, 1 running, 2 done
    dbp_status status = DBP_OK;
    std::string err;
    double t_submit = 0, t_start = 0, t_finish = 0;
    int slot = -1;
    size_t off_in = 0, b_in = 0, off_out = 0, b_out = 0, off_lab = 0, b_lab = 0, off_beta = 0, b_beta = 0;
    size_t off_h = 0, b_h = 0;
    bool owns_h = false;
    Resident *res = nullptr;
    int factor_index = -1;
    bool storing_factor = false;
    bool hit = false;
    cudaEvent_t done = nullptr;
};

}  // namespace

struct dbp_server {
    dbp_context *h = nullptr;
    int nslots = 4;
    std::vector<cudaStream_t> streams;
    std::vector<int> slot_busy;
    std::vector<size_t> slot_energy;  // arena offsets of per-slot accumulators
    Arena arena;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> pending;
    std::vector<Job *> running;
    std::unordered_map<uint64_t, std::unique_ptr<Job>> jobs;
    std::map<uint64_t, std::unique_ptr<Resident>> resident;   // by channel key
    std::thread thr;
    bool stopping = false;
    uint64_t next_ticket = 1, use_clock = 0;
    Clock::time_point origin;

    double now_us() const {
        return std::chrono::duration<double, std::micro>(Clock::now() - origin).count();
    }

    static bool on_device(const Job &j) { return (j.req.flags & DBP_REQ_DEVICE_BUFFERS) != 0; }
    size_t in_bytes(const Job &j) const {
        const dbp_frame_desc &d = j.req.desc;
        const size_t e = dbp_in_elem_bytes(d.precision);
        return (j.req.kind == DBP_KIND_DOWNLINK_ADMM) ? (size_t)d.W * d.N * d.U * e : (size_t)d.W * d.N * d.B * e;
    }
    size_t out_size(const Job &j) const {
        const dbp_frame_desc &d = j.req.desc;
        const size_t e = dbp_out_elem_bytes(d.precision);
        return (j.req.kind == DBP_KIND_DOWNLINK_ADMM) ? (size_t)d.W * d.N * d.B * e : (size_t)d.W * d.N * d.U * e;
    }
    size_t h_size(const dbp_frame_desc &d) const {
        return (size_t)d.W * d.B * d.U * dbp_in_elem_bytes(d.precision);
    }
    size_t factor_size(const dbp_frame_desc &d) const {
        const size_t ut = (size_t)dbp_padded_users(d.U);
        return (size_t)d.W * d.C * ut * ut * sizeof(float2);
    }

    // Free resident channels nobody is using, least recently used first,
    // until `need` bytes could fit (best effort).
    void evict_for(size_t need) {
        std::vector<Resident *> cand;
        for (auto &kv : resident)
            if (kv.second->users == 0) cand.push_back(kv.second.get());
        std::sort(cand.begin(), cand.end(), [](Resident *a, Resident *b) { return a->last_use < b->last_use; });
        for (Resident *r : cand) {
            size_t probe;
            if (arena.alloc(need, &probe)) {
                arena.release(probe, need);
                return;
            }
            drop_resident(r);
        }
    }
    void drop_resident(Resident *r) {
        if (r->h_bytes) arena.release(r->h_off, r->h_bytes);
        for (Factor &f : r->factors)
            if (f.bytes) arena.release(f.off, f.bytes);
        if (r->uploaded) cudaEventDestroy(r->uploaded);
        resident.erase(r->key);
    }

    bool admit(Job *j);
    void launch(Job *j);
    void reap();
    void loop();
};

// Allocate device memory and a slot for a queued frame; false if it does not
// fit yet (nothing is held then).
bool dbp_server::admit(Job *j) {
    int slot = -1;
    for (int i = 0; i < nslots; ++i)
        if (!slot_busy[i]) {
            slot = i;
            break;
        }
    if (slot < 0) return false;
    const dbp_request &r = j->req;
    const dbp_frame_desc &d = r.desc;
    const bool dev = on_device(*j);   // caller's device buffers: nothing staged
    j->b_in = dev ? 0 : in_bytes(*j);
    j->b_out = dev ? 0 : out_size(*j);
    j->b_lab = (!dev && r.kind != DBP_KIND_DOWNLINK_ADMM && r.labels && d.qam_order > 0) ? (size_t)d.W * d.N * d.U : 0;
    j->b_beta = (!dev && r.kind == DBP_KIND_DOWNLINK_ADMM && r.beta_out && (d.flags & DBP_FLAG_NORMALIZE)) ? 8 : 0;

    // Resident channel of this coherence block.
    Resident *res = nullptr;
    bool new_res = false;
    if (r.channel_key != 0) {
        auto it = resident.find(r.channel_key);
        if (it != resident.end()) {
            Resident *e = it->second.get();
            const bool same = e->epoch == r.coherence_epoch && e->B == d.B && e->U == d.U && e->W == d.W &&
                              e->C == d.C && e->prec == d.precision;
            if (same) {
                res = e;
                res->users++;        // pinned: eviction below cannot drop it
            } else if (e->users == 0) {
                drop_resident(e);
            } else {
                return false;        // the old block is still in use: wait
            }
        }
        if (!res) new_res = true;
    }
    std::vector<std::pair<size_t, size_t>> taken;
    auto take = [&](size_t bytes, size_t *off) -> bool {
        if (bytes == 0) return true;
        if (!arena.alloc(bytes, off)) {
            evict_for(bytes);
            if (!arena.alloc(bytes, off)) return false;
        }
        taken.push_back({*off, bytes});
        return true;
    };
    auto undo = [&]() {
        for (auto &t : taken) arena.release(t.first, t.second);
        if (res) res->users--;
    };
    const size_t hb = dev ? 0 : h_size(d);
    if (!res && hb) {
        if (!take(hb, &j->off_h)) { undo(); return false; }
        j->b_h = hb;
    }
    if (!take(j->b_in, &j->off_in) || !take(j->b_out, &j->off_out) || !take(j->b_lab, &j->off_lab) ||
        !take(j->b_beta, &j->off_beta)) {
        undo();
        return false;
    }
    if (new_res) {
        auto e = std::make_unique<Resident>();
        e->key = r.channel_key;
        e->epoch = r.coherence_epoch;
        e->B = d.B; e->U = d.U; e->W = d.W; e->C = d.C; e->prec = d.precision;
        e->h_off = j->off_h;
        e->h_bytes = hb;                 // 0 for device buffers: no resident copy
        cudaEventCreateWithFlags(&e->uploaded, cudaEventDisableTiming);
        res = e.get();
        resident[r.channel_key] = std::move(e);
        j->owns_h = false;           // the resident entry owns it now
    } else if (!res) {
        j->owns_h = hb != 0;
    }
    if (res) {
        j->res = res;
        j->hit = !new_res;
        j->off_h = res->h_off;
        if (new_res) res->users++;   // a hit was pinned above
        res->last_use = ++use_clock;
        // resident operator for this kind and rho
        const double rho = (r.kind == DBP_KIND_UPLINK_CG) ? 0.0 : d.rho;
        int fi = -1;
        for (size_t k = 0; k < res->factors.size(); ++k)
            if (res->factors[k].kind == r.kind && res->factors[k].rho == rho) fi = (int)k;
        if (fi < 0) {
            Factor f;
            f.kind = r.kind;
            f.rho = rho;
            f.bytes = factor_size(d);
            if (arena.alloc(f.bytes, &f.off)) {
                res->factors.push_back(f);
                fi = (int)res->factors.size() - 1;
            }
        }
        j->factor_index = fi;
    }
    j->slot = slot;
    slot_busy[slot] = 1;
    return true;
}

void dbp_server::launch(Job *j) {
    cudaStream_t st = streams[j->slot];
    const dbp_request &r = j->req;
    const dbp_frame_desc &d = r.desc;
    cudaError_t e = cudaSuccess;
    const bool dev = on_device(*j);
    char *dH = dev ? const_cast<char *>(static_cast<const char *>(r.H)) : arena.at(j->off_h);
    if (dev) {
        // the caller's device buffers are used in place
    } else if (j->res && j->hit) {
        if (j->res->upload_recorded) e = cudaStreamWaitEvent(st, j->res->uploaded, 0);
    } else {
        e = cudaMemcpyAsync(dH, r.H, h_size(d), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && j->res) {
            e = cudaEventRecord(j->res->uploaded, st);
            j->res->upload_recorded = true;
        }
    }
    if (e == cudaSuccess && !dev)
        e = cudaMemcpyAsync(arena.at(j->off_in), r.in, j->b_in, cudaMemcpyHostToDevice, st);
    void *d_in = dev ? const_cast<void *>(r.in) : arena.at(j->off_in);
    void *d_out = dev ? r.out : arena.at(j->off_out);
    uint8_t *d_lab = dev ? ((r.kind != DBP_KIND_DOWNLINK_ADMM && d.qam_order > 0) ? r.labels : nullptr)
                         : (j->b_lab ? reinterpret_cast<uint8_t *>(arena.at(j->off_lab)) : nullptr);
    double *d_beta = dev ? r.beta_out : (j->b_beta ? reinterpret_cast<double *>(arena.at(j->off_beta)) : nullptr);
    DbpExec ex;
    ex.energy = reinterpret_cast<double *>(arena.at(slot_energy[j->slot]));
    Factor *f = (j->res && j->factor_index >= 0) ? &j->res->factors[j->factor_index] : nullptr;
    if (f) {
        ex.factor = reinterpret_cast<float2 *>(arena.at(f->off));
        if (f->valid) ex.factor_mode = 2;
        else if (!f->pending) {
            ex.factor_mode = 1;
            f->pending = true;
            j->storing_factor = true;
        }
    }
    dbp_status stt = DBP_OK;
    if (e == cudaSuccess) {
        bool used = false;
        stt = dbp_run_internal(h, &d, r.kind, dH, d_in, d_out, d_lab, d_beta, st, &ex, &used, &j->err);
        if (j->storing_factor && !used) {   // the kernel that ran cannot store it
            f->pending = false;
            j->storing_factor = false;
        }
    }
    if (e == cudaSuccess && stt == DBP_OK && !dev) {
        e = cudaMemcpyAsync(r.out, arena.at(j->off_out), j->b_out, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && j->b_lab)
            e = cudaMemcpyAsync(r.labels, arena.at(j->off_lab), j->b_lab, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && j->b_beta)
            e = cudaMemcpyAsync(r.beta_out, arena.at(j->off_beta), 8, cudaMemcpyDeviceToHost, st);
    }
    if (e != cudaSuccess) {
        stt = DBP_ERR_CUDA;
        j->err = cudaGetErrorString(e);
    }
    j->status = stt;
    cudaEventCreateWithFlags(&j->done, cudaEventDisableTiming);
    cudaEventRecord(j->done, st);
    j->t_start = now_us();
    j->phase = 1;
    running.push_back(j);
}

void dbp_server::reap() {
    for (size_t i = 0; i < running.size();) {
        Job *j = running[i];
        const cudaError_t q = cudaEventQuery(j->done);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        if (q != cudaSuccess && j->status == DBP_OK) {
            j->status = DBP_ERR_CUDA;
            j->err = cudaGetErrorString(q);
        }
        j->t_finish = now_us();
        cudaEventDestroy(j->done);
        j->done = nullptr;
        if (j->b_in) arena.release(j->off_in, j->b_in);
        if (j->b_out) arena.release(j->off_out, j->b_out);
        if (j->b_lab) arena.release(j->off_lab, j->b_lab);
        if (j->b_beta) arena.release(j->off_beta, j->b_beta);
        if (j->owns_h) arena.release(j->off_h, j->b_h);
        if (j->res) {
            j->res->users--;
            if (j->storing_factor && j->factor_index >= 0) {
                Factor &f = j->res->factors[j->factor_index];
                f.pending = false;
                f.valid = (j->status == DBP_OK);
            }
        }
        slot_busy[j->slot] = 0;
        j->phase = 2;
        running[i] = running.back();
        running.pop_back();
        cv_done.notify_all();
    }
}

void dbp_server::loop() {
    cudaSetDevice(h->device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        reap();
        bool progressed = false;
        if (!stopping) {
            for (auto it = pending.begin(); it != pending.end();) {
                Job *j = *it;
                if (admit(j)) {
                    it = pending.erase(it);
                    launch(j);
                    progressed = true;
                    continue;
                }
                // a frame that has waited too long blocks the ones behind it
                if (now_us() - j->t_submit > kBypassLimitUs) break;
                ++it;
            }
        }
        if (stopping && running.empty()) break;
        if (!progressed) cv_work.wait_for(lk, std::chrono::microseconds(running.empty() ? 2000 : 20));
    }
}

void dbp_server_destroy(dbp_server *s) {
    if (!s) return;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->stopping = true;
        for (Job *j : s->pending) {
            j->status = DBP_ERR_TIMEOUT;
            j->err = "request loop stopped before the frame was admitted";
            j->phase = 2;
            j->t_finish = s->now_us();
        }
        s->pending.clear();
    }
    s->cv_work.notify_all();
    // In-flight frames finish on their own; wait for the loop (bounded).
    const auto deadline = Clock::now() + std::chrono::seconds(30);
    while (Clock::now() < deadline) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->running.empty()) break;
        }
        std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
    if (s->thr.joinable()) s->thr.join();
    cudaSetDevice(s->h->device);
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto &kv : s->resident)
        if (kv.second->uploaded) cudaEventDestroy(kv.second->uploaded);
    s->resident.clear();
    s->arena.destroy();
    delete s;
}

extern "C" {

dbp_status dbp_server_start(dbp_handle_t h, const dbp_server_config *cfg) {
    if (!h) return DBP_ERR_INVALID_ARG;
    if (h->server) return DBP_ERR_INVALID_ARG;
    auto *s = new (std::nothrow) dbp_server();
    if (!s) return DBP_ERR_NOMEM;
    s->h = h;
    s->nslots = (cfg && cfg->streams > 0) ? cfg->streams : 4;
    if (s->nslots > 64) s->nslots = 64;
    size_t bytes = (cfg && cfg->hbm_bytes) ? cfg->hbm_bytes : ((size_t)2 << 30);
    if (h->budget) {
        const size_t left = h->budget > h->used ? (size_t)(h->budget - h->used) : 0;
        if (!(cfg && cfg->hbm_bytes) && bytes > left) bytes = left;   // default pool: what the budget leaves
        if (bytes > left || bytes < 4096) {
            h->err = "dbp_server_start: the pool does not fit the handle's HBM budget";
            delete s;
            return DBP_ERR_NOMEM;
        }
    }
    if (cudaSetDevice(h->device) != cudaSuccess) {
        delete s;
        return DBP_ERR_CUDA;
    }
    if (!s->arena.init(bytes)) {
        delete s;
        return DBP_ERR_NOMEM;
    }
    h->used += bytes;
    s->streams.resize(s->nslots);
    s->slot_busy.assign(s->nslots, 0);
    s->slot_energy.resize(s->nslots);
    for (int i = 0; i < s->nslots; ++i) {
        if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            !s->arena.alloc(sizeof(double), &s->slot_energy[i])) {
            for (int k = 0; k < i; ++k) cudaStreamDestroy(s->streams[k]);
            s->arena.destroy();
            delete s;
            return DBP_ERR_CUDA;
        }
    }
    s->origin = Clock::now();
    h->server = s;
    s->thr = std::thread([s] { s->loop(); });
    return DBP_OK;
}

dbp_status dbp_server_stop(dbp_handle_t h) {
    if (!h || !h->server) return DBP_ERR_INVALID_ARG;
    const size_t pool = h->server->arena.size();
    h->used = h->used > pool ? h->used - pool : 0;
    dbp_server_destroy(h->server);
    h->server = nullptr;
    return DBP_OK;
}

dbp_status dbp_submit(dbp_handle_t h, const dbp_request *req, uint64_t *ticket) {
    if (!h || !h->server || !req || !ticket) return DBP_ERR_INVALID_ARG;
    if (req->kind < DBP_KIND_UPLINK_ADMM || req->kind > DBP_KIND_DOWNLINK_ADMM) return DBP_ERR_INVALID_ARG;
    dbp_server *s = h->server;
    std::string err;
    dbp_status v = dbp_validate_internal(h, &req->desc, req->kind, &err);
    if (v != DBP_OK) {
        std::lock_guard<std::mutex> lk(s->mu);
        h->err = err;
        return v;
    }
    const dbp_frame_desc &d = req->desc;
    if ((long long)d.W * d.N > 0 && (!req->H || !req->in || !req->out)) return DBP_ERR_INVALID_ARG;
    if (req->flags & ~DBP_REQ_DEVICE_BUFFERS) {
        std::lock_guard<std::mutex> lk(s->mu);
        h->err = "dbp_submit: unknown request flags";
        return DBP_ERR_INVALID_ARG;
    }
    auto j = std::make_unique<Job>();
    j->req = *req;
    if (!(req->flags & DBP_REQ_DEVICE_BUFFERS)) {
        // the staged inputs and outputs must fit the pool at all (besides the
        // slots' accumulators), or the frame could never be admitted
        const bool lab = req->kind != DBP_KIND_DOWNLINK_ADMM && req->labels && d.qam_order > 0;
        const size_t need = align_up(s->h_size(d)) + align_up(s->in_bytes(*j)) + align_up(s->out_size(*j)) +
                            (lab ? align_up((size_t)d.W * d.N * d.U) : 0) + align_up(8);
        const size_t avail = s->arena.size() - (size_t)s->nslots * kAlign;
        if (need > avail) {
            std::lock_guard<std::mutex> lk(s->mu);
            h->err = "dbp_submit: the frame needs " + std::to_string(need) + " bytes of the request pool, which has " +
                     std::to_string(avail);
            return DBP_ERR_NOMEM;
        }
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) return DBP_ERR_INVALID_ARG;
        j->ticket = s->next_ticket++;
        j->t_submit = s->now_us();
        *ticket = j->ticket;
        s->pending.push_back(j.get());
        s->jobs[j->ticket] = std::move(j);
    }
    s->cv_work.notify_one();
    return DBP_OK;
}

dbp_status dbp_cancel(dbp_handle_t h, uint64_t ticket) {
    if (!h || !h->server) return DBP_ERR_INVALID_ARG;
    dbp_server *s = h->server;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end() || it->second->phase == 2) return DBP_ERR_INVALID_ARG;
    Job *j = it->second.get();
    if (j->phase != 0) return DBP_PENDING;       // admitted: runs to completion
    for (auto p = s->pending.begin(); p != s->pending.end(); ++p)
        if (*p == j) {
            s->pending.erase(p);
            break;
        }
    j->status = DBP_ERR_CANCELLED;
    j->err = "cancelled before admission";
    j->t_finish = s->now_us();
    j->phase = 2;
    s->cv_done.notify_all();
    return DBP_OK;
}

static void fill_result(const Job &j, dbp_result *res) {
    res->status = j.status;
    res->resident_hit = j.hit ? 1 : 0;
    res->user_tag = j.req.user_tag;
    res->submit_us = j.t_submit;
    res->start_us = j.t_start;
    res->finish_us = j.t_finish;
}

dbp_status dbp_poll(dbp_handle_t h, uint64_t ticket, dbp_result *res) {
    if (!h || !h->server || !res) return DBP_ERR_INVALID_ARG;
    dbp_server *s = h->server;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return DBP_ERR_INVALID_ARG;
    if (it->second->phase != 2) return DBP_PENDING;
    fill_result(*it->second, res);
    if (it->second->status != DBP_OK) h->err = it->second->err;
    s->jobs.erase(it);
    return DBP_OK;
}

dbp_status dbp_wait(dbp_handle_t h, uint64_t ticket, double timeout_s, dbp_result *res) {
    if (!h || !h->server || !res) return DBP_ERR_INVALID_ARG;
    dbp_server *s = h->server;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return DBP_ERR_INVALID_ARG;
    Job *j = it->second.get();
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
    while (j->phase != 2) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && j->phase != 2) return DBP_ERR_TIMEOUT;
    }
    fill_result(*j, res);
    if (j->status != DBP_OK) h->err = j->err;
    s->jobs.erase(it);
    return DBP_OK;
}

}  // extern "C"
