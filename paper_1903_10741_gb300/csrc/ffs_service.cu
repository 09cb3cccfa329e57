// ffs_service.cu -- the rescheduling service: continuous batching of rescheduling
// requests on one GPU, admission by device memory, warm populations kept per instance;
// and the arena that gives the service's populations their memory.
//
// One worker thread per service does all device work.  Each admitted request owns a slot
// (a stream and a completion event); its generations are queued on that stream at once,
// so the fused generation kernels of all active requests interleave on the SMs.  The
// worker retires a request when its event has completed (decode and commit of the best
// schedule), which frees the slot for the next queued request.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "ffs_internal.h"

using namespace ffs_rt;

// ====================================================================== arena
// First-fit sub-allocation of one cudaMalloc'd block, with coalescing of free neighbours.
// Blocks are returned by host bookkeeping only: the caller guarantees that no queued
// device work still uses them (the service frees a population only after its stream has
// drained).
struct ffs_rt::Arena {
    char *base = nullptr;
    size_t size = 0, used = 0, peak = 0;
    std::map<size_t, size_t> free_;            // offset -> bytes
    std::unordered_map<size_t, size_t> live_;  // offset -> bytes

    void reset(char *b, size_t n) {
        base = b;
        size = n;
        free_.clear();
        live_.clear();
        free_.emplace(0, n);
        used = peak = 0;
    }
    void *alloc(size_t bytes) {
        bytes = (bytes + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_.emplace(off + bytes, rest);
            live_.emplace(off, bytes);
            used += bytes;
            peak = std::max(peak, used);
            return base + off;
        }
        return nullptr;
    }
    bool owns(const void *p) const {
        const char *c = static_cast<const char *>(p);
        return c >= base && c < base + size;
    }
    void release(void *p) {
        const size_t off = static_cast<size_t>(static_cast<char *>(p) - base);
        auto it = live_.find(off);
        if (it == live_.end()) return;
        size_t start = off, len = it->second;
        used -= it->second;
        live_.erase(it);
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && start + len == nx->first) {
            len += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == start) {
                start = pv->first;
                len += pv->second;
                free_.erase(pv);
            }
        }
        free_.emplace(start, len);
    }
};

namespace {
std::mutex g_arena_mu;
std::vector<ffs_rt::Arena *> g_arenas;
}  // namespace

thread_local ffs_rt::Arena *ffs_rt::t_arena = nullptr;

cudaError_t ffs_rt::raw_alloc(void **p, size_t bytes) {
    if (!t_arena) return cudaMalloc(p, bytes);
    std::lock_guard<std::mutex> lk(g_arena_mu);
    *p = t_arena->alloc(bytes);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}

void ffs_rt::raw_free(void *p) {
    {
        std::lock_guard<std::mutex> lk(g_arena_mu);
        for (Arena *a : g_arenas)
            if (a->owns(p)) {
                a->release(p);
                return;
            }
    }
    cudaFree(p);
}

// ====================================================================== service
namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    int64_t ticket = 0;
    ffs_instance *inst = nullptr;
    bool has_arrivals = false;
    int32_t n_arr = 0, t_now = 0, generations = 0;
    std::vector<int32_t> proc, release, due, proc_machine, power_machine;
    bool prepared = false;          // ffs_reschedule applied, footprint known
    ga_params par{};
    ffs_request_info info{};
    ffs_result res{};
    std::vector<int32_t> S, M;
    std::string err_text;
    bool stop = false;              // ffs_service_stop_request was called (under mu)
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;     // recorded after the chunk of generations in flight
    Request *req = nullptr;
    ga_population *pop = nullptr;
    int run = 0, left = 0;          // generations enqueued so far; still to enqueue
};

// Generations enqueued at a time for an admitted request: the worker enqueues the next
// chunk when one completes, so a stop request takes effect within a chunk.  A multiple of
// the 8-generation graphs, so the launches are those of one ga_run.
constexpr int kChunk = 64;

bool stop_requested(ffs_service *s, const Request *r);

struct InstState {
    ga_population *warm = nullptr;  // last population, kept on the device (worker only)
    int32_t solves = 0;             // requests admitted so far (worker only)
    bool active = false;            // a request of the instance is on the device (worker only)
    uint64_t last_use = 0;          // worker only
    int pending = 0;                // queued or active requests (under mu)
};

enum AdmitResult { kAdmitted, kFinished, kWaitMemory };

}  // namespace

struct ffs_service {
    ffs_service_config cfg{};
    int device = 0;
    Arena arena;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;                        // submitted, not admitted (under mu)
    std::map<int64_t, std::unique_ptr<Request>> reqs;   // every request (under mu)
    std::unordered_map<ffs_instance *, InstState> insts;  // structure under mu; fields as marked
    std::atomic<int> kept{0};                           // kept populations
    std::vector<ffs_instance *> forget;                 // kept populations to drop (under mu)
    int64_t next_ticket = 1, completed = 0, failed = 0;
    int active = 0;                                     // under mu
    bool stop = false;                                  // under mu
    uint64_t tick = 0;
    std::thread worker;
};

namespace {

bool stop_requested(ffs_service *s, const Request *r) {
    std::lock_guard<std::mutex> lk(s->mu);
    return r->stop;
}

// Records the end of a request (under the lock) and wakes waiters.
void finish_request(ffs_service *s, Request *r, int rc, bool was_active) {
    if (rc != FFS_OK) r->err_text = ffs_last_error();
    std::lock_guard<std::mutex> lk(s->mu);
    r->info.state = rc == FFS_OK ? FFS_REQ_DONE : FFS_REQ_FAILED;
    r->info.status = rc;
    r->info.done_ns = now_ns();
    s->insts[r->inst].pending--;
    if (was_active) s->active--;
    if (rc == FFS_OK) s->completed++;
    else s->failed++;
    s->cv_done.notify_all();
}

// The instance's entry (created at submission).  Entries are inserted and erased under the
// lock; the returned pointer stays valid until the worker itself erases the entry.
InstState *inst_state(ffs_service *s, ffs_instance *in) {
    std::lock_guard<std::mutex> lk(s->mu);
    return &s->insts[in];
}

void set_warm(ffs_service *s, InstState *is, ga_population *pop) {
    if (is->warm) {
        ga_population_destroy(is->warm);
        s->kept--;
    }
    is->warm = pop;
    if (pop) s->kept++;
}

size_t arena_free(ffs_service *s) {
    std::lock_guard<std::mutex> lk(g_arena_mu);
    return s->arena.size - s->arena.used;
}

// Drops the least recently used kept population other than `keep`'s; instances with no
// request waiting go first.  False if there is none.
bool evict_one(ffs_service *s, ffs_instance *keep) {
    InstState *victim = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        std::pair<int, uint64_t> vkey{0, 0};
        for (auto &kv : s->insts) {
            if (!kv.second.warm || kv.first == keep) continue;
            const std::pair<int, uint64_t> key{kv.second.pending > 0 ? 1 : 0, kv.second.last_use};
            if (!victim || key < vkey) {
                victim = &kv.second;
                vkey = key;
            }
        }
    }
    if (!victim) return false;
    set_warm(s, victim, nullptr);
    return true;
}

AdmitResult admit(ffs_service *s, Slot &slot, Request *r) {
    InstState &is = *inst_state(s, r->inst);
    if (!r->prepared) {
        ffs_arrivals a{r->n_arr, r->proc.data(), r->release.data(), r->due.data(),
                       r->proc_machine.empty() ? nullptr : r->proc_machine.data(),
                       r->power_machine.empty() ? nullptr : r->power_machine.data()};
        int rc = ffs_reschedule(r->inst, r->has_arrivals ? &a : nullptr, r->t_now);
        if (rc == FFS_OK) rc = sync_device(r->inst);
        r->par = s->cfg.ga;
        r->par.instance_id = (int32_t)((uint32_t)s->cfg.ga.instance_id + (uint32_t)is.solves);
        int64_t fp = 0;
        if (rc == FFS_OK) rc = population_footprint(r->inst, &r->par, &fp);
        if (rc != FFS_OK) {
            finish_request(s, r, rc, false);
            return kFinished;
        }
        r->prepared = true;
        r->info.footprint = fp;
        r->info.n_ops = r->inst->N * r->inst->g;
    }
    r->par.cuda_stream = slot.st;
    // the warm start also holds the gene map for a moment
    const size_t prevK = is.warm ? (size_t)is.warm->K : 0;
    const size_t transient = ((prevK + r->inst->K) * 4 + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
    const size_t need = (size_t)r->info.footprint + transient;
    if (need > s->arena.size) {
        std::snprintf(g_last_error, sizeof(g_last_error), "population needs %zu bytes, the service holds %zu",
                      need, s->arena.size);
        finish_request(s, r, FFS_E_ADMISSION, false);
        return kFinished;
    }
    bool others_active;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        others_active = s->active > 0;
    }
    ga_population *pop = nullptr;
    for (;;) {
        while (arena_free(s) < need && evict_one(s, r->inst)) {
        }
        if (arena_free(s) < need) {
            if (others_active) return kWaitMemory;
            if (!is.warm) break;  // cannot happen: nothing else holds memory
            set_warm(s, &is, nullptr);  // last resort: start cold
            continue;
        }
        t_arena = &s->arena;
        const int rc = population_create(r->inst, &r->par, is.warm, &pop);
        t_arena = nullptr;
        if (rc == FFS_OK) break;
        if (rc == FFS_E_NOMEM) {  // fragmented: free more, or wait for the active requests
            if (evict_one(s, r->inst)) continue;
            if (others_active) return kWaitMemory;
            if (is.warm) {
                set_warm(s, &is, nullptr);
                continue;
            }
        }
        finish_request(s, r, rc, false);
        return kFinished;
    }
    if (!pop) {
        finish_request(s, r, FFS_E_ADMISSION, false);
        return kFinished;
    }
    r->info.warm = is.warm ? 1 : 0;
    set_warm(s, &is, nullptr);  // its rows were read before create returned
    is.solves++;
    is.active = true;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
        r->info.state = FFS_REQ_ACTIVE;
        r->info.admit_ns = now_ns();
        s->active++;
    }
    // a request stopped while it waited runs no generation past generation 0
    const int first = stop_requested(s, r) ? 0 : std::min(r->generations, kChunk);
    int rc = ga_enqueue(pop, first);
    if (rc == FFS_OK) rc = cuda_rc(cudaEventRecord(slot.done, slot.st));
    if (rc != FFS_OK) {
        cudaStreamSynchronize(slot.st);
        ga_population_destroy(pop);
        is.active = false;
        finish_request(s, r, rc, true);
        return kFinished;
    }
    slot.req = r;
    slot.pop = pop;
    slot.run = first;
    slot.left = stop_requested(s, r) ? 0 : r->generations - first;
    return kAdmitted;
}

void retire(ffs_service *s, Slot &slot, int rc) {
    Request *r = slot.req;
    ga_population *pop = slot.pop;
    r->info.generations = slot.run;
    slot.req = nullptr;
    slot.pop = nullptr;
    if (rc == FFS_OK) {
        r->S.assign((size_t)pop->NG, 0);
        r->M.assign((size_t)pop->NG, 0);
        r->res = ffs_result{};
        r->res.start = r->S.data();
        r->res.machine = r->M.data();
        rc = ga_finish(pop, &r->res);
    }
    InstState &is = *inst_state(s, r->inst);
    is.active = false;
    is.last_use = ++s->tick;
    if (rc == FFS_OK) {
        population_trim(pop);  // kept only as the next request's warm-start source
        set_warm(s, &is, pop);
    } else {
        ga_population_destroy(pop);
    }
    finish_request(s, r, rc, true);
}

void worker_main(ffs_service *s) {
    cudaSetDevice(s->device);
    for (;;) {
        bool progress = false;
        // kept populations the caller released
        std::vector<ffs_instance *> drop;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            drop.swap(s->forget);
        }
        for (ffs_instance *in : drop) {
            InstState *is = nullptr;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                auto it = s->insts.find(in);
                if (it == s->insts.end() || it->second.pending > 0) continue;
                is = &it->second;
            }
            set_warm(s, is, nullptr);
            std::lock_guard<std::mutex> lk(s->mu);
            auto it = s->insts.find(in);
            if (it != s->insts.end() && it->second.pending == 0) s->insts.erase(it);
        }
        // next chunks, or retire
        for (Slot &sl : s->slots) {
            if (!sl.req) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            int rc = q == cudaSuccess ? FFS_OK : cuda_rc(q);
            if (rc == FFS_OK && sl.left > 0 && !stop_requested(s, sl.req)) {
                const int n = std::min(sl.left, kChunk);
                rc = ga_enqueue(sl.pop, n);
                if (rc == FFS_OK) rc = cuda_rc(cudaEventRecord(sl.done, sl.st));
                if (rc == FFS_OK) {
                    sl.left -= n;
                    sl.run += n;
                    progress = true;
                    continue;
                }
                cudaStreamSynchronize(sl.st);
            }
            retire(s, sl, rc);
            progress = true;
        }
        // queued requests stopped before their rescheduling was applied end unchanged
        {
            std::vector<Request *> gone;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                for (auto it = s->queue.begin(); it != s->queue.end();) {
                    if ((*it)->stop && !(*it)->prepared) {
                        gone.push_back(*it);
                        it = s->queue.erase(it);
                    } else {
                        ++it;
                    }
                }
            }
            for (Request *r : gone) {
                std::snprintf(g_last_error, sizeof(g_last_error), "request stopped before it was admitted");
                finish_request(s, r, FFS_E_STOPPED, false);
                progress = true;
            }
        }
        // admit, first come first served
        std::vector<Request *> cand;
        bool stopping;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            stopping = s->stop;
            if (!stopping) cand.assign(s->queue.begin(), s->queue.end());
        }
        if (stopping) {
            std::vector<Request *> cancel;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                cancel.assign(s->queue.begin(), s->queue.end());
                s->queue.clear();
            }
            for (Request *r : cancel) finish_request(s, r, FFS_E_STATE, false);
            bool any = false;
            for (Slot &sl : s->slots) any = any || sl.req;
            if (!any) return;
        }
        std::unordered_set<ffs_instance *> seen;
        for (Request *r : cand) {
            Slot *free_slot = nullptr;
            for (Slot &sl : s->slots)
                if (!sl.req) {
                    free_slot = &sl;
                    break;
                }
            if (!free_slot) break;
            const bool first_of_instance = seen.insert(r->inst).second;
            if (!first_of_instance || inst_state(s, r->inst)->active) continue;
            const AdmitResult ar = admit(s, *free_slot, r);
            if (ar == kWaitMemory) break;
            progress = true;
        }
        if (progress) continue;
        bool any_active = false;
        for (Slot &sl : s->slots) any_active = any_active || sl.req;
        if (any_active) {
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        } else {
            std::unique_lock<std::mutex> lk(s->mu);
            const size_t n = s->queue.size();
            s->cv_work.wait_for(lk, std::chrono::milliseconds(50),
                                [&] { return s->stop || s->queue.size() != n || !s->forget.empty(); });
        }
    }
}

}  // namespace

extern "C" {

int ffs_service_create(const ffs_service_config *cfg, ffs_service **out) {
    if (!cfg || !out) return FFS_E_ARG;
    *out = nullptr;
    if (cfg->max_active < 1 || cfg->max_active > 1024 || cfg->memory_bytes <= 0) return FFS_E_ARG;
    {
        ga_params probe = cfg->ga;
        FFS_TRY(check_modes(probe.order_mode, probe.machine_mode));
        const int P = probe.pop, I = probe.island;
        if (P < 2 || P % 2 || I < 2 || I % 2 || P % I) return FFS_E_ARG;
    }
    std::unique_ptr<ffs_service> s(new (std::nothrow) ffs_service());
    if (!s) return FFS_E_NOMEM;
    s->cfg = *cfg;
    FFS_CUDA(cudaGetDevice(&s->device));
    void *base = nullptr;
    if (cudaMalloc(&base, (size_t)cfg->memory_bytes) != cudaSuccess) {
        cudaGetLastError();
        return FFS_E_NOMEM;
    }
    s->arena.reset(static_cast<char *>(base), (size_t)cfg->memory_bytes);
    s->slots.resize(cfg->max_active);
    int rc = FFS_OK;
    for (Slot &sl : s->slots) {
        if (rc == FFS_OK) rc = cuda_rc(cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking));
        if (rc == FFS_OK) rc = cuda_rc(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
    }
    if (rc != FFS_OK) {
        for (Slot &sl : s->slots) {
            if (sl.st) cudaStreamDestroy(sl.st);
            if (sl.done) cudaEventDestroy(sl.done);
        }
        cudaFree(base);
        return rc;
    }
    {
        std::lock_guard<std::mutex> lk(g_arena_mu);
        g_arenas.push_back(&s->arena);
    }
    ffs_service *raw = s.get();
    s->worker = std::thread(worker_main, raw);
    *out = s.release();
    return FFS_OK;
}

int ffs_service_destroy(ffs_service *s) {
    if (!s) return FFS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &kv : s->insts) ga_population_destroy(kv.second.warm);
    s->insts.clear();
    for (Slot &sl : s->slots) {
        if (sl.pop) {
            cudaStreamSynchronize(sl.st);
            ga_population_destroy(sl.pop);
        }
        cudaStreamDestroy(sl.st);
        cudaEventDestroy(sl.done);
    }
    {
        std::lock_guard<std::mutex> lk(g_arena_mu);
        g_arenas.erase(std::find(g_arenas.begin(), g_arenas.end(), &s->arena));
    }
    cudaFree(s->arena.base);
    delete s;
    return FFS_OK;
}

int ffs_service_submit(ffs_service *s, ffs_instance *inst, const ffs_arrivals *arr, int32_t t_now,
                       int32_t generations, int64_t *ticket) {
    if (!s || !inst || !ticket || generations < 0) return FFS_E_ARG;
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return FFS_E_NOMEM;
    r->inst = inst;
    r->t_now = t_now;
    r->generations = generations;
    if (arr) {
        const int n = arr->job_count;
        if (n < 0 || (n > 0 && (!arr->release || !arr->due))) return FFS_E_ARG;
        if (n > 0 && (inst->unrel ? (!arr->proc_machine || !arr->power_machine) : !arr->proc)) return FFS_E_ARG;
        r->has_arrivals = true;
        r->n_arr = n;
        if (arr->proc) r->proc.assign(arr->proc, arr->proc + (size_t)n * inst->g);
        if (inst->unrel && n > 0) {
            r->proc_machine.assign(arr->proc_machine, arr->proc_machine + (size_t)n * inst->M);
            r->power_machine.assign(arr->power_machine, arr->power_machine + (size_t)n * inst->M);
        }
        r->release.assign(arr->release, arr->release + n);
        r->due.assign(arr->due, arr->due + n);
    }
    r->info.state = FFS_REQ_QUEUED;
    r->info.generations = generations;
    r->info.submit_ns = now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return FFS_E_STATE;
        r->ticket = s->next_ticket++;
        *ticket = r->ticket;
        s->insts[inst].pending++;
        s->queue.push_back(r.get());
        s->reqs.emplace(r->ticket, std::move(r));
    }
    s->cv_work.notify_all();
    return FFS_OK;
}

int ffs_service_wait(ffs_service *s, int64_t ticket, int32_t timeout_ms, ffs_request_info *info,
                     ffs_result *best) {
    if (!s) return FFS_E_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return FFS_E_ARG;
    Request *r = it->second.get();
    auto finished = [&] { return r->info.state >= FFS_REQ_DONE; };
    if (!finished()) {
        if (timeout_ms < 0) s->cv_done.wait(lk, finished);
        else if (timeout_ms > 0) s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished);
    }
    if (info) *info = r->info;
    if (!finished()) return FFS_E_TIMEOUT;
    if (r->info.state == FFS_REQ_FAILED) {
        std::snprintf(g_last_error, sizeof(g_last_error), "%s", r->err_text.c_str());
        return r->info.status;
    }
    if (best) {
        best->objective = r->res.objective;
        best->total_tardiness = r->res.total_tardiness;
        best->makespan = r->res.makespan;
        best->n_ops = r->res.n_ops;
        if (best->start) std::memcpy(best->start, r->S.data(), 4 * r->S.size());
        if (best->machine) std::memcpy(best->machine, r->M.data(), 4 * r->M.size());
    }
    return FFS_OK;
}

int ffs_service_stop_request(ffs_service *s, int64_t ticket) {
    if (!s) return FFS_E_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return FFS_E_ARG;
        it->second->stop = true;
    }
    s->cv_work.notify_all();
    return FFS_OK;
}

int ffs_service_forget(ffs_service *s, ffs_instance *inst) {
    if (!s || !inst) return FFS_E_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->insts.find(inst);
        if (it == s->insts.end()) return FFS_OK;
        if (it->second.pending > 0) return FFS_E_STATE;
        s->forget.push_back(inst);
    }
    s->cv_work.notify_all();
    return FFS_OK;
}

int ffs_service_stats_read(ffs_service *s, ffs_service_stats *st) {
    if (!s || !st) return FFS_E_ARG;
    *st = ffs_service_stats{};
    {
        std::lock_guard<std::mutex> lk(s->mu);
        st->active = s->active;
        st->queued = (int32_t)s->queue.size();
        st->completed = s->completed;
        st->failed = s->failed;
    }
    st->warm = s->kept.load();
    {
        std::lock_guard<std::mutex> lk(g_arena_mu);
        st->memory_bytes = (int64_t)s->arena.size;
        st->used_bytes = (int64_t)s->arena.used;
        st->peak_bytes = (int64_t)s->arena.peak;
    }
    return FFS_OK;
}

}  // extern "C"
