// psort_server.cu -- ps_server_*: a request loop that sorts device buffers
// submitted from any host thread, with continuous batching under a device-
// memory budget (see include/psort.h).
//
// One worker thread owns the device work.  Submitted requests wait in a FIFO
// queue; whenever a stream slot is free and the in-flight limit and the memory
// budget allow, the worker admits the queue's head requests as one round,
// sorts each (dtype, pivot mode) group of the round with the batched pipeline
// in place (every request a segment read from and written back to its own
// buffer; a scratch buffer of the group's size carries the passes in
// between), and queues a host callback that retires the round.  Rounds run
// on several streams, so a round admitted while earlier ones are on the GPU
// overlaps with them.  A request's result is bit-identical to ps_sort on it
// alone: batching changes only which launches carry it.
#include <algorithm>
#include <climits>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "psort_internal.h"

namespace ps {

namespace {

constexpr int NSLOT = 3;          // rounds that may be on the GPU at once
constexpr size_t LONG_QUEUE = 16;  // queued requests beyond which rounds are not capped

struct Req {
    uint64_t id;
    void* keys;
    int64_t n;
    int dtype, mode;
    size_t cost;
};

struct Server;

struct Round {
    Server* srv;
    int slot;
    std::vector<Req> reqs;
    size_t cost;
    int status;
    std::atomic<bool> retired{false};
};

struct Slot {
    cudaStream_t stream = nullptr;
    bool busy = false;
    bool dead = false;          // its stream failed: never reused
    Round* cur = nullptr;       // the slot's last round (kept until replaced)
    int64_t* pinned = nullptr;  // page-locked staging of the round's instance tables
    size_t pinned_cap = 0;      // in int64
};

struct Done {
    uint64_t id;
    int status;
};

size_t key_bytes(int dtype) { return (dtype == PS_I32 || dtype == PS_F32 || dtype == PS_U32) ? 4 : 8; }

struct Server {
    int dev = 0;
    size_t budget = 0;
    int max_inflight = 1;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req> pending;
    std::vector<Done> done;
    bool closing = false;
    size_t used = 0;
    int inflight = 0;
    uint64_t next_id = 1;
    Slot slots[NSLOT];
    std::thread worker;
    // host-side failure injection (ps_server_debug_fail): rounds to fail at
    // launch, and idle slots to retire as if their streams had failed
    int fail_rounds = 0;
    int kill_slots = 0;
    // smallest round size in keys (PS_SERVER_ROUND_KEYS in the environment
    // overrides), and the keys waiting in the queue
    int64_t round_keys = int64_t(1) << 23;
    int64_t pending_keys = 0;

    // Retire a round once: from its stream's host callback (no CUDA calls
    // there), or from the worker when the stream reports an error.
    static void retire_with(Round* r, int status)
    {
        if (r->retired.exchange(true)) return;
        Server* s = r->srv;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (const Req& q : r->reqs) s->done.push_back(Done{q.id, status});
            s->used -= r->cost;
            s->inflight -= (int)r->reqs.size();
            s->slots[r->slot].busy = false;
        }
        s->cv.notify_all();
    }
    static void CUDART_CB retire(void* p)
    {
        Round* r = (Round*)p;
        retire_with(r, r->status);
    }

    // Queue one round on its slot's stream: gather, batched sort, scatter.
    int launch(Round* r)
    {
        Slot& sl = slots[r->slot];
        cudaStream_t st = sl.stream;
        int rc = PS_OK;
        bool inject = false;
        {
            std::lock_guard<std::mutex> lk(mu);
            if (fail_rounds > 0) {
                fail_rounds--;
                inject = true;
            }
        }
        // one pinned table for the whole round (3 int64 per request: start,
        // length, buffer; plus one counter slot per group, at most one per
        // request); every group stages its instance table in its own part of
        // it, and the slot reuses it only after the round has retired
        const size_t need = 4 * r->reqs.size();
        if (sl.pinned_cap < need) {
            if (sl.pinned) cudaFreeHost(sl.pinned);
            sl.pinned = nullptr;
            sl.pinned_cap = 0;
            if (cudaHostAlloc((void**)&sl.pinned, need * 8, cudaHostAllocDefault) == cudaSuccess) sl.pinned_cap = need;
            else sl.pinned = nullptr;
        }
        size_t pin_at = 0;
        if (inject) rc = PS_ERR_CUDA;  // as if a launch had failed: nothing is queued
        // group by (dtype, mode): each group is one batched sort
        std::vector<bool> taken(r->reqs.size(), false);
        for (size_t i = 0; i < r->reqs.size() && rc == PS_OK; i++) {
            if (taken[i]) continue;
            std::vector<size_t> grp;
            for (size_t j = i; j < r->reqs.size(); j++)
                if (!taken[j] && r->reqs[j].dtype == r->reqs[i].dtype && r->reqs[j].mode == r->reqs[i].mode) {
                    grp.push_back(j);
                    taken[j] = true;
                }
            const int dtype = r->reqs[i].dtype, mode = r->reqs[i].mode;
            const size_t kb = key_bytes(dtype);
            std::vector<int64_t> off(grp.size() + 1, 0);
            for (size_t k = 0; k < grp.size(); k++) off[k + 1] = off[k] + r->reqs[grp[k]].n;
            const int64_t total = off.back();
            int64_t* pin = sl.pinned ? sl.pinned + pin_at : nullptr;
            const size_t pin_cap = sl.pinned ? 3 * grp.size() + 1 : 0;
            pin_at += 3 * grp.size() + 1;
            std::vector<void*> own(grp.size());
            for (size_t k = 0; k < grp.size(); k++) own[k] = r->reqs[grp[k]].keys;
            void* stage = nullptr;  // the passes between the first and the last
            rc = ws_alloc(&stage, (size_t)total * kb, st);
            if (rc != PS_OK) break;
            rc = batch_sort(off, stage, dtype, mode, st, pin, pin_cap, nullptr, &own);
            ws_free(stage, st);
        }
        r->status = rc;
        cudaError_t e = cudaLaunchHostFunc(st, retire, r);
        if (e != cudaSuccess) {
            // the callback could not be queued: the stream is unusable
            std::lock_guard<std::mutex> lk(mu);
            sl.dead = true;
        }
        if (e != cudaSuccess) retire_with(r, fail_cuda(e));
        return rc;
    }

    // Busy slots whose stream reports an error will never run their
    // completion callbacks: retire their rounds here and retire the slot.
    void check_streams(std::unique_lock<std::mutex>& lk)
    {
        Round* rs[NSLOT];
        cudaStream_t ss[NSLOT];
        int k = 0;
        for (int i = 0; i < NSLOT; i++)
            if (slots[i].busy && slots[i].cur && !slots[i].dead) {
                rs[k] = slots[i].cur;
                ss[k++] = slots[i].stream;
            }
        lk.unlock();  // no CUDA call while holding the lock the callbacks take
        for (int i = 0; i < k; i++) {
            const cudaError_t e = cudaStreamQuery(ss[i]);
            if (e == cudaSuccess || e == cudaErrorNotReady) continue;
            {
                std::lock_guard<std::mutex> g(mu);
                slots[rs[i]->slot].dead = true;
            }
            retire_with(rs[i], fail_cuda(e));
        }
        lk.lock();
    }

    void run()
    {
        cudaSetDevice(dev);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            int slot = -1;
            int live = 0;
            for (int i = 0; i < NSLOT; i++) {
                if (!slots[i].dead && !slots[i].busy && kill_slots > 0) {
                    slots[i].dead = true;  // injected stream failure of an idle slot
                    kill_slots--;
                }
                if (slots[i].dead) continue;
                live++;
                if (!slots[i].busy && slot < 0) slot = i;
            }
            if (live == 0) {
                // every stream failed: fail what is queued
                while (!pending.empty()) {
                    done.push_back(Done{pending.front().id, PS_ERR_CUDA});
                    pending.pop_front();
                }
                pending_keys = 0;
                if (closing && inflight == 0) break;
            }
            const bool can = slot >= 0 && !pending.empty() && inflight < max_inflight &&
                             used + pending.front().cost <= budget;
            if (!can) {
                if (closing && pending.empty() && inflight == 0) break;
                // bounded wait: wake up to look for failed streams
                cv.wait_for(lk, std::chrono::milliseconds(50));
                check_streams(lk);
                continue;
            }
            delete slots[slot].cur;  // retired: the slot is free
            Round* r = new Round{this, slot, {}, 0, PS_OK};
            slots[slot].cur = r;
            // a round takes queued requests in order.  With a short queue it
            // stops at round_keys keys (at least one request), so that small
            // requests are not held back behind large ones; with a long queue
            // (the GPU is saturated) it takes everything admissible, as large
            // rounds keep the GPU busiest.
            const int64_t cap = pending.size() > LONG_QUEUE ? INT64_MAX : round_keys;
            int64_t keys = 0;
            while (!pending.empty() && inflight + (int)r->reqs.size() < max_inflight &&
                   used + r->cost + pending.front().cost <= budget &&
                   (r->reqs.empty() || keys + pending.front().n <= cap)) {
                keys += pending.front().n;
                pending_keys -= pending.front().n;
                r->cost += pending.front().cost;
                r->reqs.push_back(pending.front());
                pending.pop_front();
            }
            used += r->cost;
            inflight += (int)r->reqs.size();
            slots[slot].busy = true;
            lk.unlock();
            launch(r);
            lk.lock();
        }
    }
};

}  // namespace
}  // namespace ps

using namespace ps;

struct ps_server {
    Server s;
};

extern "C" {

int ps_server_open(size_t mem_budget_bytes, int max_inflight, ps_server** out)
{
    if (!out || mem_budget_bytes == 0 || max_inflight < 1) return PS_ERR_INVALID_ARG;
    *out = nullptr;
    ps_server* p = new (std::nothrow) ps_server();
    if (!p) return PS_ERR_NO_MEMORY;
    Server& s = p->s;
    s.budget = mem_budget_bytes;
    s.max_inflight = max_inflight;
    if (const char* v = getenv("PS_SERVER_ROUND_KEYS")) {
        const long long k = atoll(v);
        if (k > 0) s.round_keys = k;
    }
    cudaError_t e = cudaGetDevice(&s.dev);
    for (int i = 0; i < NSLOT && e == cudaSuccess; i++) e = cudaStreamCreateWithFlags(&s.slots[i].stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        for (int i = 0; i < NSLOT; i++)
            if (s.slots[i].stream) cudaStreamDestroy(s.slots[i].stream);
        delete p;
        return fail_cuda(e);
    }
    s.worker = std::thread([&s] { s.run(); });
    *out = p;
    return PS_OK;
}

int ps_server_submit(ps_server* p, void* dev_keys, int64_t n, int dtype, int pivot_mode, uint64_t* req_id)
{
    if (!p || !req_id || n < 0) return PS_ERR_INVALID_ARG;
    if (dtype < PS_I32 || dtype > PS_U64) return PS_ERR_UNSUPPORTED;
    if (pivot_mode != PS_PIVOT_REGULAR && pivot_mode != PS_PIVOT_EXACT) return PS_ERR_UNSUPPORTED;
    const size_t kb = key_bytes(dtype);
    if (n > 1 && (!dev_keys || (uintptr_t)dev_keys % kb != 0)) return PS_ERR_INVALID_ARG;
    Server& s = p->s;
    // staging copy plus the sort's workspace for this request
    const size_t cost = n > 1 ? (size_t)n * kb + sort_ws_bytes(n, dtype) : 0;
    {
        std::lock_guard<std::mutex> lk(s.mu);
        if (s.closing) return PS_ERR_INVALID_ARG;
        if (cost > s.budget) return PS_ERR_BUSY;  // could never be admitted
        *req_id = s.next_id++;
        if (n <= 1) s.done.push_back(Done{*req_id, PS_OK});
        else {
            s.pending.push_back(Req{*req_id, dev_keys, n, dtype, pivot_mode, cost});
            s.pending_keys += n;
        }
    }
    s.cv.notify_all();
    return PS_OK;
}

int ps_server_poll(ps_server* p, uint64_t* done_ids, int* statuses, int cap, int* n_done)
{
    if (!p || !n_done || cap < 0 || (cap > 0 && (!done_ids || !statuses))) return PS_ERR_INVALID_ARG;
    Server& s = p->s;
    std::lock_guard<std::mutex> lk(s.mu);
    const int k = (int)std::min<size_t>((size_t)cap, s.done.size());
    for (int i = 0; i < k; i++) {
        done_ids[i] = s.done[i].id;
        statuses[i] = s.done[i].status;
    }
    s.done.erase(s.done.begin(), s.done.begin() + k);
    *n_done = k;
    return PS_OK;
}

int ps_server_debug_fail(ps_server* p, int what, int count)
{
    if (!p || count < 0 || (what != 0 && what != 1)) return PS_ERR_INVALID_ARG;
    Server& s = p->s;
    {
        std::lock_guard<std::mutex> lk(s.mu);
        if (what == 0) s.fail_rounds += count;
        else s.kill_slots += count;
    }
    s.cv.notify_all();
    return PS_OK;
}

int ps_server_close(ps_server* p)
{
    if (!p) return PS_ERR_INVALID_ARG;
    Server& s = p->s;
    {
        std::lock_guard<std::mutex> lk(s.mu);
        s.closing = true;
    }
    s.cv.notify_all();
    if (s.worker.joinable()) s.worker.join();
    for (int i = 0; i < NSLOT; i++) {
        if (s.slots[i].stream) {
            cudaStreamSynchronize(s.slots[i].stream);
            cudaStreamDestroy(s.slots[i].stream);
        }
        if (s.slots[i].pinned) cudaFreeHost(s.slots[i].pinned);
        delete s.slots[i].cur;
    }
    delete p;
    return PS_OK;
}

}  // extern "C"
