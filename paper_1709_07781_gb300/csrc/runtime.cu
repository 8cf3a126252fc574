// Actor layer of libka (Sec. 3.2-3.5 of the paper, rebuilt on one CUDA stream):
//
//   * Ref      - the paper's mem_ref<T>: a typed, sized device buffer with a
//                device-resident count word (the configuration word of
//                Sec. 4.1), pool-owned or borrowed; dropping the last holder
//                returns its memory to the pool (Sec. 3.5).
//   * Actor    - a stage actor wraps one kernel; a composite C = B (.) A is the
//                flattened list of its stage actors (Sec. 3.5).
//   * Mailbox  - lock-free multi-producer single-consumer queue per stage actor.
//                One dispatcher thread drains the actors that have mail (the
//                mailbox-to-command-queue mapping of Sec. 3.6): each message
//                becomes kernel launches on the system stream, and the output
//                references are forwarded to the next stage's mailbox before
//                the kernels finish (stream order replaces OpenCL events).
//   * Request  - the promise of the composition: after the last stage the
//                dispatcher records an event. A receiver that is waiting polls
//                that event itself; otherwise a completion thread waits for it.
//                Whichever claims the request first reads the result length
//                (and, in value mode, the data) and fulfils the promise.
//   * Inline dispatch - a request whose first actor has no mail queued is
//                dispatched on the requesting thread, under the same lock the
//                dispatcher holds while it runs actors, so each actor still
//                takes one message at a time and in mailbox order; the
//                dispatcher thread carries the rest.
// Memory: a dedicated CUDA memory pool with stream-ordered allocation on the
// system stream, and a byte budget over the live references.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ka_internal.h"

namespace ka {
namespace rt {

// ---------------------------------------------------------------------------
// Intrusive lock-free MPSC queue (Vyukov): push from any thread, pop from one.
struct QNode {
    std::atomic<QNode *> next{nullptr};
};

class MpscQueue {
  public:
    MpscQueue() : head_(&stub_), tail_(&stub_) {}
    void push(QNode *n) {
        n->next.store(nullptr, std::memory_order_relaxed);
        QNode *prev = head_.exchange(n, std::memory_order_acq_rel);
        prev->next.store(n, std::memory_order_release);
    }
    // nullptr when empty (or when a push is half-way; the caller retries later)
    QNode *pop() {
        QNode *t = tail_;
        QNode *next = t->next.load(std::memory_order_acquire);
        if (t == &stub_) {
            if (!next) return nullptr;
            tail_ = next;
            t = next;
            next = next->next.load(std::memory_order_acquire);
        }
        if (next) {
            tail_ = next;
            return t;
        }
        if (t != head_.load(std::memory_order_acquire)) return nullptr;
        push(&stub_);
        next = t->next.load(std::memory_order_acquire);
        if (next) {
            tail_ = next;
            return t;
        }
        return nullptr;
    }
    bool maybe_nonempty() const {
        return tail_->next.load(std::memory_order_acquire) != nullptr || head_.load(std::memory_order_acquire) != tail_;
    }

  private:
    std::atomic<QNode *> head_;
    QNode *tail_;
    QNode stub_;
};

// ---------------------------------------------------------------------------
// Handle tables: opaque handles are (generation << 32 | slot + 1), so a
// released handle is detected (KA_E_STALE) even if its slot is reused.
template <class T>
class HandleTable {
  public:
    uint64_t add(T *obj) {
        std::lock_guard<std::mutex> l(mu_);
        return add_locked(obj);
    }
    uint64_t add_locked(T *obj) {
        uint32_t slot;
        if (!free_.empty()) {
            slot = free_.back();
            free_.pop_back();
        } else {
            slot = uint32_t(slots_.size());
            slots_.push_back({nullptr, 1});
        }
        slots_[slot].obj = obj;
        return (uint64_t(slots_[slot].gen) << 32) | (uint64_t(slot) + 1);
    }
    T *get(uint64_t h) {
        std::lock_guard<std::mutex> l(mu_);
        return get_locked(h);
    }
    // Removes the handle; returns the object or nullptr if stale.
    T *remove(uint64_t h) {
        std::lock_guard<std::mutex> l(mu_);
        return remove_locked(h);
    }
    T *remove_locked(uint64_t h) {
        T *o = get_locked(h);
        if (!o) return nullptr;
        const uint32_t slot = uint32_t(h & 0xFFFFFFFFu) - 1;
        slots_[slot].obj = nullptr;
        slots_[slot].gen++;
        free_.push_back(slot);
        return o;
    }
    // Removes every handle whose object satisfies pred; returns the objects.
    template <class Pred>
    std::vector<T *> remove_if(Pred pred) {
        std::lock_guard<std::mutex> l(mu_);
        std::vector<T *> out;
        for (uint32_t i = 0; i < slots_.size(); ++i) {
            Slot &e = slots_[i];
            if (e.obj && pred(e.obj)) {
                out.push_back(e.obj);
                e.obj = nullptr;
                e.gen++;
                free_.push_back(i);
            }
        }
        return out;
    }
    std::mutex &mutex() { return mu_; }
    T *get_locked(uint64_t h) {
        const uint64_t s = h & 0xFFFFFFFFu;
        if (s == 0 || s > slots_.size()) return nullptr;
        auto &e = slots_[s - 1];
        if (e.gen != uint32_t(h >> 32) || !e.obj) return nullptr;
        return e.obj;
    }

  private:
    struct Slot {
        T *obj;
        uint32_t gen;
    };
    std::mutex mu_;
    std::vector<Slot> slots_;
    std::vector<uint32_t> free_;
};

struct System;

struct Ref {
    std::atomic<int> rc{1};
    std::atomic<int> ext{0};  // external holders (valid handle while > 0)
    uint64_t handle = 0;
    System *sys = nullptr;
    void *ptr = nullptr;          // element data
    uint32_t *d_count = nullptr;  // device count word (nullptr: n_host is the length)
    uint64_t n_host = 0;
    uint64_t capacity = 0;
    uint64_t bytes = 0;  // pool bytes held (0 for borrowed memory)
    void *block = nullptr;
    int32_t dtype = KA_U32;
    int32_t access = KA_READ_WRITE;
};

struct StageSpec {
    int32_t kind = KA_STAGE_EMPTY;
    PredDev pred{};
    uint32_t mul = 1;
    ka_tile tile{0, 0};
    int in_arity = 1, out_arity = 1;
    uint32_t width = 0, height = 0, iters = 0;  // KA_STAGE_MANDELBROT
};

struct Actor {
    std::atomic<int> rc{1};
    uint64_t handle = 0;
    System *sys = nullptr;
    bool composite = false;
    StageSpec spec;
    std::vector<Actor *> stages;  // composite: stage actors, first stage first
    int in_arity = 1, out_arity = 1;
    MpscQueue mailbox;
    QNode run_node;
    std::atomic<bool> scheduled{false};
    std::atomic<int32_t> fail_after{-1};
    std::atomic<uint64_t> processed{0};
};

struct Request;

// The message of a request: its references as it travels from stage to stage
// (one message per request, kept inside the request object).
struct Msg : QNode {
    Request *req = nullptr;
    int stage = 0;
    int n_refs = 0;
    Ref *refs[KA_MSG_MAX_REFS] = {nullptr, nullptr, nullptr, nullptr};
    uint64_t seed = 0;
    uint64_t gen_n = 0;
};

struct Request {
    uint64_t handle = 0;
    Msg msg;  // travels through the stages while the request is in flight
    System *sys = nullptr;
    std::vector<Actor *> stages;  // retained
    // value mode
    uint32_t *h_out = nullptr;
    uint64_t h_out_cap = 0;
    // result
    std::vector<Ref *> result;
    uint64_t count = 0;
    ka_status status = KA_OK;
    uint32_t *pinned_count = nullptr;  // host-mapped slot: length, device error word, completion tag
    uint32_t *pinned_dev = nullptr;    // the same slot as the device addresses it
    uint32_t seq = 0;                  // completion tag of the current use (changes every use)
    bool tagged = false;               // the publish kernel stores `seq` when the stream gets there
    cudaEvent_t event = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::atomic<bool> done{false};
    bool debug_check = false;
    // holders: the caller's handle; the last holder recycles the request
    std::atomic<int> holders{1};
    std::atomic<bool> recorded{false};  // event recorded after the last stage
    std::atomic<bool> blocked{false};   // a receiver is (about to be) blocked on cv
    // The two words the completion thread watches while a receiver polls, on
    // a cache line of their own: the fulfilling receiver's writes to the
    // result fields above then do not contend with the watcher's reads.
    // claim = (use << 1) | taken: one thread per use fulfils the request.
    // Recycling starts the next use unclaimed, so the completion queue's
    // entry for an earlier use (which holds no reference) cannot claim it.
    alignas(64) std::atomic<uint64_t> claim{0};
    std::atomic<bool> waiting{false};  // a receiver is polling for completion
    char pad_[55];
};

// A request of the completion queue: the object (kept while its system
// lives) and the use the entry is for.
struct Completion {
    Request *req;
    uint64_t use;
};

static bool try_claim(Request *r, uint64_t use) {
    uint64_t open = use << 1;
    return r->claim.compare_exchange_strong(open, open | 1u, std::memory_order_acq_rel);
}
static uint64_t current_use(const Request *r) { return r->claim.load(std::memory_order_acquire) >> 1; }
static bool is_claimed(const Request *r) { return (r->claim.load(std::memory_order_acquire) & 1u) != 0; }

struct System {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t readback = nullptr;
    std::mutex readback_mu;  // value-mode copies on `readback` (one claimer at a time)
    cudaMemPool_t pool = nullptr;
    uint64_t budget = 0;
    std::atomic<uint64_t> in_use{0};  // budget held: blocks handed out plus blocks in the cache
    // Freed pool blocks kept for reuse, by size: every use of a block is
    // ordered on `stream`, so a block freed by one request can serve the next
    // without a cudaFreeAsync / cudaMallocFromPoolAsync pair (a few
    // microseconds of host time each).
    std::mutex cache_mu;
    std::unordered_map<uint64_t, std::vector<void *>> cache;
    uint64_t cached_bytes = 0;
    // Released Ref objects kept for reuse (under cache_mu, taken with a
    // cached block in one critical section): a stage's output costs no heap
    // allocation.
    std::vector<Ref *> ref_free;
    bool debug = false;

    // workspace for the single-pass kernels (grown on demand, stream-ordered)
    void *ws = nullptr;
    uint64_t ws_bytes = 0;

    // pinned slots for result counts
    std::mutex pin_mu;
    uint32_t *pinned = nullptr;
    uint32_t *pinned_dev = nullptr;  // device address of `pinned` (host-mapped)
    std::vector<uint32_t> pin_free;

    // finished requests kept for reuse, each with its pinned count slot and
    // completion event
    std::mutex req_mu;
    std::vector<Request *> req_free;

    MpscQueue runq;
    // held while actors run (dispatcher or inline dispatch on a requesting
    // thread): actors take one message at a time, launches stay in order
    std::mutex dispatch_mu;
    std::mutex wake_mu;
    std::condition_variable wake_cv;
    std::atomic<bool> sleeping{false};
    std::atomic<bool> stop{false};
    std::atomic<bool> dead{false};
    std::atomic<bool> kill_requested{false};
    std::thread dispatcher;

    std::mutex comp_mu;
    std::condition_variable comp_cv;
    std::deque<Completion> comp_q;
    bool comp_kick = false;  // (under comp_mu) a receiver about to block, or shutdown: sweep now
    std::thread completer;

    std::atomic<int64_t> inflight{0};
    ka_monitor_fn monitor = nullptr;
    void *monitor_user = nullptr;
    std::atomic<bool> monitor_fired{false};
};

HandleTable<System> g_systems;
HandleTable<Ref> g_refs;
HandleTable<Actor> g_actors;
HandleTable<Request> g_requests;

constexpr uint32_t kPinnedSlots = 65536;
constexpr uint32_t kPinnedWords = 4;  // per slot: length, device error word, completion tag, unused

// ---------------------------------------------------------------------------
// References and the pool.
constexpr uint64_t kCacheMaxBytes = 4ull << 30;

// Returns every cached block to the pool (stream ordered).
static void cache_flush(System *s) {
    std::lock_guard<std::mutex> l(s->cache_mu);
    for (auto &kv : s->cache)
        for (void *p : kv.second) {
            cudaFreeAsync(p, s->stream);
            s->in_use.fetch_sub(kv.first);
        }
    s->cache.clear();
    s->cached_bytes = 0;
}

constexpr size_t kRefFreeMax = 4096;

// A new pool block of `bytes` (not from the cache), within the budget.
static ka_status pool_alloc_new(System *s, uint64_t bytes, void **out) {
    uint64_t cur = s->in_use.load();
    bool flushed = false;
    for (;;) {
        if (cur + bytes > s->budget) {
            if (flushed) return KA_E_BUDGET;
            cache_flush(s);  // cached blocks count against the budget: give them back first
            flushed = true;
            cur = s->in_use.load();
            continue;
        }
        if (s->in_use.compare_exchange_weak(cur, cur + bytes)) break;
    }
    cudaError_t e = cudaMallocFromPoolAsync(out, bytes, s->pool, s->stream);
    if (e != cudaSuccess) {
        s->in_use.fetch_sub(bytes);
        cudaGetLastError();
        return KA_E_OOM;
    }
    return KA_OK;
}

static ka_status new_owned_ref(System *s, uint64_t capacity, Ref **out) {
    const uint64_t data = (capacity * 4 + 255) / 256 * 256;
    const uint64_t bytes = data + 256;
    void *blk = nullptr;
    Ref *r = nullptr;
    {
        std::lock_guard<std::mutex> l(s->cache_mu);
        auto it = s->cache.find(bytes);
        if (it != s->cache.end() && !it->second.empty()) {
            blk = it->second.back();
            it->second.pop_back();
            s->cached_bytes -= bytes;
        }
        if (!s->ref_free.empty()) {
            r = s->ref_free.back();
            s->ref_free.pop_back();
        }
    }
    if (!blk) {
        const ka_status st = pool_alloc_new(s, bytes, &blk);
        if (st != KA_OK) {
            delete r;
            return st;
        }
    }
    if (r) {  // a recycled object: back to a new Ref's state
        r->rc.store(1, std::memory_order_relaxed);
        r->ext.store(0, std::memory_order_relaxed);
        r->handle = 0;
        r->n_host = 0;
        r->dtype = KA_U32;
        r->access = KA_READ_WRITE;
    } else {
        r = new Ref;
    }
    r->sys = s;
    r->block = blk;
    r->ptr = blk;
    r->d_count = reinterpret_cast<uint32_t *>(static_cast<char *>(blk) + data);
    r->capacity = capacity;
    r->bytes = bytes;
    *out = r;
    return KA_OK;
}

static void ref_retain(Ref *r) { r->rc.fetch_add(1, std::memory_order_relaxed); }

// The last holder let go: the block goes to the cache (or back to the pool)
// and the object to the free list, in one critical section.
static void ref_drop(Ref *r) {
    if (!r) return;
    if (r->rc.fetch_sub(1, std::memory_order_acq_rel) != 1) return;
    System *s = r->sys;
    void *blk = r->block;
    uint64_t bytes = r->bytes;
    {
        std::lock_guard<std::mutex> l(s->cache_mu);
        if (bytes && s->cached_bytes + bytes <= kCacheMaxBytes && s->cached_bytes + bytes <= s->budget / 4) {
            s->cache[bytes].push_back(blk);
            s->cached_bytes += bytes;
            bytes = 0;
        }
        if (s->ref_free.size() < kRefFreeMax) {
            s->ref_free.push_back(r);
            r = nullptr;  // (another thread may take it from here on)
        }
    }
    if (bytes) {
        cudaFreeAsync(blk, s->stream);
        s->in_use.fetch_sub(bytes);
    }
    delete r;
}

// One more external holder, given one of r's holds (the caller's). A
// reference has one handle at a time: its first external holder makes it,
// later ones (the same reference returned by another receive, as an empty
// stage passes its input on, or retained) share it, and the last release
// ends it.
static uint64_t ref_export(Ref *r) {
    std::lock_guard<std::mutex> l(g_refs.mutex());
    if (r->ext.fetch_add(1) == 0) r->handle = g_refs.add_locked(r);
    return r->handle;
}

// Length arguments for a kernel reading `r`: (n, n_ptr).
static inline void ref_len(const Ref *r, uint64_t *n, const uint32_t **n_ptr) {
    if (r->d_count) {
        *n = r->capacity;
        *n_ptr = r->d_count;
    } else {
        *n = r->n_host;
        *n_ptr = nullptr;
    }
}

static ka_status ensure_workspace(System *s, uint64_t capacity) {
    uint64_t need = workspace_bytes_for_tiles(tiles_for(capacity, 512) + 1);
    if (need <= s->ws_bytes) return KA_OK;
    if (need < (1ull << 20)) need = 1ull << 20;
    void *p = nullptr;
    if (cudaMallocFromPoolAsync(&p, need, s->pool, s->stream) != cudaSuccess) {
        cudaGetLastError();
        return KA_E_OOM;
    }
    if (s->ws) cudaFreeAsync(s->ws, s->stream);
    s->ws = p;
    s->ws_bytes = need;
    return ka_workspace_init(p, need, s->stream);
}

// ---------------------------------------------------------------------------
// Dispatcher.
static void wake_dispatcher(System *s) {
    if (s->sleeping.load(std::memory_order_acquire)) {
        std::lock_guard<std::mutex> l(s->wake_mu);
        s->wake_cv.notify_one();
    }
}

static void schedule(Actor *a) {
    if (!a->scheduled.exchange(true, std::memory_order_acq_rel)) {
        a->sys->runq.push(&a->run_node);
        wake_dispatcher(a->sys);
    }
}

static void post(Actor *a, Msg *m) {
    a->mailbox.push(m);
    schedule(a);
}

static void complete(Request *r, ka_status st) {
    System *s = r->sys;
    r->status = st;
    r->done.store(true, std::memory_order_seq_cst);
    // A receiver that polls sees `done`; one that blocks on cv has set
    // `blocked` first (both sequentially consistent, so at least one side sees
    // the other), and is woken under the lock.
    if (r->blocked.load(std::memory_order_seq_cst)) {
        { std::lock_guard<std::mutex> l(r->mu); }
        r->cv.notify_all();
    }
    s->inflight.fetch_sub(1);
}

static void release_msg_refs(Msg *m) {
    for (int i = 0; i < m->n_refs; ++i) ref_drop(m->refs[i]);
    m->n_refs = 0;
}

static void fail_request(Msg *m, ka_status st) {
    release_msg_refs(m);
    complete(m->req, st);
}

// Runs one stage for message m; on success fills outs/n_outs.
// Name of a stage's NVTX range: each stage's launches show as one range on
// the issuing thread in a profiler's timeline.
static const char *stage_name(int32_t kind) {
    switch (kind) {
    case KA_STAGE_GENERATE: return "ka stage: generate";
    case KA_STAGE_MAP_HASH: return "ka stage: map hash";
    case KA_STAGE_PREDICATE: return "ka stage: predicate";
    case KA_STAGE_EXSCAN: return "ka stage: exclusive scan";
    case KA_STAGE_SCATTER: return "ka stage: scatter";
    case KA_STAGE_COMPACT: return "ka stage: compact";
    case KA_STAGE_PREPARE: return "ka stage: prepare index";
    case KA_STAGE_EMPTY: return "ka stage: empty";
    case KA_STAGE_MANDELBROT: return "ka stage: mandelbrot";
    default: return "ka stage";
    }
}

static ka_status run_stage(System *s, const StageSpec &sp, Msg *m, Ref **outs, int *n_outs) {
    cudaStream_t st = s->stream;
    *n_outs = 0;
    Ref *x = m->n_refs > 0 ? m->refs[0] : nullptr;
    uint64_t n = 0;
    const uint32_t *n_ptr = nullptr;
    if (x) ref_len(x, &n, &n_ptr);
    ka_status e = KA_OK;
    switch (sp.kind) {
    case KA_STAGE_GENERATE: {
        Ref *y;
        if ((e = new_owned_ref(s, m->gen_n, &y)) != KA_OK) return e;
        e = launch_generate(static_cast<uint32_t *>(y->ptr), m->gen_n, m->seed, y->d_count, st);
        outs[(*n_outs)++] = y;
        return e;
    }
    case KA_STAGE_MANDELBROT: {
        Ref *y;
        const uint64_t pixels = uint64_t(sp.width) * sp.height;
        if ((e = new_owned_ref(s, pixels, &y)) != KA_OK) return e;
        // the rectangle of the paper's workload (Sec. 5.4)
        e = launch_mandelbrot(static_cast<uint32_t *>(y->ptr), sp.width, sp.height, -0.5f, -0.7375f, 0.1f, -0.1375f,
                              sp.iters, y->d_count, st);
        outs[(*n_outs)++] = y;
        return e;
    }
    case KA_STAGE_MAP_HASH: {
        Ref *y;
        if ((e = new_owned_ref(s, x->capacity, &y)) != KA_OK) return e;
        e = launch_map_hash(static_cast<const uint32_t *>(x->ptr), n, n_ptr, static_cast<uint32_t *>(y->ptr),
                            y->d_count, st);
        outs[(*n_outs)++] = y;
        return e;
    }
    case KA_STAGE_PREDICATE: {
        Ref *f;
        if ((e = new_owned_ref(s, x->capacity, &f)) != KA_OK) return e;
        e = launch_predicate(static_cast<const uint32_t *>(x->ptr), n, n_ptr, sp.pred, static_cast<uint32_t *>(f->ptr),
                             f->d_count, st);
        ref_retain(x);
        outs[(*n_outs)++] = x;
        outs[(*n_outs)++] = f;
        return e;
    }
    case KA_STAGE_EXSCAN: {
        Ref *f = m->refs[1];
        Ref *o;
        if ((e = new_owned_ref(s, f->capacity, &o)) != KA_OK) return e;
        if ((e = ensure_workspace(s, f->capacity)) != KA_OK) {
            ref_drop(o);
            return e;
        }
        uint64_t fn;
        const uint32_t *fn_ptr;
        ref_len(f, &fn, &fn_ptr);
        const ka_tile t = resolve_tile(KA_KERNEL_SCAN, fn, &sp.tile);
        e = launch_exclusive_scan(static_cast<const uint32_t *>(f->ptr), fn, fn_ptr, static_cast<uint32_t *>(o->ptr),
                                  o->d_count, s->ws, s->ws_bytes, t, st);
        ref_retain(x);
        ref_retain(f);
        outs[(*n_outs)++] = x;
        outs[(*n_outs)++] = f;
        outs[(*n_outs)++] = o;
        return e;
    }
    case KA_STAGE_SCATTER: {
        Ref *f = m->refs[1], *o = m->refs[2];
        Ref *y;
        if ((e = new_owned_ref(s, x->capacity, &y)) != KA_OK) return e;
        e = launch_scatter(static_cast<const uint32_t *>(x->ptr), static_cast<const uint32_t *>(f->ptr),
                           static_cast<const uint32_t *>(o->ptr), n, n_ptr, static_cast<uint32_t *>(y->ptr),
                           y->d_count, st);
        outs[(*n_outs)++] = y;
        return e;
    }
    case KA_STAGE_COMPACT: {
        Ref *y;
        if ((e = new_owned_ref(s, x->capacity, &y)) != KA_OK) return e;
        if ((e = ensure_workspace(s, x->capacity)) != KA_OK) {
            ref_drop(y);
            return e;
        }
        CompactLaunch L;
        L.in = static_cast<const uint32_t *>(x->ptr);
        L.out = static_cast<uint32_t *>(y->ptr);
        L.n_ptr = n_ptr;
        L.count = y->d_count;
        L.n = n;
        L.pred = sp.pred;
        L.mul = sp.mul;
        L.ws = s->ws;
        L.ws_bytes = s->ws_bytes;
        L.tile = resolve_tile(KA_KERNEL_COMPACT, x->capacity, &sp.tile);
        e = launch_compact(L, st);
        outs[(*n_outs)++] = y;
        return e;
    }
    case KA_STAGE_PREPARE: {
        const Ref *b = m->refs[1];
        Ref *y;
        if ((e = new_owned_ref(s, 2 * x->capacity, &y)) != KA_OK) return e;
        e = launch_prepare_index(static_cast<const uint32_t *>(x->ptr), static_cast<const uint32_t *>(b->ptr), n,
                                 n_ptr, static_cast<uint32_t *>(y->ptr), y->d_count, st);
        outs[(*n_outs)++] = y;
        return e;
    }
    case KA_STAGE_EMPTY: {
        e = launch_empty(st);
        for (int i = 0; i < m->n_refs; ++i) {
            ref_retain(m->refs[i]);
            outs[(*n_outs)++] = m->refs[i];
        }
        return e;
    }
    default: return KA_E_ARG;
    }
}

// Runs actor a on message m (the caller holds dispatch_mu). Returns the next
// stage's actor, to which m is to be posted, or nullptr once m is consumed
// (the request failed, or its last stage has been issued).
static Actor *process(System *s, Actor *a, Msg *m) {
    Request *r = m->req;
    if (s->stop.load()) {
        fail_request(m, KA_E_CLOSED);
        return nullptr;
    }
    // (fault injection: messages are counted only while it is armed)
    const int32_t fa = a->fail_after.load(std::memory_order_relaxed);
    if (fa >= 0 && a->processed.fetch_add(1) >= uint64_t(fa)) {
        fail_request(m, KA_E_INJECTED);
        return nullptr;
    }
    if (m->n_refs != a->spec.in_arity) {
        fail_request(m, KA_E_TYPE);
        return nullptr;
    }
    Ref *outs[KA_MSG_MAX_REFS];
    int n_outs = 0;
    nvtxRangePushA(stage_name(a->spec.kind));
    const ka_status e = run_stage(s, a->spec, m, outs, &n_outs);
    nvtxRangePop();
    if (e != KA_OK) {
        for (int i = 0; i < n_outs; ++i) ref_drop(outs[i]);
        fail_request(m, e);
        return nullptr;
    }
    release_msg_refs(m);
    const int next = m->stage + 1;
    if (next < int(r->stages.size())) {
        m->stage = next;
        m->n_refs = n_outs;
        for (int i = 0; i < n_outs; ++i) m->refs[i] = outs[i];
        return r->stages[next];
    }
    // Last stage: read the result length back and fulfil the promise once the
    // stream reaches this point.
    r->result.assign(outs, outs + n_outs);
    // The length (and in debug mode the device error word) is stored into the
    // request's host-mapped slot by a one-thread kernel on the stream.
    Ref *first = n_outs ? outs[0] : nullptr;
    const uint32_t *err = r->debug_check && s->ws ? &static_cast<WsHeader *>(s->ws)->error : nullptr;
    r->pinned_count[0] = first && !first->d_count ? uint32_t(first->n_host) : 0u;
    r->pinned_count[1] = 0;
    ka_status pub = KA_OK;
    r->tagged = false;
    if ((first && first->d_count) || err) {
        // the kernel stores a tag new to this use last: a receiver that sees
        // it knows the result is complete without asking the driver
        r->seq = r->seq + 1 ? r->seq + 1 : 1;
        pub = launch_publish(first ? first->d_count : nullptr, 1, r->pinned_count[0], err, r->pinned_dev,
                             r->pinned_dev + 1, s->stream, r->pinned_dev + 2, r->seq);
        r->tagged = pub == KA_OK;
    }
    cudaError_t rec = cudaSuccess;
    if (pub == KA_OK && !r->event) rec = cudaEventCreateWithFlags(&r->event, cudaEventDisableTiming);
    if (pub == KA_OK && rec == cudaSuccess) rec = cudaEventRecord(r->event, s->stream);
    if (pub != KA_OK || rec != cudaSuccess) {
        if (rec != cudaSuccess) cudaGetLastError();
        r->claim.fetch_or(1u, std::memory_order_acq_rel);
        complete(r, pub != KA_OK ? pub : cuda_status(rec));
        return nullptr;
    }
    // The use is read before `recorded` is set: from then on a polling
    // receiver may fulfil the request and its caller recycle it.
    const uint64_t use = current_use(r);
    r->recorded.store(true, std::memory_order_release);
    bool kick = false;
    {
        // (no reference: the caller's hold keeps the object; its use number
        // tells the completion thread whether the entry is still current)
        std::lock_guard<std::mutex> l(s->comp_mu);
        s->comp_q.push_back({r, use});
        // A receiver that blocked before this push found no entry to sweep:
        // wake the thread for it. (It sets `blocked` before it kicks, and
        // both sides hold comp_mu, so one of the two sweeps sees the entry.)
        if (r->blocked.load(std::memory_order_acquire)) kick = s->comp_kick = true;
    }
    // (otherwise no wake-up: the completion thread sweeps its queue every
    // kCompleterPeriodUs, and a receiver that stops polling wakes it)
    if (kick) s->comp_cv.notify_one();
    return nullptr;
}

// An actor with no mail queued and not waiting on the run queue: a message
// dispatched to it now cannot overtake one sent to it earlier.
static bool actor_idle(Actor *a) {
    return !a->scheduled.load(std::memory_order_acquire) && !a->mailbox.maybe_nonempty();
}

static void fire_monitor(System *s, ka_status reason) {
    if (s->monitor && !s->monitor_fired.exchange(true)) s->monitor(s->monitor_user, reason);
}

static void drain_with(System *s, ka_status st) {
    // fail every message still queued
    for (;;) {
        QNode *n = s->runq.pop();
        if (!n) break;
        Actor *a = reinterpret_cast<Actor *>(reinterpret_cast<char *>(n) - offsetof(Actor, run_node));
        for (;;) {
            QNode *q = a->mailbox.pop();
            if (!q) break;
            fail_request(static_cast<Msg *>(q), st);
        }
        a->scheduled.store(false);
    }
}

// Host-side spin windows (microseconds) before a thread blocks: a blocked
// thread costs a futex wake-up (several microseconds) when work arrives.
constexpr int kDispatcherSpinUs = 2000;
constexpr int kCompleterPeriodUs = 2000;
constexpr int kReceiveSpinUs = 2000;

static void dispatcher_main(System *s) {
    cudaSetDevice(s->device);
    auto idle_since = std::chrono::steady_clock::now();
    while (!s->stop.load(std::memory_order_acquire)) {
        if (s->kill_requested.load()) {
            // mark the actor dead only after its queued work has been failed
            // and its monitor has been told, so an observer of `dead` sees both
            drain_with(s, KA_E_CLOSED);
            fire_monitor(s, KA_E_CLOSED);
            s->dead.store(true);
            return;
        }
        QNode *n = s->runq.pop();
        if (!n) {
            const auto now = std::chrono::steady_clock::now();
            // stay awake for a while after the last message: a request that
            // follows soon (the usual request/receive loop) then costs no wake-up
            if (now - idle_since < std::chrono::microseconds(kDispatcherSpinUs)) {
                std::this_thread::yield();
                continue;
            }
            std::unique_lock<std::mutex> l(s->wake_mu);
            s->sleeping.store(true, std::memory_order_release);
            if (!s->runq.maybe_nonempty() && !s->stop.load() && !s->kill_requested.load())
                s->wake_cv.wait_for(l, std::chrono::milliseconds(2));
            s->sleeping.store(false, std::memory_order_release);
            continue;
        }
        idle_since = std::chrono::steady_clock::now();
        Actor *a = reinterpret_cast<Actor *>(reinterpret_cast<char *>(n) - offsetof(Actor, run_node));
        {
            std::lock_guard<std::mutex> dl(s->dispatch_mu);
            for (int k = 0; k < 64; ++k) {
                QNode *q = a->mailbox.pop();
                if (!q) break;
                Msg *m = static_cast<Msg *>(q);
                if (Actor *nx = process(s, a, m)) post(nx, m);
            }
            a->scheduled.store(false, std::memory_order_release);
        }
        if (a->mailbox.maybe_nonempty()) schedule(a);
    }
    drain_with(s, KA_E_CLOSED);
}

// Fulfils request r once its event has completed (status st of the wait):
// result length, device error word, value-mode data. Run by the one thread
// that claimed r.
static void finalize(System *s, Request *r, ka_status st) {
    r->count = r->pinned_count[0];
    if (st == KA_OK && r->pinned_count[1] != 0) st = -int32_t(r->pinned_count[1]);
    if (st == KA_OK && r->h_out && !r->result.empty()) {
        Ref *y = r->result[0];
        uint64_t k = r->count < r->h_out_cap ? r->count : r->h_out_cap;
        if (k > y->capacity) k = y->capacity;
        if (k) {
            std::lock_guard<std::mutex> l(s->readback_mu);
            st = cuda_status(cudaMemcpyAsync(r->h_out, y->ptr, k * 4, cudaMemcpyDeviceToHost, s->readback));
            if (st == KA_OK) st = cuda_status(cudaStreamSynchronize(s->readback));
        }
    }
    complete(r, st);
}

// Wakes the completion thread for a sweep now.
static void kick_completer(System *s) {
    {
        std::lock_guard<std::mutex> l(s->comp_mu);
        s->comp_kick = true;
    }
    s->comp_cv.notify_one();
}

// The completion thread sweeps its queue every kCompleterPeriodUs (100 us
// once the system is stopping), or at once when kicked. An entry whose use is
// fulfilled (and maybe reused: the claim word then reads otherwise) is
// dropped; one whose receiver is polling is kept for a later sweep (that
// receiver fulfils it itself, and the thread stays out of the driver and off
// the request's cache lines meanwhile); any other is fulfilled here once its
// event completes. Requests do not wake the thread, so a request/receive loop
// leaves it asleep.
static void completer_main(System *s) {
    cudaSetDevice(s->device);
    std::deque<Completion> mine;
    for (;;) {
        {
            std::unique_lock<std::mutex> l(s->comp_mu);
            if (!s->comp_kick) {
                const auto period = std::chrono::microseconds(s->stop.load() ? 100 : kCompleterPeriodUs);
                s->comp_cv.wait_for(l, period, [s] { return s->comp_kick; });
            }
            s->comp_kick = false;
            while (!s->comp_q.empty()) {
                mine.push_back(s->comp_q.front());
                s->comp_q.pop_front();
            }
        }
        for (auto it = mine.begin(); it != mine.end();) {
            Request *r = it->req;
            const uint64_t open = it->use << 1;  // the entry's use, not yet claimed
            if (r->claim.load(std::memory_order_acquire) != open) {
                it = mine.erase(it);
                continue;
            }
            if (r->waiting.load(std::memory_order_acquire)) {
                ++it;
                continue;
            }
            const ka_status st = cuda_status(cudaEventSynchronize(r->event));
            if (try_claim(r, it->use)) finalize(s, r, st);
            it = mine.erase(it);
        }
        if (s->stop.load() && s->inflight.load() <= 0) return;
    }
}

// ---------------------------------------------------------------------------
static Actor *actor_of(ka_actor *h) { return g_actors.get(reinterpret_cast<uint64_t>(h)); }
static Ref *ref_of(const ka_ref *h) { return g_refs.get(reinterpret_cast<uint64_t>(h)); }
static System *sys_of(ka_system *h) { return g_systems.get(reinterpret_cast<uint64_t>(h)); }

static void actor_drop(Actor *a) {
    if (a->rc.fetch_sub(1) == 1) {
        for (Actor *c : a->stages)
            if (c != a) actor_drop(c);
        delete a;
    }
}

static uint32_t *take_pinned(System *s) {
    std::lock_guard<std::mutex> l(s->pin_mu);
    if (s->pin_free.empty()) return nullptr;
    const uint32_t i = s->pin_free.back();
    s->pin_free.pop_back();
    return s->pinned + kPinnedWords * i;
}

// A request object: a recycled one when the system has one, else a new one
// with its own pinned count slot (nullptr when the slots are used up).
static Request *request_new(System *s) {
    {
        std::lock_guard<std::mutex> l(s->req_mu);
        if (!s->req_free.empty()) {
            Request *r = s->req_free.back();
            s->req_free.pop_back();
            return r;
        }
    }
    uint32_t *pin = take_pinned(s);
    if (!pin) return nullptr;
    Request *r = new Request;
    r->sys = s;
    r->pinned_count = pin;
    r->pinned_dev = s->pinned_dev + (pin - s->pinned);
    return r;
}

// Returns an unused request (no handle, no stages, no result) for reuse.
static void request_recycle(Request *r) {
    r->handle = 0;
    r->h_out = nullptr;
    r->h_out_cap = 0;
    r->count = 0;
    r->status = KA_OK;
    r->debug_check = false;
    r->done.store(false, std::memory_order_relaxed);
    r->holders.store(1, std::memory_order_relaxed);
    r->recorded.store(false, std::memory_order_relaxed);
    r->claim.store(((r->claim.load(std::memory_order_relaxed) >> 1) + 1u) << 1, std::memory_order_release);
    r->waiting.store(false, std::memory_order_relaxed);
    r->blocked.store(false, std::memory_order_relaxed);
    System *s = r->sys;
    std::lock_guard<std::mutex> l(s->req_mu);
    s->req_free.push_back(r);
}

// Drops one holder of r; the last one releases what it holds and recycles it.
static void request_unhold(Request *r) {
    if (r->holders.fetch_sub(1, std::memory_order_acq_rel) != 1) return;
    for (Ref *x : r->result) ref_drop(x);
    r->result.clear();
    for (Actor *a : r->stages) actor_drop(a);
    r->stages.clear();
    request_recycle(r);
}

}  // namespace rt

ka_status system_exec_info(ka_system *h, int *device, uint64_t *budget) {
    rt::System *s = rt::sys_of(h);
    if (!s) return KA_E_STALE;
    *device = s->device;
    *budget = s->budget;
    return KA_OK;
}

}  // namespace ka

using namespace ka;
using namespace ka::rt;

extern "C" {

ka_status ka_system_create(const ka_config *cfg, ka_system **out) {
    if (!out) return KA_E_ARG;
    System *s = new System;
    s->device = cfg ? cfg->device : 0;
    s->debug = cfg && cfg->debug;
    s->budget = (cfg && cfg->budget_bytes) ? cfg->budget_bytes : (64ull << 30);
    if (const cudaError_t e = cudaSetDevice(s->device); e != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return cuda_status(e);
    }
    ka_status st = KA_OK;
    if (cfg && cfg->stream) {
        s->stream = static_cast<cudaStream_t>(cfg->stream);
    } else {
        st = cuda_status(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
        s->own_stream = true;
    }
    if (st == KA_OK) st = cuda_status(cudaStreamCreateWithFlags(&s->readback, cudaStreamNonBlocking));
    if (st == KA_OK) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = s->device;
        st = cuda_status(cudaMemPoolCreate(&s->pool, &props));
        if (st == KA_OK) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    if (st == KA_OK) st = cuda_status(cudaHostAlloc(&s->pinned, size_t(kPinnedSlots) * kPinnedWords * 4, cudaHostAllocMapped));
    if (st == KA_OK)
        st = cuda_status(cudaHostGetDevicePointer(reinterpret_cast<void **>(&s->pinned_dev), s->pinned, 0));
    if (st != KA_OK) {
        if (s->pinned) cudaFreeHost(s->pinned);
        if (s->readback) cudaStreamDestroy(s->readback);
        if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
        if (s->pool) cudaMemPoolDestroy(s->pool);
        delete s;
        return st;
    }
    // Zero every slot: a completion tag of 0 is never issued, while pinned
    // memory comes back uncleared (a slot of a destroyed system could still
    // hold the tag a new request is about to wait for).
    std::memset(s->pinned, 0, size_t(kPinnedSlots) * kPinnedWords * 4);
    s->pin_free.reserve(kPinnedSlots);
    for (uint32_t i = kPinnedSlots; i-- > 0;) s->pin_free.push_back(i);
    if (cfg && cfg->autotune_cache) ka_autotune_load(cfg->autotune_cache);
    s->dispatcher = std::thread(dispatcher_main, s);
    s->completer = std::thread(completer_main, s);
    *out = reinterpret_cast<ka_system *>(g_systems.add(s));
    return KA_OK;
}

ka_status ka_system_destroy(ka_system *h, int32_t force) {
    System *s = sys_of(h);
    if (!s) return KA_E_STALE;
    if (s->inflight.load() > 0 && !force) return KA_E_ARG;
    g_systems.remove(reinterpret_cast<uint64_t>(h));
    s->stop.store(true);
    {
        std::lock_guard<std::mutex> l(s->wake_mu);
        s->wake_cv.notify_all();
    }
    if (s->dispatcher.joinable()) s->dispatcher.join();
    // requests already launched finish normally; wait for the completer
    for (int i = 0; i < 200000 && s->inflight.load() > 0; ++i) {
        kick_completer(s);
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    kick_completer(s);
    if (s->completer.joinable()) s->completer.join();
    cudaStreamSynchronize(s->stream);
    // Every handle of this system becomes stale (KA_E_STALE from then on):
    // requests never received (their results and actors released), the
    // caller's references (pool memory returned), and the actors.
    for (Request *r : g_requests.remove_if([s](Request *r) { return r->sys == s; })) {
        for (Ref *x : r->result) ref_drop(x);
        for (Actor *a : r->stages) actor_drop(a);
        if (r->event) cudaEventDestroy(r->event);
        delete r;
    }
    for (Ref *r : g_refs.remove_if([s](Ref *r) { return r->sys == s; })) {
        if (r->bytes) cudaFreeAsync(r->block, s->stream);
        delete r;
    }
    for (Actor *a : g_actors.remove_if([s](Actor *a) { return a->sys == s; })) actor_drop(a);
    cache_flush(s);
    for (Ref *r : s->ref_free) delete r;
    s->ref_free.clear();
    if (s->ws) cudaFreeAsync(s->ws, s->stream);
    cudaStreamSynchronize(s->stream);
    for (Request *r : s->req_free) {
        if (r->event) cudaEventDestroy(r->event);
        delete r;
    }
    if (s->pinned) cudaFreeHost(s->pinned);
    cudaStreamDestroy(s->readback);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    cudaMemPoolDestroy(s->pool);
    delete s;
    return KA_OK;
}

ka_status ka_system_pool_bytes(ka_system *h, uint64_t *in_use, uint64_t *budget) {
    System *s = sys_of(h);
    if (!s) return KA_E_STALE;
    if (in_use) {
        std::lock_guard<std::mutex> l(s->cache_mu);
        *in_use = s->in_use.load() - s->cached_bytes;  // bytes held by live references
    }
    if (budget) *budget = s->budget;
    return KA_OK;
}

ka_status ka_system_monitor(ka_system *h, ka_monitor_fn fn, void *user) {
    System *s = sys_of(h);
    if (!s) return KA_E_STALE;
    s->monitor_user = user;
    s->monitor = fn;
    if (s->dead.load()) fire_monitor(s, KA_E_CLOSED);
    return KA_OK;
}

ka_status ka_debug_kill_dispatcher(ka_system *h) {
    System *s = sys_of(h);
    if (!s) return KA_E_STALE;
    s->kill_requested.store(true);
    {
        std::lock_guard<std::mutex> l(s->wake_mu);
        s->wake_cv.notify_all();
    }
    for (int i = 0; i < 100000 && !s->dead.load(); ++i) std::this_thread::sleep_for(std::chrono::microseconds(20));
    return s->dead.load() ? KA_OK : KA_E_TIMEOUT;
}

// --- references --------------------------------------------------------------
ka_status ka_ref_wrap(ka_system *h, void *d_ptr, uint64_t n, uint64_t capacity, ka_dtype dtype, ka_access access,
                      ka_ref **out) {
    System *s = sys_of(h);
    if (!s) return KA_E_STALE;
    if (!out || dtype != KA_U32 || n > capacity || capacity > 0xFFFFFFFFull || (capacity && !d_ptr))
        return KA_E_ARG;
    if (access < KA_READ || access > KA_READ_WRITE) return KA_E_ARG;
    Ref *r = new Ref;
    r->sys = s;
    r->ptr = d_ptr;
    r->n_host = n;
    r->capacity = capacity;
    r->dtype = dtype;
    r->access = access;
    *out = reinterpret_cast<ka_ref *>(ref_export(r));
    return KA_OK;
}

ka_status ka_ref_alloc(ka_system *h, uint64_t capacity, ka_dtype dtype, ka_ref **out) {
    System *s = sys_of(h);
    if (!s) return KA_E_STALE;
    if (!out || dtype != KA_U32 || capacity > 0xFFFFFFFFull) return KA_E_ARG;
    Ref *r = nullptr;
    const ka_status st = new_owned_ref(s, capacity, &r);
    if (st != KA_OK) return st;
    r->d_count = nullptr;  // caller-filled memory: length = capacity until a stage writes one
    r->n_host = capacity;
    *out = reinterpret_cast<ka_ref *>(ref_export(r));
    return KA_OK;
}

ka_status ka_ref_count(ka_ref *h, uint64_t *n) {
    Ref *r = ref_of(h);
    if (!r) return KA_E_STALE;
    if (!n) return KA_E_ARG;
    if (!r->d_count) {
        *n = r->n_host;
        return KA_OK;
    }
    ka_status st = cuda_status(cudaStreamSynchronize(r->sys->stream));
    if (st != KA_OK) return st;
    uint32_t v = 0;
    st = cuda_status(cudaMemcpy(&v, r->d_count, 4, cudaMemcpyDeviceToHost));
    if (st == KA_OK) *n = v;
    return st;
}

ka_status ka_ref_info(ka_ref *h, void **d_ptr, uint64_t *capacity, int32_t *dtype, int32_t *access) {
    Ref *r = ref_of(h);
    if (!r) return KA_E_STALE;
    if (d_ptr) *d_ptr = r->ptr;
    if (capacity) *capacity = r->capacity;
    if (dtype) *dtype = r->dtype;
    if (access) *access = r->access;
    return KA_OK;
}

ka_status ka_ref_retain(ka_ref *h) {
    std::lock_guard<std::mutex> l(g_refs.mutex());
    Ref *r = g_refs.get_locked(reinterpret_cast<uint64_t>(h));
    if (!r) return KA_E_STALE;
    r->ext.fetch_add(1);
    ref_retain(r);
    return KA_OK;
}

ka_status ka_ref_release(ka_ref *h) {
    Ref *r = nullptr;
    {
        std::lock_guard<std::mutex> l(g_refs.mutex());
        r = g_refs.get_locked(reinterpret_cast<uint64_t>(h));
        if (!r) return KA_E_STALE;
        // the last external holder makes the handle stale
        if (r->ext.fetch_sub(1) == 1) g_refs.remove_locked(reinterpret_cast<uint64_t>(h));
    }
    ref_drop(r);
    return KA_OK;
}

ka_status ka_ref_serialize(const ka_ref *, void *, uint64_t, uint64_t *written) {
    if (written) *written = 0;
    return KA_E_NOT_SERIALIZABLE;
}

// --- actors ------------------------------------------------------------------
ka_status ka_spawn_stage(ka_system *h, const ka_stage_desc *d, ka_actor **out) {
    System *s = sys_of(h);
    if (!s) return KA_E_STALE;
    if (!d || !out) return KA_E_ARG;
    StageSpec sp;
    sp.kind = d->kind;
    sp.tile = d->tile;
    if (d->tile.block || d->tile.ipt) {
        const int32_t kernel = d->kind == KA_STAGE_EXSCAN ? KA_KERNEL_SCAN : KA_KERNEL_COMPACT;
        if (!tile_supported_for(kernel, d->tile.block, d->tile.ipt)) return KA_E_ARG;
    }
    switch (d->kind) {
    case KA_STAGE_GENERATE: sp.in_arity = 0; sp.out_arity = 1; break;
    case KA_STAGE_MAP_HASH: sp.in_arity = 1; sp.out_arity = 1; break;
    case KA_STAGE_PREDICATE:
        if (make_pred(d->pred, d->param, &sp.pred) != KA_OK) return KA_E_ARG;
        sp.in_arity = 1;
        sp.out_arity = 2;
        break;
    case KA_STAGE_EXSCAN: sp.in_arity = 2; sp.out_arity = 3; break;
    case KA_STAGE_SCATTER: sp.in_arity = 3; sp.out_arity = 1; break;
    case KA_STAGE_COMPACT:
        if (make_pred(d->pred, d->param, &sp.pred) != KA_OK) return KA_E_ARG;
        if (d->xform > KA_XFORM_HASH) return KA_E_ARG;
        sp.mul = d->xform == KA_XFORM_HASH ? kHashMul : 1u;
        sp.in_arity = 1;
        sp.out_arity = 1;
        break;
    case KA_STAGE_PREPARE: sp.in_arity = 2; sp.out_arity = 1; break;
    case KA_STAGE_EMPTY: sp.in_arity = 1; sp.out_arity = 1; break;
    case KA_STAGE_MANDELBROT:
        sp.width = uint32_t(d->pred);
        sp.height = d->xform;
        sp.iters = d->param;
        if (d->pred <= 0 || d->xform == 0 || uint64_t(sp.width) * sp.height > 0xFFFFFFFFull) return KA_E_ARG;
        sp.in_arity = 0;
        sp.out_arity = 1;
        break;
    default: return KA_E_ARG;
    }
    Actor *a = new Actor;
    a->sys = s;
    a->spec = sp;
    a->in_arity = sp.in_arity;
    a->out_arity = sp.out_arity;
    a->stages.push_back(a);
    a->handle = g_actors.add(a);
    *out = reinterpret_cast<ka_actor *>(a->handle);
    return KA_OK;
}

ka_status ka_compose(ka_actor *hb, ka_actor *ha, ka_actor **out) {
    Actor *b = actor_of(hb), *a = actor_of(ha);
    if (!a || !b) return KA_E_STALE;
    if (!out || a->sys != b->sys) return KA_E_ARG;
    if (a->out_arity != b->in_arity) return KA_E_TYPE;
    Actor *c = new Actor;
    c->sys = a->sys;
    c->composite = true;
    c->in_arity = a->in_arity;
    c->out_arity = b->out_arity;
    for (Actor *x : a->stages) {
        x->rc.fetch_add(1);
        c->stages.push_back(x);
    }
    for (Actor *x : b->stages) {
        x->rc.fetch_add(1);
        c->stages.push_back(x);
    }
    c->handle = g_actors.add(c);
    *out = reinterpret_cast<ka_actor *>(c->handle);
    return KA_OK;
}

ka_status ka_actor_arity(ka_actor *h, int32_t *in_refs, int32_t *out_refs) {
    Actor *a = actor_of(h);
    if (!a) return KA_E_STALE;
    if (in_refs) *in_refs = a->in_arity;
    if (out_refs) *out_refs = a->out_arity;
    return KA_OK;
}

ka_status ka_actor_release(ka_actor *h) {
    Actor *a = g_actors.remove(reinterpret_cast<uint64_t>(h));
    if (!a) return KA_E_STALE;
    actor_drop(a);
    return KA_OK;
}

ka_status ka_debug_fail_stage(ka_actor *h, int32_t fail_after) {
    Actor *a = actor_of(h);
    if (!a) return KA_E_STALE;
    if (a->composite) return KA_E_ARG;
    a->processed.store(0);
    a->fail_after.store(fail_after);
    return KA_OK;
}

// --- messages ----------------------------------------------------------------
ka_status ka_request(ka_actor *h, const ka_msg *in, ka_request_h **out) {
    Actor *c = actor_of(h);
    if (!c) return KA_E_STALE;
    if (!in || !out) return KA_E_ARG;
    System *s = c->sys;
    if (s->stop.load() || s->dead.load()) return KA_E_CLOSED;
    if (in->n_refs > KA_MSG_MAX_REFS) return KA_E_ARG;
    Request *r = request_new(s);
    if (!r) return KA_E_OOM;
    Msg *m = &r->msg;
    m->n_refs = 0;
    m->seed = in->seed;
    m->gen_n = in->gen_n;
    // resolve references (the request holds its own)
    {
        std::lock_guard<std::mutex> l(g_refs.mutex());
        for (uint32_t i = 0; i < in->n_refs; ++i) {
            Ref *x = g_refs.get_locked(reinterpret_cast<uint64_t>(in->refs[i]));
            if (!x) {
                release_msg_refs(m);
                request_recycle(r);
                return KA_E_STALE;
            }
            ref_retain(x);
            m->refs[m->n_refs++] = x;
        }
    }
    r->h_out = in->h_out;
    r->h_out_cap = in->h_out_cap;
    r->debug_check = s->debug;
    // value mode in: the first stage's input is uploaded from host memory
    if (in->h_in) {
        if (m->n_refs > 0) {
            ref_drop(m->refs[0]);
        } else {
            m->n_refs = 1;
        }
        Ref *u = nullptr;
        ka_status st = new_owned_ref(s, in->h_n, &u);
        if (st == KA_OK) {
            u->n_host = in->h_n;
            u->d_count = nullptr;
            if (in->h_n)
                st = cuda_status(cudaMemcpyAsync(u->ptr, in->h_in, in->h_n * 4, cudaMemcpyHostToDevice, s->stream));
        }
        if (st != KA_OK) {
            if (u) ref_drop(u);
            m->refs[0] = nullptr;
            for (int j = 1; j < m->n_refs; ++j) ref_drop(m->refs[j]);
            m->n_refs = 0;
            request_recycle(r);
            return st;
        }
        m->refs[0] = u;
    }
    for (Actor *a : c->stages) {
        a->rc.fetch_add(1);
        r->stages.push_back(a);
    }
    m->req = r;
    m->stage = 0;
    s->inflight.fetch_add(1);
    // Inline dispatch: while no thread runs actors and the next actor has no
    // mail queued, run the stages here; the rest goes through the mailboxes.
    // The handle is registered after the first launches: only the caller
    // uses it, and the request stays alive on the caller's hold until it
    // receives.
    Actor *a = r->stages[0];
    if (!s->kill_requested.load() && s->dispatch_mu.try_lock()) {
        while (a && actor_idle(a)) a = process(s, a, m);
        s->dispatch_mu.unlock();
    }
    r->handle = g_requests.add(r);
    *out = reinterpret_cast<ka_request_h *>(r->handle);
    if (a) post(a, m);
    return KA_OK;
}

ka_status ka_receive(ka_request_h *h, int64_t timeout_ns, ka_msg *out) {
    Request *r = g_requests.get(reinterpret_cast<uint64_t>(h));
    if (!r) return KA_E_STALE;
    // Spin for a while (no wake-up latency for results that come soon),
    // polling the request's event once it is recorded and fulfilling the
    // request on this thread if it claims it first; then block.
    if (!r->done.load(std::memory_order_acquire)) {
        System *s = r->sys;
        r->waiting.store(true, std::memory_order_release);
        const auto t0 = std::chrono::steady_clock::now();
        // (a time-out shorter than the spin window bounds the spin too)
        const auto spin = timeout_ns >= 0 && timeout_ns < int64_t(kReceiveSpinUs) * 1000
                              ? std::chrono::nanoseconds(timeout_ns)
                              : std::chrono::nanoseconds(int64_t(kReceiveSpinUs) * 1000);
        while (!r->done.load(std::memory_order_acquire) && std::chrono::steady_clock::now() - t0 < spin) {
            if (!r->recorded.load(std::memory_order_acquire) || is_claimed(r)) continue;
            if (r->tagged) {
                // the publish kernel's tag: every stage has finished (a failed
                // launch never stores it; the completion thread reports that)
                if (__atomic_load_n(&r->pinned_count[2], __ATOMIC_ACQUIRE) != r->seq) continue;
                if (try_claim(r, current_use(r))) finalize(s, r, KA_OK);
                continue;
            }
            const cudaError_t q = cudaEventQuery(r->event);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) cudaGetLastError();
            if (try_claim(r, current_use(r))) finalize(s, r, cuda_status(q));
        }
        r->waiting.store(false, std::memory_order_release);
        if (!r->done.load(std::memory_order_acquire)) {
            r->blocked.store(true, std::memory_order_seq_cst);
            kick_completer(s);  // it fulfils r from here
            std::unique_lock<std::mutex> l(r->mu);
            if (timeout_ns < 0) {
                r->cv.wait(l, [&] { return r->done.load(); });
            } else {
                const auto left = std::chrono::nanoseconds(timeout_ns) - (std::chrono::steady_clock::now() - t0);
                if (!r->cv.wait_for(l, left, [&] { return r->done.load(); })) return KA_E_TIMEOUT;
            }
        }
    }
    g_requests.remove(reinterpret_cast<uint64_t>(h));
    const ka_status st = r->status;
    if (out) {
        out->status = st;
        out->count = st == KA_OK ? r->count : 0;
        out->n_refs = 0;
        for (int i = 0; i < KA_MSG_MAX_REFS; ++i) out->refs[i] = nullptr;
        if (st == KA_OK) {
            for (Ref *x : r->result) {
                if (out->n_refs < KA_MSG_MAX_REFS) {
                    out->refs[out->n_refs++] = reinterpret_cast<ka_ref *>(ref_export(x));
                } else {
                    ref_drop(x);
                }
            }
            r->result.clear();
        }
    }
    request_unhold(r);
    return st;
}

}  // extern "C"
