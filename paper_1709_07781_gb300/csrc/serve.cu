// Serving loop: compaction pipelines arriving over time.
//
// Each request is a pipeline of 1-4 compaction stages (a hash map is the stage
// "keep everything, hash first") over a fresh seeded array of n entries. The
// loop replays the requests' arrival times against the wall clock, admits a
// request once the device memory it needs (one buffer of n entries: every
// stage compacts in place, the live length travelling in a device word)
// fits the budget, and reports when each result was ready on the host.
//
// Mode 0, continuous batching. Admitted requests are grouped into ticks. A
// tick is one batched generate launch for its requests' inputs, then one
// batched compaction launch per stage depth (all first stages, then all
// second stages, ...), each a single persistent kernel over every item of
// that depth, then one copy of the tick's counts to the host. Up to kTicks
// ticks are in flight: while the GPU runs one, the host admits the requests
// that have arrived since and queues the next, so new requests join without
// waiting for the running ones to finish and their work overlaps on the
// device. Descriptor tables are double-buffered per tick slot.
//
// In mode 0 each tick slot's sequence is captured once per depth as a CUDA
// graph (tables of kTickItems entries, the unused ones empty) and a tick is
// one graph launch; mode 2 issues the same ticks as separate calls.
//
// Mode 1, plain launches: the same admission, but every request is issued on
// arrival as its own launches (generate, then one compaction per stage).
//
// Both modes run on one stream of the system's device and allocate request
// buffers from their own stream-ordered memory pool.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ka_internal.h"

namespace ka {
namespace {

using Clock = std::chrono::steady_clock;

constexpr uint32_t kTickItems = 1024;        // requests per tick at most
constexpr uint64_t kTickElems = 1ull << 28;  // input entries per tick at most
constexpr int kTicks = 2;                    // ticks in flight at most
constexpr int kDepth = 4;                    // stages per request at most
constexpr uint64_t kPoolReserve = 4ull << 30;  // pool memory reserved at set-up (at most the budget)

uint64_t bytes_for(uint32_t n) { return n ? (uint64_t(n) * 4 + 255) / 256 * 256 : 256; }

struct Tick {
    char *dev = nullptr;   // gen items | stage tables | counts | error word
    char *host = nullptr;      // pinned, host-mapped mirror of the same layout
    char *host_dev = nullptr;  // the mirror's device address
    cudaEvent_t ev = nullptr;
    std::vector<uint32_t> reqs;  // request indices, tick position = vector index
    uint32_t depth = 0;          // stages of the deepest request
    bool busy = false;
    bool lone = false;           // issued as one request's plain launches (errors in ws_plain)
    // graph mode: the tick's whole sequence for each depth, captured once;
    // host table entries past the current tick are kept zero (empty items)
    cudaGraphExec_t graph[kDepth] = {nullptr, nullptr, nullptr, nullptr};
    uint32_t hw_gen = 0, hw_items[kDepth] = {0, 0, 0, 0};  // entries written by the previous tick

    static constexpr size_t kGenOff = 0;
    static constexpr size_t kItemsOff = kGenOff + sizeof(ka_gen_item) * kTickItems;
    static constexpr size_t kCntOff = kItemsOff + sizeof(ka_batch_item) * kTickItems * kDepth;
    static constexpr size_t kErrOff = kCntOff + sizeof(uint32_t) * kTickItems * kDepth;
    static constexpr size_t kBytes = kErrOff + 256;

    ka_gen_item *gen(char *base) const { return reinterpret_cast<ka_gen_item *>(base + kGenOff); }
    ka_batch_item *items(char *base, int s) const {
        return reinterpret_cast<ka_batch_item *>(base + kItemsOff) + size_t(s) * kTickItems;
    }
    uint32_t *cnt(char *base, int s) const {
        return reinterpret_cast<uint32_t *>(base + kCntOff) + size_t(s) * kTickItems;
    }
    uint32_t *err(char *base) const { return reinterpret_cast<uint32_t *>(base + kErrOff); }
};

struct Run {
    const ka_serve_request *reqs = nullptr;
    uint32_t n = 0;
    ka_serve_result *res = nullptr;
    ka_serve_stats st{};
    uint32_t mode = 0;
    uint64_t budget = 0;
    uint32_t max_inflight = 0;
    double scale = 1.0;
    ka_tile tile{0, 0};

    cudaStream_t stream = nullptr;
    cudaStream_t readback = nullptr;
    cudaMemPool_t pool = nullptr;
    Clock::time_point t0;

    std::vector<uint32_t> order;  // request indices by arrival time
    size_t next = 0;
    std::deque<uint32_t> waiting;
    std::vector<void *> buf;  // per request
    uint64_t in_use = 0;
    uint32_t inflight = 0;
    uint32_t finished = 0;
    double last_done = 0;

    // batched mode
    Tick ticks[kTicks];
    int tick_head = 0;  // oldest tick in flight
    int tick_used = 0;
    void *ws_gen = nullptr, *ws_cmp = nullptr;
    uint64_t ws_gen_bytes = 0, ws_cmp_bytes = 0;
    ka_tile batch_tile{0, 0};
    uint32_t grid_max = 0;  // blocks of a full persistent launch
    bool graphs = false;    // ticks replay captured graphs
    bool batch_lone = false;  // a tick of one request is batched too (else plain launches)

    // plain mode
    struct Slot {
        uint32_t req;
        cudaEvent_t ev;
        uint32_t idx;
    };
    std::deque<Slot> plain_inflight;
    std::vector<uint32_t> plain_free;
    uint32_t *d_cnt = nullptr;  // kDepth words per slot
    uint32_t *h_cnt = nullptr;      // final count per slot (host-mapped)
    uint32_t *h_cnt_dev = nullptr;  // its device address
    std::vector<cudaEvent_t> plain_ev;
    void *ws_plain = nullptr;
    uint64_t ws_plain_bytes = 0;

    // value-mode read-backs in flight on `readback` (oldest first), each with
    // the event recorded after its copy; and events free for reuse
    struct Readback {
        uint32_t req;
        cudaEvent_t ev;
    };
    std::deque<Readback> rb_pending;
    std::vector<cudaEvent_t> rb_free;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
    double arrival(uint32_t r) const { return reqs[r].arrival_s * scale; }
};

ka_status check_request(const ka_serve_request &q) {
    if (q.n_stages < 1 || q.n_stages > uint32_t(kDepth)) return KA_E_ARG;
    for (uint32_t s = 0; s < q.n_stages; ++s) {
        PredDev p;
        if (make_pred(q.stages[s].pred, q.stages[s].param, &p) != KA_OK) return KA_E_ARG;
        if (q.stages[s].xform != KA_XFORM_NONE && q.stages[s].xform != KA_XFORM_HASH) return KA_E_ARG;
    }
    return KA_OK;
}

// Request r is complete: its result (and in value mode its data) is on the host.
void mark_done(Run &R, uint32_t r) {
    ka_serve_result &o = R.res[r];
    o.done_s = R.now();
    R.last_done = o.done_s;
    if (o.status == KA_OK) R.st.elements += R.reqs[r].n;
    R.finished += 1;
}

// Read-backs whose copies have landed complete their requests, in order.
ka_status poll_readbacks(Run &R) {
    while (!R.rb_pending.empty()) {
        const Run::Readback rb = R.rb_pending.front();
        const cudaError_t e = cudaEventQuery(rb.ev);
        if (e == cudaErrorNotReady) break;
        R.rb_pending.pop_front();
        R.rb_free.push_back(rb.ev);
        if (e != cudaSuccess) R.res[rb.req].status = cuda_status(e);
        mark_done(R, rb.req);
    }
    return KA_OK;
}

// Marks request r finished with status s and returns its buffer to the pool.
// In value mode the data is copied out on the read-back stream first: the
// buffer is freed on that stream after the copy, and the request completes
// when poll_readbacks sees the copy done, so the loop never waits for it.
void finish(Run &R, uint32_t r, uint32_t count, ka_status s) {
    ka_serve_result &o = R.res[r];
    const ka_serve_request &q = R.reqs[r];
    o.count = count;
    o.status = s;
    if (s == KA_OK && q.h_out && R.buf[r]) {
        const uint64_t m = std::min<uint64_t>(count, q.h_out_cap);
        if (m) {
            cudaEvent_t ev = nullptr;
            if (!R.rb_free.empty()) {
                ev = R.rb_free.back();
                R.rb_free.pop_back();
            }
            cudaError_t e = ev ? cudaSuccess : cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaMemcpyAsync(q.h_out, R.buf[r], m * 4, cudaMemcpyDeviceToHost, R.readback);
            if (e == cudaSuccess) e = cudaEventRecord(ev, R.readback);
            if (e == cudaSuccess) {
                cudaFreeAsync(R.buf[r], R.readback);  // after the copy, in the read-back stream's order
                R.buf[r] = nullptr;
                R.in_use -= bytes_for(q.n);
                R.inflight -= 1;
                R.rb_pending.push_back({r, ev});
                return;
            }
            if (ev) R.rb_free.push_back(ev);
            o.status = cuda_status(e);
            cudaStreamSynchronize(R.readback);  // the buffer may still be read: wait before freeing it
        }
    }
    if (R.buf[r]) {
        const double t_free = R.now();
        cudaFreeAsync(R.buf[r], R.stream);
        R.st.max_free_s = std::max(R.st.max_free_s, R.now() - t_free);
        R.buf[r] = nullptr;
        R.in_use -= bytes_for(q.n);
        R.inflight -= 1;
    }
    mark_done(R, r);
}

// Admits the request at the head of the queue if the budget and the in-flight
// limit allow: allocates its buffer. Returns false if it has to wait.
bool admit_head(Run &R, uint32_t *out) {
    if (R.waiting.empty() || R.inflight >= R.max_inflight) return false;
    const uint32_t r = R.waiting.front();
    const uint64_t b = bytes_for(R.reqs[r].n);
    if (R.in_use + b > R.budget) return false;
    void *p = nullptr;
    const double t_alloc = R.now();
    const cudaError_t ea = cudaMallocFromPoolAsync(&p, b, R.pool, R.stream);
    R.st.max_alloc_s = std::max(R.st.max_alloc_s, R.now() - t_alloc);
    if (ea != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    R.waiting.pop_front();
    R.buf[r] = p;
    R.in_use += b;
    R.inflight += 1;
    R.st.peak_bytes = std::max(R.st.peak_bytes, R.in_use);
    R.st.max_inflight_seen = std::max(R.st.max_inflight_seen, R.inflight);
    R.res[r].admit_s = R.now();
    *out = r;
    return true;
}

// ----------------------------------------------------------------- batched mode
// The tick's per-stage counts and the batch workspace's error word, stored
// into the tick's host-mapped mirror by one small launch.
ka_status publish_counts(Run &R, Tick &T, uint32_t depth) {
    return launch_publish(T.cnt(T.dev, 0), kTickItems * depth, 0, &static_cast<WsHeader *>(R.ws_cmp)->error,
                          T.cnt(T.host_dev, 0), T.err(T.host_dev), R.stream);
}

ka_status issue_tick_launches(Run &R, bool *issued);

// One tick's launches, as one NVTX range on the serving thread.
ka_status issue_tick(Run &R, bool *issued) {
    *issued = false;
    if (R.tick_used == kTicks || R.waiting.empty()) return KA_OK;
    nvtxRangePushA("ka serve: tick");
    const ka_status s = issue_tick_launches(R, issued);
    nvtxRangePop();
    return s;
}

ka_status issue_tick_launches(Run &R, bool *issued) {
    Tick &T = R.ticks[(R.tick_head + R.tick_used) % kTicks];
    T.reqs.clear();
    T.depth = 0;
    uint64_t elems = 0;
    uint32_t r;
    while (T.reqs.size() < kTickItems && !R.waiting.empty() &&
           (T.reqs.empty() || elems + R.reqs[R.waiting.front()].n <= kTickElems) && admit_head(R, &r)) {
        T.reqs.push_back(r);
        elems += R.reqs[r].n;
        T.depth = std::max(T.depth, R.reqs[r].n_stages);
    }
    if (T.reqs.empty()) return KA_OK;
    const uint32_t k = uint32_t(T.reqs.size());
    T.lone = k == 1 && !R.batch_lone;
    if (T.lone) {
        // one request: its plain launch sequence into the tick's count table
        const ka_serve_request &q = R.reqs[T.reqs[0]];
        uint32_t *b = static_cast<uint32_t *>(R.buf[T.reqs[0]]);
        cudaStream_t st = R.stream;
        ka_status s = launch_generate(b, q.n, q.seed, nullptr, st);
        R.st.launches += 1;
        for (uint32_t d = 0; d < q.n_stages && s == KA_OK; ++d) {
            CompactLaunch L;
            s = make_pred(q.stages[d].pred, q.stages[d].param, &L.pred);
            if (s != KA_OK) break;
            L.in = b;
            L.out = b;
            L.n_ptr = d ? T.cnt(T.dev, int(d) - 1) : nullptr;
            L.count = T.cnt(T.dev, int(d));
            L.n = q.n;
            L.mul = q.stages[d].xform == KA_XFORM_HASH ? kHashMul : 1u;
            L.ws = R.ws_plain;
            L.ws_bytes = R.ws_plain_bytes;
            L.tile = resolve_tile(KA_KERNEL_COMPACT, q.n, nullptr);
            s = launch_compact(L, st);
            R.st.launches += 1;
        }
        if (s == KA_OK)
            s = launch_publish(T.cnt(T.dev, 0), kTickItems * T.depth, 0, &static_cast<WsHeader *>(R.ws_plain)->error,
                               T.cnt(T.host_dev, 0), T.err(T.host_dev), st);
        R.st.launches += 1;
        if (s == KA_OK) s = cuda_status(cudaEventRecord(T.ev, st));
        if (s != KA_OK) return s;
        T.busy = true;
        R.tick_used += 1;
        R.st.iterations += 1;
        R.st.lone_ticks += 1;
        *issued = true;
        return KA_OK;
    }
    uint32_t per_stage[kDepth] = {0, 0, 0, 0};
    uint64_t tiles[kDepth] = {0, 0, 0, 0};  // tiles of each stage launch: no more blocks than tiles
    const uint32_t te = R.batch_tile.block * R.batch_tile.ipt;
    for (uint32_t i = 0; i < k; ++i) {
        const ka_serve_request &q = R.reqs[T.reqs[i]];
        uint32_t *b = static_cast<uint32_t *>(R.buf[T.reqs[i]]);
        T.gen(T.host)[i] = ka_gen_item{b, q.seed, q.n, 0};
        for (uint32_t s = 0; s < q.n_stages; ++s) {
            ka_batch_item &it = T.items(T.host, int(s))[per_stage[s]];
            it.in = b;
            it.out = b;
            it.n_ptr = s ? T.cnt(T.dev, int(s) - 1) + i : nullptr;
            it.count = T.cnt(T.dev, int(s)) + i;
            it.n = q.n;
            it.pred = q.stages[s].pred;
            it.param = q.stages[s].param;
            it.xform = q.stages[s].xform;
            per_stage[s] += 1;
            tiles[s] += (uint64_t(q.n) + te - 1) / te;
        }
    }
    cudaStream_t st = R.stream;
    if (R.graphs) {
        // zero the entries the previous tick used beyond this one's, then replay
        if (T.hw_gen > k) std::memset(T.gen(T.host) + k, 0, sizeof(ka_gen_item) * (T.hw_gen - k));
        T.hw_gen = k;
        for (uint32_t d = 0; d < T.depth; ++d) {
            if (T.hw_items[d] > per_stage[d])
                std::memset(T.items(T.host, int(d)) + per_stage[d], 0,
                            sizeof(ka_batch_item) * (T.hw_items[d] - per_stage[d]));
            T.hw_items[d] = per_stage[d];
        }
        ka_status s = cuda_status(cudaGraphLaunch(T.graph[T.depth - 1], st));
        R.st.launches += 2 + 2 * T.depth;
        R.st.graph_launches += 1;
        if (s == KA_OK) s = cuda_status(cudaEventRecord(T.ev, st));
        if (s != KA_OK) return s;
        T.busy = true;
        R.tick_used += 1;
        R.st.iterations += 1;
        *issued = true;
        return KA_OK;
    }
    ka_status s = cuda_status(
        cudaMemcpyAsync(T.gen(T.dev), T.gen(T.host), sizeof(ka_gen_item) * k, cudaMemcpyHostToDevice, st));
    for (uint32_t d = 0; d < T.depth && s == KA_OK; ++d)
        s = cuda_status(cudaMemcpyAsync(T.items(T.dev, int(d)), T.items(T.host, int(d)),
                                        sizeof(ka_batch_item) * per_stage[d], cudaMemcpyHostToDevice, st));
    if (s == KA_OK) s = ka_generate_batch(T.gen(T.dev), k, kTickItems, R.ws_gen, R.ws_gen_bytes, st);
    R.st.launches += 2;
    for (uint32_t d = 0; d < T.depth && s == KA_OK; ++d) {
        const uint32_t grid = uint32_t(std::min<uint64_t>(std::max<uint64_t>(tiles[d], 1), R.grid_max));
        s = ka_compact_batch(T.items(T.dev, int(d)), per_stage[d], kTickItems, R.ws_cmp, R.ws_cmp_bytes,
                             &R.batch_tile, grid, st);
        R.st.launches += 2;
    }
    if (s == KA_OK) {
        s = publish_counts(R, T, T.depth);
        R.st.launches += 1;
    }
    if (s == KA_OK) s = cuda_status(cudaEventRecord(T.ev, st));
    if (s != KA_OK) return s;
    T.busy = true;
    R.tick_used += 1;
    R.st.iterations += 1;
    *issued = true;
    return KA_OK;
}

// The device work of a tick of `depth` stages over full tables (kTickItems
// entries each, the unused ones empty), on the run's stream: what a tick
// graph holds.
ka_status full_tick_ops(Run &R, Tick &T, uint32_t depth) {
    cudaStream_t st = R.stream;
    ka_status s = cuda_status(cudaMemcpyAsync(T.gen(T.dev), T.gen(T.host), sizeof(ka_gen_item) * kTickItems,
                                              cudaMemcpyHostToDevice, st));
    for (uint32_t d = 0; d < depth && s == KA_OK; ++d)
        s = cuda_status(cudaMemcpyAsync(T.items(T.dev, int(d)), T.items(T.host, int(d)),
                                        sizeof(ka_batch_item) * kTickItems, cudaMemcpyHostToDevice, st));
    if (s == KA_OK) s = ka_generate_batch(T.gen(T.dev), kTickItems, kTickItems, R.ws_gen, R.ws_gen_bytes, st);
    for (uint32_t d = 0; d < depth && s == KA_OK; ++d)
        s = ka_compact_batch(T.items(T.dev, int(d)), kTickItems, kTickItems, R.ws_cmp, R.ws_cmp_bytes, &R.batch_tile,
                             0, st);
    if (s == KA_OK) s = publish_counts(R, T, depth);
    return s;
}

// Captures every tick slot's graph for depths 1..kDepth. The kernels run
// once first outside any capture (their launch set-up happens then). On any
// failure the run keeps issuing ticks directly.
void build_graphs(Run &R) {
    R.graphs = false;
    if (full_tick_ops(R, R.ticks[0], kDepth) != KA_OK || cudaStreamSynchronize(R.stream) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    for (Tick &T : R.ticks) {
        for (uint32_t d = 1; d <= uint32_t(kDepth); ++d) {
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(R.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                cudaGetLastError();
                return;
            }
            const ka_status s = full_tick_ops(R, T, d);
            const cudaError_t e = cudaStreamEndCapture(R.stream, &g);
            if (s != KA_OK || e != cudaSuccess || !g ||
                cudaGraphInstantiate(&T.graph[d - 1], g, 0) != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                return;
            }
            cudaGraphDestroy(g);
        }
    }
    R.graphs = true;
}

ka_status poll_ticks(Run &R, bool *progressed) {
    *progressed = false;
    while (R.tick_used) {
        Tick &T = R.ticks[R.tick_head];
        const cudaError_t q = cudaEventQuery(T.ev);
        if (q == cudaErrorNotReady) return KA_OK;
        if (q != cudaSuccess) return cuda_status(q);
        const uint32_t err = *T.err(T.host);
        for (uint32_t i = 0; i < T.reqs.size(); ++i) {
            const uint32_t r = T.reqs[i];
            const uint32_t last = R.reqs[r].n_stages - 1;
            finish(R, r, T.cnt(T.host, int(last))[i], err ? -int32_t(err) : KA_OK);
        }
        if (err) {  // clear the error so later ticks report only their own
            ka_status s = T.lone ? ka_workspace_init(R.ws_plain, R.ws_plain_bytes, R.stream)
                                 : ka_workspace_init(R.ws_cmp, R.ws_cmp_bytes, R.stream);
            if (s != KA_OK) return s;
        }
        T.busy = false;
        R.tick_head = (R.tick_head + 1) % kTicks;
        R.tick_used -= 1;
        *progressed = true;
    }
    return KA_OK;
}

// ------------------------------------------------------------------- plain mode
ka_status issue_plain(Run &R, bool *issued) {
    *issued = false;
    while (!R.plain_free.empty() && !R.waiting.empty()) {
        uint32_t r;
        if (!admit_head(R, &r)) return KA_OK;
        const uint32_t slot = R.plain_free.back();
        R.plain_free.pop_back();
        const ka_serve_request &q = R.reqs[r];
        uint32_t *b = static_cast<uint32_t *>(R.buf[r]);
        uint32_t *cnt = R.d_cnt + size_t(slot) * kDepth;
        ka_status s = launch_generate(b, q.n, q.seed, nullptr, R.stream);
        R.st.launches += 1;
        for (uint32_t d = 0; d < q.n_stages && s == KA_OK; ++d) {
            CompactLaunch L;
            s = make_pred(q.stages[d].pred, q.stages[d].param, &L.pred);
            if (s != KA_OK) break;
            L.in = b;
            L.out = b;
            L.n_ptr = d ? cnt + d - 1 : nullptr;
            L.count = cnt + d;
            L.n = q.n;
            L.mul = q.stages[d].xform == KA_XFORM_HASH ? kHashMul : 1u;
            L.ws = R.ws_plain;
            L.ws_bytes = R.ws_plain_bytes;
            L.tile = resolve_tile(KA_KERNEL_COMPACT, q.n, R.tile.block ? &R.tile : nullptr);
            s = launch_compact(L, R.stream);
            R.st.launches += 1;
        }
        if (s == KA_OK)
            s = launch_publish(cnt + q.n_stages - 1, 1, 0, nullptr, R.h_cnt_dev + slot, nullptr, R.stream);
        if (s == KA_OK) s = cuda_status(cudaEventRecord(R.plain_ev[slot], R.stream));
        if (s != KA_OK) return s;
        R.plain_inflight.push_back(Run::Slot{r, R.plain_ev[slot], slot});
        R.st.iterations += 1;
        *issued = true;
    }
    return KA_OK;
}

ka_status poll_plain(Run &R, bool *progressed) {
    *progressed = false;
    while (!R.plain_inflight.empty()) {
        const Run::Slot sl = R.plain_inflight.front();
        const cudaError_t q = cudaEventQuery(sl.ev);
        if (q == cudaErrorNotReady) return KA_OK;
        if (q != cudaSuccess) return cuda_status(q);
        R.plain_inflight.pop_front();
        finish(R, sl.req, R.h_cnt[sl.idx], KA_OK);
        R.plain_free.push_back(sl.idx);
        *progressed = true;
    }
    return KA_OK;
}

// ----------------------------------------------------------------- set-up
ka_status setup(Run &R, uint32_t max_n) {
    ka_status s = cuda_status(cudaStreamCreateWithFlags(&R.stream, cudaStreamNonBlocking));
    if (s == KA_OK) s = cuda_status(cudaStreamCreateWithFlags(&R.readback, cudaStreamNonBlocking));
    if (s != KA_OK) return s;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    s = cuda_status(cudaMemPoolCreate(&R.pool, &props));
    if (s != KA_OK) return s;
    uint64_t keep = ~0ull;  // keep freed memory in the pool for the next requests
    cudaMemPoolSetAttribute(R.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    // Reserve the pool's memory before the loop starts (allocated and freed
    // here, kept by the release threshold above): growing a pool maps new
    // memory, and inside the loop that took milliseconds (up to 62 ms once a
    // backlog had built up), holding up the loop's other stream calls
    // (frees, polls) meanwhile and so lengthening the backlog that caused it.
    {
        const uint64_t reserve = std::min<uint64_t>(R.budget, kPoolReserve);
        void *p = nullptr;
        if (reserve && cudaMallocFromPoolAsync(&p, reserve, R.pool, R.stream) == cudaSuccess)
            cudaFreeAsync(p, R.stream);
        else
            cudaGetLastError();  // no reservation: the pool grows on demand
    }
    if (R.mode != 1) {
        R.batch_tile = resolve_tile(KA_KERNEL_BATCH, kBatchTileKey, R.tile.block ? &R.tile : nullptr);
        R.grid_max = uint32_t(device_info().sm_count) * 8;
        s = ka_batch_workspace_size(kTickItems, 0, nullptr, &R.ws_gen_bytes);
        if (s == KA_OK)
            s = ka_batch_workspace_size(kTickItems, std::max<uint64_t>(kTickElems, max_n),
                                        R.tile.block ? &R.tile : nullptr, &R.ws_cmp_bytes);
        if (s == KA_OK) s = cuda_status(cudaMalloc(&R.ws_gen, R.ws_gen_bytes));
        if (s == KA_OK) s = cuda_status(cudaMalloc(&R.ws_cmp, R.ws_cmp_bytes));
        if (s == KA_OK) s = ka_workspace_init(R.ws_gen, R.ws_gen_bytes, R.stream);
        if (s == KA_OK) s = ka_workspace_init(R.ws_cmp, R.ws_cmp_bytes, R.stream);
        // ticks of one request run the plain compaction on a workspace of their own
        if (s == KA_OK) s = ka_workspace_size(max_n ? max_n : 1, nullptr, &R.ws_plain_bytes);
        if (s == KA_OK) s = cuda_status(cudaMalloc(&R.ws_plain, R.ws_plain_bytes));
        if (s == KA_OK) s = ka_workspace_init(R.ws_plain, R.ws_plain_bytes, R.stream);
        for (int i = 0; i < kTicks && s == KA_OK; ++i) {
            s = cuda_status(cudaMalloc(&R.ticks[i].dev, Tick::kBytes));
            if (s == KA_OK) s = cuda_status(cudaHostAlloc(&R.ticks[i].host, Tick::kBytes, cudaHostAllocMapped));
            if (s == KA_OK)
                s = cuda_status(
                    cudaHostGetDevicePointer(reinterpret_cast<void **>(&R.ticks[i].host_dev), R.ticks[i].host, 0));
            if (s == KA_OK) s = cuda_status(cudaEventCreateWithFlags(&R.ticks[i].ev, cudaEventDisableTiming));
            if (s == KA_OK) s = cuda_status(cudaMemsetAsync(R.ticks[i].dev, 0, Tick::kBytes, R.stream));
            if (s == KA_OK) std::memset(R.ticks[i].host, 0, Tick::kBytes);  // zero entries are empty items
        }
        if (s == KA_OK && R.mode == 0) build_graphs(R);
    } else {
        const uint32_t slots = R.max_inflight;
        s = ka_workspace_size(max_n ? max_n : 1, nullptr, &R.ws_plain_bytes);
        if (s == KA_OK) s = cuda_status(cudaMalloc(&R.ws_plain, R.ws_plain_bytes));
        if (s == KA_OK) s = ka_workspace_init(R.ws_plain, R.ws_plain_bytes, R.stream);
        if (s == KA_OK) s = cuda_status(cudaMalloc(&R.d_cnt, sizeof(uint32_t) * kDepth * slots));
        if (s == KA_OK) s = cuda_status(cudaHostAlloc(&R.h_cnt, sizeof(uint32_t) * slots, cudaHostAllocMapped));
        if (s == KA_OK) s = cuda_status(cudaHostGetDevicePointer(reinterpret_cast<void **>(&R.h_cnt_dev), R.h_cnt, 0));
        R.plain_ev.assign(slots, nullptr);
        for (uint32_t i = 0; i < slots && s == KA_OK; ++i) {
            s = cuda_status(cudaEventCreateWithFlags(&R.plain_ev[i], cudaEventDisableTiming));
            R.plain_free.push_back(slots - 1 - i);
        }
    }
    if (s == KA_OK) s = cuda_status(cudaStreamSynchronize(R.stream));
    return s;
}

void teardown(Run &R) {
    if (R.stream) cudaStreamSynchronize(R.stream);
    if (R.readback) cudaStreamSynchronize(R.readback);
    for (const Run::Readback &rb : R.rb_pending) cudaEventDestroy(rb.ev);
    for (cudaEvent_t e : R.rb_free) cudaEventDestroy(e);
    for (void *&p : R.buf)
        if (p) {
            cudaFreeAsync(p, R.stream);
            p = nullptr;
        }
    if (R.stream) cudaStreamSynchronize(R.stream);
    for (Tick &T : R.ticks) {
        for (cudaGraphExec_t &g : T.graph)
            if (g) cudaGraphExecDestroy(g);
        if (T.dev) cudaFree(T.dev);
        if (T.host) cudaFreeHost(T.host);
        if (T.ev) cudaEventDestroy(T.ev);
    }
    for (cudaEvent_t e : R.plain_ev)
        if (e) cudaEventDestroy(e);
    if (R.d_cnt) cudaFree(R.d_cnt);
    if (R.h_cnt) cudaFreeHost(R.h_cnt);
    if (R.ws_gen) cudaFree(R.ws_gen);
    if (R.ws_cmp) cudaFree(R.ws_cmp);
    if (R.ws_plain) cudaFree(R.ws_plain);
    if (R.pool) cudaMemPoolDestroy(R.pool);
    if (R.readback) cudaStreamDestroy(R.readback);
    if (R.stream) cudaStreamDestroy(R.stream);
}

}  // namespace
}  // namespace ka

using namespace ka;

extern "C" ka_status ka_serve_run(ka_system *sys, const ka_serve_request *reqs, uint32_t n_reqs,
                                  const ka_serve_options *opt, ka_serve_result *results, ka_serve_stats *stats) {
    if (!sys || !opt || (n_reqs && (!reqs || !results))) return KA_E_ARG;
    if (opt->mode > 2) return KA_E_ARG;
    int device = 0;
    uint64_t sys_budget = 0;
    ka_status s = system_exec_info(sys, &device, &sys_budget);
    if (s != KA_OK) return s;
    s = cuda_status(cudaSetDevice(device));
    if (s != KA_OK) return s;
    if (opt->tile.block || opt->tile.ipt) {
        const int32_t k = opt->mode == 1 ? KA_KERNEL_COMPACT : KA_KERNEL_BATCH;
        if (!tile_supported_for(k, opt->tile.block, opt->tile.ipt)) return KA_E_ARG;
    }
    Run R;
    R.reqs = reqs;
    R.n = n_reqs;
    R.res = results;
    R.mode = opt->mode;
    R.budget = opt->budget_bytes ? opt->budget_bytes : sys_budget;
    R.max_inflight = opt->max_inflight ? opt->max_inflight : 4096;
    R.scale = opt->time_scale > 0 ? opt->time_scale : 1.0;
    R.tile = opt->tile;
    R.batch_lone = (opt->flags & KA_SERVE_BATCH_LONE) != 0;
    R.buf.assign(n_reqs, nullptr);
    R.order.resize(n_reqs);
    uint32_t max_n = 0;
    for (uint32_t i = 0; i < n_reqs; ++i) {
        R.order[i] = i;
        results[i] = ka_serve_result{0, 0, 0, KA_OK};
        max_n = std::max(max_n, reqs[i].n);
    }
    std::stable_sort(R.order.begin(), R.order.end(),
                     [&](uint32_t a, uint32_t b) { return reqs[a].arrival_s < reqs[b].arrival_s; });
    s = setup(R, max_n);
    if (s == KA_OK) {
        R.t0 = Clock::now();
        double step_t0 = 0.0;
        while (R.finished < R.n) {
            const double t = R.now();
            if (step_t0 > 0.0) {
                const double step = t - step_t0;
                R.st.max_step_s = std::max(R.st.max_step_s, step);
                if (step > 1e-3) R.st.slow_steps += 1;
            }
            step_t0 = t;
            while (R.next < R.n && R.arrival(R.order[R.next]) <= t) {
                const uint32_t r = R.order[R.next++];
                const ka_status v = check_request(reqs[r]);
                if (v != KA_OK || bytes_for(reqs[r].n) > R.budget) {
                    results[r].admit_s = t;
                    if (v == KA_OK) R.st.rejected += 1;
                    finish(R, r, 0, v != KA_OK ? v : KA_E_BUDGET);
                    continue;
                }
                R.waiting.push_back(r);
            }
            bool done_some = false, issued = false;
            const double t_poll = R.now();
            s = R.mode != 1 ? poll_ticks(R, &done_some) : poll_plain(R, &done_some);
            if (s == KA_OK) s = poll_readbacks(R);
            const double t_issue = R.now();
            R.st.max_poll_s = std::max(R.st.max_poll_s, t_issue - t_poll);
            if (s == KA_OK) s = R.mode != 1 ? issue_tick(R, &issued) : issue_plain(R, &issued);
            R.st.max_issue_s = std::max(R.st.max_issue_s, R.now() - t_issue);
            if (s != KA_OK) break;
            const bool busy = (R.mode != 1 ? R.tick_used > 0 : !R.plain_inflight.empty()) || !R.rb_pending.empty();
            if (!done_some && !issued) {
                if (!busy && R.waiting.empty() && R.next < R.n) {
                    // Idle until the next arrival: short sleeps while it is more
                    // than half a millisecond away (a sleep may overrun by tens of
                    // microseconds, and a long one by much more when the thread
                    // is descheduled), then spin.
                    const double wait = R.arrival(R.order[R.next]) - R.now();
                    if (wait > 5e-4) std::this_thread::sleep_for(std::chrono::microseconds(200));
                    step_t0 = 0.0;  // an idle wait is not a stall
                } else if (!busy && !R.waiting.empty()) {
                    // the head request cannot be admitted and nothing will free memory
                    const uint32_t r = R.waiting.front();
                    R.waiting.pop_front();
                    results[r].admit_s = R.now();
                    finish(R, r, 0, KA_E_OOM);
                }
            }
        }
        R.st.wall_s = R.last_done;
    }
    teardown(R);
    if (stats) *stats = R.st;
    return s;
}
