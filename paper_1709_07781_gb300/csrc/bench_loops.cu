// Timing loops in native code for the actor-overhead measurements (the
// paper's Sec. 5.2 and 5.3 compare an actor against the same kernel driven
// through the native API, one task after another). Both loops run the same
// kernels on the same stream; only the actor layer differs.
#include <chrono>
#include <vector>

#include "ka_internal.h"

namespace ka {
namespace {

struct Buf {
    uint32_t *ptr = nullptr;
    uint32_t *count = nullptr;  // device count word (nullptr: host length n)
    uint64_t cap = 0;
    uint64_t n = 0;
};

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace
}  // namespace ka

using namespace ka;

extern "C" {

ka_status ka_bench_request_loop(ka_actor *actor, const ka_msg *msg, uint32_t iters, uint32_t inflight,
                                double *seconds, uint64_t *last_count) {
    if (!actor || !msg || !seconds || iters == 0) return KA_E_ARG;
    if (inflight == 0) inflight = 1;
    std::vector<ka_request_h *> ring(inflight, nullptr);
    uint64_t last = 0;
    ka_status first_err = KA_OK;
    auto finish = [&](ka_request_h *q) {
        ka_msg out;
        const ka_status s = ka_receive(q, -1, &out);
        if (s != KA_OK && first_err == KA_OK) first_err = s;
        if (s == KA_OK) {
            last = out.count;
            for (uint32_t i = 0; i < out.n_refs; ++i) ka_ref_release(out.refs[i]);
        }
    };
    const double t0 = now_s();
    for (uint32_t i = 0; i < iters; ++i) {
        ka_request_h *&slot = ring[i % inflight];
        if (slot) finish(slot);
        const ka_status s = ka_request(actor, msg, &slot);
        if (s != KA_OK) return s;
    }
    for (uint32_t i = 0; i < iters && i < inflight; ++i) {
        ka_request_h *&slot = ring[(iters + i) % inflight];
        if (slot) finish(slot);
        slot = nullptr;
    }
    *seconds = now_s() - t0;
    if (last_count) *last_count = last;
    return first_err;
}

ka_status ka_bench_direct_chain(const ka_stage_desc *stages, uint32_t n_stages, const uint32_t *d_in, uint64_t n,
                                uint32_t iters, void *stream, uint32_t flags, double *seconds, uint64_t *last_count) {
    if (!stages || n_stages == 0 || !seconds || iters == 0 || n > 0xFFFFFFFFull) return KA_E_ARG;
    if (flags & ~KA_BENCH_WAIT_TAG) return KA_E_ARG;
    const bool wait_tag = (flags & KA_BENCH_WAIT_TAG) != 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // buffers: one output (+ count word) per stage output, allocated once
    std::vector<void *> allocs;
    auto alloc = [&](uint64_t cap, Buf *b) -> ka_status {
        void *p = nullptr;
        const uint64_t data = (cap * 4 + 255) / 256 * 256;
        if (cudaMalloc(&p, data + 256) != cudaSuccess) return KA_E_OOM;
        allocs.push_back(p);
        b->ptr = static_cast<uint32_t *>(p);
        b->count = reinterpret_cast<uint32_t *>(static_cast<char *>(p) + data);
        b->cap = cap;
        return KA_OK;
    };
    ka_status s = KA_OK;
    void *ws = nullptr;
    const uint64_t ws_bytes = workspace_bytes_for_tiles(tiles_for(n ? n : 1, 512) + 1);
    if (cudaMalloc(&ws, ws_bytes) != cudaSuccess) return KA_E_OOM;
    allocs.push_back(ws);
    s = ka_workspace_init(ws, ws_bytes, st);
    uint32_t *pinned = nullptr, *pinned_dev = nullptr;  // host-mapped result slot, as the actor layer uses
    uint32_t seq = 0;                                     // completion tag of the current run
    cudaEvent_t done = nullptr;
    if (s == KA_OK) s = cuda_status(cudaHostAlloc(&pinned, 16, cudaHostAllocMapped));
    if (s == KA_OK) s = cuda_status(cudaHostGetDevicePointer(reinterpret_cast<void **>(&pinned_dev), pinned, 0));
    if (s == KA_OK && wait_tag) s = cuda_status(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    // plan: per stage, its outputs (same arity conventions as the actor stages)
    std::vector<std::vector<Buf>> outs(n_stages);
    std::vector<Buf> cur;
    Buf in;
    in.ptr = const_cast<uint32_t *>(d_in);
    in.cap = n;
    in.n = n;
    cur.push_back(in);
    std::vector<PredDev> preds(n_stages);
    for (uint32_t i = 0; i < n_stages && s == KA_OK; ++i) {
        const ka_stage_desc &d = stages[i];
        std::vector<Buf> o;
        Buf y;
        switch (d.kind) {
        case KA_STAGE_MAP_HASH:
        case KA_STAGE_COMPACT:
        case KA_STAGE_SCATTER:
            if (cur.empty()) s = KA_E_TYPE;
            if (s == KA_OK) s = alloc(cur[0].cap, &y);
            o.push_back(y);
            break;
        case KA_STAGE_PREDICATE:
            if (cur.size() != 1) s = KA_E_TYPE;
            if (s == KA_OK) s = alloc(cur[0].cap, &y);
            o.push_back(cur[0]);
            o.push_back(y);
            break;
        case KA_STAGE_EXSCAN:
            if (cur.size() != 2) s = KA_E_TYPE;
            if (s == KA_OK) s = alloc(cur[1].cap, &y);
            o = cur;
            o.push_back(y);
            break;
        case KA_STAGE_PREPARE:  // first stage only: d_in = k chunk ids, then k literals
            if (i != 0 || cur.size() != 1) s = KA_E_TYPE;
            if (s == KA_OK) s = alloc(2 * cur[0].cap, &y);
            o.push_back(y);
            break;
        case KA_STAGE_EMPTY: o = cur; break;
        case KA_STAGE_MANDELBROT:
            if (d.pred <= 0 || d.xform == 0) s = KA_E_ARG;
            if (s == KA_OK) s = alloc(uint64_t(d.pred) * d.xform, &y);
            o.push_back(y);
            break;
        default: s = KA_E_UNSUPPORTED;
        }
        if (s == KA_OK && (d.kind == KA_STAGE_PREDICATE || d.kind == KA_STAGE_COMPACT))
            s = make_pred(d.pred, d.param, &preds[i]);
        outs[i] = o;
        cur = o;
    }
    auto len = [](const Buf &b, uint64_t *nn, const uint32_t **np) {
        if (b.count) {
            *nn = b.cap;
            *np = b.count;
        } else {
            *nn = b.n;
            *np = nullptr;
        }
    };
    auto run_once = [&]() -> ka_status {
        std::vector<Buf> c;
        c.push_back(in);
        for (uint32_t i = 0; i < n_stages; ++i) {
            const ka_stage_desc &d = stages[i];
            const std::vector<Buf> &o = outs[i];
            uint64_t nn;
            const uint32_t *np;
            len(c[0], &nn, &np);
            ka_status e = KA_OK;
            switch (d.kind) {
            case KA_STAGE_MAP_HASH: e = launch_map_hash(c[0].ptr, nn, np, o[0].ptr, o[0].count, st); break;
            case KA_STAGE_COMPACT: {
                CompactLaunch L{c[0].ptr, o[0].ptr, np, o[0].count, nn, preds[i],
                                d.xform == KA_XFORM_HASH ? kHashMul : 1u, ws, ws_bytes,
                                resolve_tile(KA_KERNEL_COMPACT, c[0].cap, &d.tile)};
                e = launch_compact(L, st);
                break;
            }
            case KA_STAGE_PREDICATE:
                e = launch_predicate(c[0].ptr, nn, np, preds[i], o[1].ptr, o[1].count, st);
                break;
            case KA_STAGE_EXSCAN: {
                uint64_t fn;
                const uint32_t *fp;
                len(c[1], &fn, &fp);
                e = launch_exclusive_scan(c[1].ptr, fn, fp, o[2].ptr, o[2].count, ws, ws_bytes,
                                          resolve_tile(KA_KERNEL_SCAN, fn, &d.tile), st);
                break;
            }
            case KA_STAGE_SCATTER:
                e = launch_scatter(c[0].ptr, c[1].ptr, c[2].ptr, nn, np, o[0].ptr, o[0].count, st);
                break;
            case KA_STAGE_PREPARE:
                e = launch_prepare_index(c[0].ptr, c[0].ptr + c[0].cap, nn, np, o[0].ptr, o[0].count, st);
                break;
            case KA_STAGE_EMPTY: e = launch_empty(st); break;
            case KA_STAGE_MANDELBROT:  // the rectangle of the paper's workload (Sec. 5.4)
                e = launch_mandelbrot(o[0].ptr, uint32_t(d.pred), d.xform, -0.5f, -0.7375f, 0.1f, -0.1375f, d.param,
                                      o[0].count, st);
                break;
            default: e = KA_E_UNSUPPORTED;
            }
            if (e != KA_OK) return e;
            c = o;
        }
        // the result length comes back to the host the way a receive delivers it
        if (!wait_tag) {
            if (c[0].count) {
                ka_status e = launch_publish(c[0].count, 1, 0, nullptr, pinned_dev, nullptr, st);
                if (e != KA_OK) return e;
            } else {
                pinned[0] = uint32_t(c[0].n);
            }
            return cuda_status(cudaStreamSynchronize(st));
        }
        // KA_BENCH_WAIT_TAG: wait as ka_receive does, on the publish kernel's
        // tag when there is a count word, else by polling an event
        if (!c[0].count) {
            pinned[0] = uint32_t(c[0].n);
            ka_status e = cuda_status(cudaEventRecord(done, st));
            cudaError_t q = cudaErrorNotReady;
            while (e == KA_OK && (q = cudaEventQuery(done)) == cudaErrorNotReady) {
            }
            return e != KA_OK ? e : cuda_status(q);
        }
        seq = seq + 1 ? seq + 1 : 1;
        ka_status e = launch_publish(c[0].count, 1, 0, nullptr, pinned_dev, nullptr, st, pinned_dev + 2, seq);
        if (e != KA_OK) return e;
        for (uint64_t spins = 1; __atomic_load_n(&pinned[2], __ATOMIC_ACQUIRE) != seq; ++spins) {
            if ((spins & 0xFFFF) == 0) {  // a failed launch never stores the tag
                const cudaError_t q = cudaStreamQuery(st);
                if (q != cudaErrorNotReady && q != cudaSuccess) return cuda_status(q);
            }
        }
        return KA_OK;
    };
    if (s == KA_OK) {
        for (int w = 0; w < 3 && s == KA_OK; ++w) s = run_once();
    }
    double t = 0;
    if (s == KA_OK) {
        const double t0 = now_s();
        for (uint32_t k = 0; k < iters && s == KA_OK; ++k) s = run_once();
        t = now_s() - t0;
    }
    if (s == KA_OK) {
        *seconds = t;
        if (last_count) *last_count = pinned[0];
    }
    cudaStreamSynchronize(st);
    if (done) cudaEventDestroy(done);
    if (pinned) cudaFreeHost(pinned);
    for (void *p : allocs) cudaFree(p);
    return s;
}

}  // extern "C"
