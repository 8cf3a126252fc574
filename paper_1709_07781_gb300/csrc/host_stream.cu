// Streaming compaction of a host array (the paper's value mode, Sec. 3.5:
// the first actor uploads the data, the last reads the result back), with
// the upload, the compaction and the read-back overlapped chunk by chunk.
//
// Chunk c goes through three streams: its upload (host -> device), its
// compactions, one per predicate, then a one-thread kernel that stores the
// chunk's counts into host-mapped memory, and finally the read-back of its
// kept entries (device -> host), placed after the kept entries of chunks
// 0 .. c-1. The host thread enqueues chunk c + 1's upload and compactions
// before it waits for chunk c's counts, so the device never idles on the
// host; uploads of later chunks and read-backs of earlier ones share the
// link in both directions at once. kBufs device buffers per role rotate.
#include <mutex>

#include "ka_internal.h"

namespace ka {
namespace {

constexpr uint64_t kHostChunkDefault = 1ull << 24;  // entries per chunk (64 MiB)
constexpr int kBufs = 3;                            // chunks in flight

uint64_t r256(uint64_t b) { return (b + 255) / 256 * 256; }

// Scratch layout for chunks of `chunk` entries and p predicates:
// input[kBufs] | output[kBufs][p] | counts[kBufs][p] | compaction workspace.
struct HostLayout {
    uint32_t *in[kBufs];
    uint32_t *out[kBufs][KA_HOST_MAX_PRED];
    uint32_t *cnt[kBufs];
    void *ws;
    uint64_t ws_bytes;
    uint64_t total;
};

uint64_t host_ws_bytes(uint64_t chunk) {
    // sized for the smallest tile, so enough for every shape
    return workspace_bytes_for_tiles(tiles_for(chunk, 512) + 1);
}

uint64_t host_scratch_bytes(uint64_t chunk, uint32_t p) {
    return kBufs * (1 + uint64_t(p)) * r256(chunk * 4) + kBufs * 256 + r256(host_ws_bytes(chunk));
}

HostLayout host_layout(void *base, uint64_t chunk, uint32_t p) {
    HostLayout L{};
    char *q = static_cast<char *>(base);
    const uint64_t buf = r256(chunk * 4);
    for (int b = 0; b < kBufs; ++b) {
        L.in[b] = reinterpret_cast<uint32_t *>(q);
        q += buf;
    }
    for (int b = 0; b < kBufs; ++b)
        for (uint32_t i = 0; i < p; ++i) {
            L.out[b][i] = reinterpret_cast<uint32_t *>(q);
            q += buf;
        }
    for (int b = 0; b < kBufs; ++b) {
        L.cnt[b] = reinterpret_cast<uint32_t *>(q);
        q += 256;
    }
    L.ws = q;
    L.ws_bytes = host_ws_bytes(chunk);
    L.total = host_scratch_bytes(chunk, p);
    return L;
}

// Streams, events and the host-mapped count slots, made once per device and
// used by one call at a time.
struct HostCtx {
    bool ready = false;
    cudaStream_t up = nullptr, comp = nullptr, down = nullptr;
    cudaEvent_t ev_up[kBufs] = {}, ev_comp[kBufs] = {}, ev_down[kBufs] = {};
    uint32_t *h_cnt = nullptr, *h_cnt_dev = nullptr;  // [kBufs][KA_HOST_MAX_PRED], host-mapped
    std::mutex mu;
};

HostCtx g_host[kMaxDevices];

ka_status host_ctx_setup(HostCtx &c) {
    if (c.ready) return KA_OK;
    ka_status s = KA_OK;
    for (cudaStream_t *st : {&c.up, &c.comp, &c.down})
        if (s == KA_OK) s = cuda_status(cudaStreamCreateWithFlags(st, cudaStreamNonBlocking));
    for (int b = 0; b < kBufs && s == KA_OK; ++b)
        for (cudaEvent_t *e : {&c.ev_up[b], &c.ev_comp[b], &c.ev_down[b]})
            if (s == KA_OK) s = cuda_status(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    if (s == KA_OK)
        s = cuda_status(cudaHostAlloc(reinterpret_cast<void **>(&c.h_cnt), kBufs * KA_HOST_MAX_PRED * 4,
                                      cudaHostAllocMapped));
    if (s == KA_OK) s = cuda_status(cudaHostGetDevicePointer(reinterpret_cast<void **>(&c.h_cnt_dev), c.h_cnt, 0));
    c.ready = s == KA_OK;
    return s;
}

}  // namespace
}  // namespace ka

using namespace ka;

extern "C" {

ka_status ka_compact_host_scratch_size(uint64_t chunk, uint32_t n_pred, uint64_t *bytes) {
    if (!bytes || n_pred == 0 || n_pred > KA_HOST_MAX_PRED) return KA_E_ARG;
    if (chunk == 0) chunk = kHostChunkDefault;
    if (chunk > 0xFFFFFFFCull) return KA_E_ARG;
    *bytes = host_scratch_bytes(chunk, n_pred);
    return KA_OK;
}

ka_status ka_compact_host(const uint32_t *h_in, uint64_t n, uint32_t n_pred, const int32_t *pred,
                          const uint32_t *param, const uint32_t *xform, uint32_t *const *h_out, uint64_t *count,
                          uint64_t chunk, void *d_scratch, uint64_t scratch_bytes) {
    if (n_pred == 0 || n_pred > KA_HOST_MAX_PRED || !pred || !param || !xform || !h_out || !count) return KA_E_ARG;
    if (chunk == 0) chunk = kHostChunkDefault;
    if (chunk > 0xFFFFFFFCull) return KA_E_ARG;
    if (n && !h_in) return KA_E_ARG;
    PredDev pd[KA_HOST_MAX_PRED];
    uint32_t mul[KA_HOST_MAX_PRED];
    for (uint32_t p = 0; p < n_pred; ++p) {
        if (n && !h_out[p]) return KA_E_ARG;
        const ka_status s = make_pred(pred[p], param[p], &pd[p]);
        if (s != KA_OK) return s;
        if (xform[p] != KA_XFORM_NONE && xform[p] != KA_XFORM_HASH) return KA_E_ARG;
        mul[p] = xform[p] == KA_XFORM_HASH ? kHashMul : 1u;
    }
    if (!d_scratch || (reinterpret_cast<uintptr_t>(d_scratch) & 255u) != 0) return KA_E_ARG;
    if (scratch_bytes < host_scratch_bytes(chunk, n_pred)) return KA_E_WORKSPACE;
    const HostLayout L = host_layout(d_scratch, chunk, n_pred);
    for (uint32_t p = 0; p < n_pred; ++p) count[p] = 0;
    if (n == 0) return KA_OK;

    int dev = 0;
    ka_status s = cuda_status(cudaGetDevice(&dev));
    if (s != KA_OK) return s;
    if (dev < 0 || dev >= kMaxDevices) return KA_E_ARG;
    HostCtx &C = g_host[dev];
    std::lock_guard<std::mutex> lock(C.mu);
    if ((s = host_ctx_setup(C)) != KA_OK) return s;

    const ka_tile tile = resolve_tile(KA_KERNEL_COMPACT, chunk, nullptr);
    s = ka_workspace_init(L.ws, L.ws_bytes, C.comp);
    uint64_t off[KA_HOST_MAX_PRED] = {0, 0, 0, 0};
    const uint64_t chunks = (n + chunk - 1) / chunk;
    // c < chunks: enqueue chunk c; c >= 1: read back chunk c - 1
    for (uint64_t c = 0; c <= chunks && s == KA_OK; ++c) {
        if (c < chunks) {
            const int b = int(c % kBufs);
            const uint64_t first = c * chunk, len = n - first < chunk ? n - first : chunk;
            // the input buffer was last read by chunk c - kBufs's compactions,
            // the output buffers by its read-back
            if (c >= kBufs) s = cuda_status(cudaStreamWaitEvent(C.up, C.ev_comp[b], 0));
            if (s == KA_OK)
                s = cuda_status(cudaMemcpyAsync(L.in[b], h_in + first, len * 4, cudaMemcpyHostToDevice, C.up));
            if (s == KA_OK) s = cuda_status(cudaEventRecord(C.ev_up[b], C.up));
            if (s == KA_OK) s = cuda_status(cudaStreamWaitEvent(C.comp, C.ev_up[b], 0));
            if (s == KA_OK && c >= kBufs) s = cuda_status(cudaStreamWaitEvent(C.comp, C.ev_down[b], 0));
            for (uint32_t p = 0; p < n_pred && s == KA_OK; ++p) {
                CompactLaunch cl;
                cl.in = L.in[b];
                cl.out = L.out[b][p];
                cl.n_ptr = nullptr;
                cl.count = L.cnt[b] + p;
                cl.n = len;
                cl.pred = pd[p];
                cl.mul = mul[p];
                cl.ws = L.ws;
                cl.ws_bytes = L.ws_bytes;
                cl.tile = tile;
                s = launch_compact(cl, C.comp);
            }
            if (s == KA_OK)
                s = launch_publish(L.cnt[b], n_pred, 0, nullptr, C.h_cnt_dev + b * KA_HOST_MAX_PRED, nullptr, C.comp);
            if (s == KA_OK) s = cuda_status(cudaEventRecord(C.ev_comp[b], C.comp));
        }
        if (c >= 1 && s == KA_OK) {
            const int pb = int((c - 1) % kBufs);
            s = cuda_status(cudaEventSynchronize(C.ev_comp[pb]));  // chunk c - 1's counts are on the host
            if (s == KA_OK) s = cuda_status(cudaStreamWaitEvent(C.down, C.ev_comp[pb], 0));
            for (uint32_t p = 0; p < n_pred && s == KA_OK; ++p) {
                const uint64_t k = C.h_cnt[pb * KA_HOST_MAX_PRED + p];
                if (k)
                    s = cuda_status(
                        cudaMemcpyAsync(h_out[p] + off[p], L.out[pb][p], k * 4, cudaMemcpyDeviceToHost, C.down));
                off[p] += k;
            }
            if (s == KA_OK) s = cuda_status(cudaEventRecord(C.ev_down[pb], C.down));
        }
    }
    // drain every stream, even after an error, so nothing is in flight on return
    const ka_status s_down = cuda_status(cudaStreamSynchronize(C.down));
    const ka_status s_comp = cuda_status(cudaStreamSynchronize(C.comp));
    const ka_status s_up = cuda_status(cudaStreamSynchronize(C.up));
    if (s == KA_OK) s = s_down != KA_OK ? s_down : s_comp != KA_OK ? s_comp : s_up;
    if (s == KA_OK) {
        ka_status dev_status = KA_OK;
        s = ka_workspace_status(L.ws, C.comp, &dev_status);
        if (s == KA_OK) s = dev_status;
    }
    if (s == KA_OK)
        for (uint32_t p = 0; p < n_pred; ++p) count[p] = off[p];
    return s;
}

}  // extern "C"
