// Fused compaction without caller-supplied scratch: ka_compact_static.
//
// ka_compact needs a device workspace (the look-back status words and the
// launch ticket), which the caller allocates. Some callers cannot allocate
// device memory at the point where they compact: code that runs inside
// another framework's allocator-managed region, code on a path that must not
// synchronise (cudaMalloc/cudaFree may), and plug-ins handed only the buffers
// they read and write. This variant keeps its workspace in a fixed-size array
// in the library's own device memory instead, so a call allocates nothing.
//
// The array is a file-scope __device__ variable: every GPU on which this
// module is loaded holds kStaticScratchBytes (about 2 MiB) of it until the
// process exits. All calls on a GPU share that one array.
#include <mutex>

#include "ka_internal.h"

namespace ka {
namespace {

// Room for the smallest tile shape (512 entries) at the largest capacity, so
// every supported shape fits: the header plus two status entries per tile.
constexpr uint64_t kStaticTiles = (uint64_t(KA_STATIC_MAX_N) + 511) / 512 + 1;
constexpr uint64_t kStaticScratchBytes = kWsHeaderBytes + ((2 * kStaticTiles * kStatusEntryBytes + 255) / 256) * 256;

// In host code this name only stands for the device array; its device address
// comes from cudaGetSymbolAddress, once per device, with that device current.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void *g_static_ptr[kMaxDevices] = {};

// Device address of the array on the current device. The first call on a
// device looks it up and initialises it (header: epoch 1, no tickets taken,
// default spin limit; every status word zero) on `stream`, then waits for
// that stream. That wait cannot happen inside a stream capture, so a first
// call made while `stream` is capturing fails with KA_E_UNSUPPORTED.
ka_status static_scratch(cudaStream_t stream, void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kMaxDevices) return KA_E_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (g_static_ptr[dev]) {
        *out = g_static_ptr[dev];
        return KA_OK;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return cuda_status(e);
    if (cap != cudaStreamCaptureStatusNone) return KA_E_UNSUPPORTED;
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_status(e);
    if ((reinterpret_cast<uintptr_t>(p) & 255u) != 0) return KA_E_WORKSPACE;
    ka_status s = ka_workspace_init(p, kStaticScratchBytes, stream);
    if (s == KA_OK) s = cuda_status(cudaStreamSynchronize(stream));
    if (s != KA_OK) return s;
    g_static_ptr[dev] = p;
    *out = p;
    return KA_OK;
}

}  // namespace
}  // namespace ka

using namespace ka;

// The launch is the one ka_compact makes, with the shared array as workspace.
// Nothing needs clearing between calls: every status word carries the epoch
// of the launch that wrote it, so words left by an earlier call read as "not
// published yet", and the last block of every launch returns the ticket count
// to zero. Two calls whose kernels overlap on the GPU (different streams, no
// ordering between them) take tickets from the same word and read each
// other's status words: they race, and their results are undefined.
extern "C" ka_status ka_compact_static(const uint32_t *d_in, uint64_t n, const uint32_t *d_n, int32_t pred,
                                       uint32_t param, uint32_t xform, uint32_t *d_out, uint32_t *d_count,
                                       const ka_tile *tile, void *stream) {
    if (n > KA_STATIC_MAX_N) return KA_E_TOO_LARGE;
    CompactLaunch L;
    ka_status s = make_pred(pred, param, &L.pred);
    if (s != KA_OK) return s;
    if (xform != KA_XFORM_NONE && xform != KA_XFORM_HASH) return KA_E_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *ws = nullptr;
    s = static_scratch(st, &ws);
    if (s != KA_OK) return s;
    L.in = d_in;
    L.out = d_out;
    L.n_ptr = d_n;
    L.count = d_count;
    L.n = n;
    L.mul = xform == KA_XFORM_HASH ? kHashMul : 1u;
    L.ws = ws;
    L.ws_bytes = kStaticScratchBytes;
    L.tile = resolve_tile(KA_KERNEL_COMPACT, n, tile);
    return launch_compact(L, st);
}

// The array as a workspace, so that the workspace calls (status, clear, spin
// limit) work on it: a device error of a call is recorded in its header.
extern "C" ka_status ka_compact_static_workspace(void *stream, void **d_ws, uint64_t *bytes) {
    if (!d_ws || !bytes) return KA_E_ARG;
    void *ws = nullptr;
    const ka_status s = static_scratch(static_cast<cudaStream_t>(stream), &ws);
    if (s != KA_OK) return s;
    *d_ws = ws;
    *bytes = kStaticScratchBytes;
    return KA_OK;
}
