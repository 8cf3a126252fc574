// Status text, device properties, predicate set-up and workspace handling.
#include <cstring>
#include <mutex>

#include "ka_internal.h"

namespace ka {

// The CUDA error behind the last KA_E_CUDA on this thread (ka_last_cuda_error).
static thread_local int g_last_cuda_error = 0;

ka_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return KA_OK;
    g_last_cuda_error = int(e);
    return KA_E_CUDA;
}

int current_device() {
    int dev = -1;
    return cudaGetDevice(&dev) == cudaSuccess ? dev : -1;
}

const DeviceInfo &device_info() {
    static std::mutex mu;
    static DeviceInfo cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lock(mu);
    DeviceInfo &d = cache[dev];
    if (d.ordinal != dev) {
        int sms = 0, smem = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        d.sm_count = sms > 0 ? sms : 1;
        d.max_smem_optin = smem;
        d.ordinal = dev;
    }
    return d;
}

ka_status make_pred(int32_t kind, uint32_t param, PredDev *out) {
    return pred_canon(kind, param, out) == 0 ? KA_OK : KA_E_ARG;
}

bool tile_supported(uint32_t block, uint32_t ipt) {
#define KA_SUPPORTED(B, I) \
    if (block == B && ipt == I) return true;
    KA_FOR_EACH_SHAPE(KA_SUPPORTED)
#undef KA_SUPPORTED
    return false;
}

bool tile_supported_for(int32_t kernel, uint32_t block, uint32_t ipt) {
    if (kernel == KA_KERNEL_BATCH) return tile_supported(block, ipt) || batch_tma_shape(block, ipt);
    return tile_supported(block, ipt) || tma_shape(block, ipt);  // every kernel has the TMA shapes
}

ka_status check_workspace(const void *ws, uint64_t ws_bytes, uint64_t tiles_needed) {
    if (!ws) return KA_E_ARG;
    if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return KA_E_ARG;
    if (ws_bytes < workspace_bytes_for_tiles(tiles_needed)) return KA_E_WORKSPACE;
    return KA_OK;
}

__global__ void k_ws_init(WsHeader *h, uint64_t *status, uint64_t words) {
    const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    if (i == 0) {
        h->ticket = 1ull << 32;  // epoch 1, no tickets taken
        h->error = 0;
        h->error_tile = 0;
        h->spin_limit = kDefaultSpinLimit;
        h->magic = kWsMagic;
    }
    for (uint64_t w = i; w < words; w += stride) status[w] = 0;
}

__global__ void k_ws_set_spin(WsHeader *h, uint32_t polls) { h->spin_limit = polls; }

}  // namespace ka

using namespace ka;

extern "C" {

const char *ka_strerror(ka_status s) {
    switch (s) {
    case KA_OK: return "ok";
    case KA_E_ARG: return "invalid argument";
    case KA_E_TYPE: return "message does not match the actor's signature";
    case KA_E_OOM: return "out of memory";
    case KA_E_BUDGET: return "request exceeds the memory budget";
    case KA_E_STALE: return "handle already released";
    case KA_E_CUDA: return "CUDA runtime error";
    case KA_E_DEVICE_TIMEOUT: return "device-side wait timed out";
    case KA_E_CLOSED: return "system or mailbox closed";
    case KA_E_NOT_SERIALIZABLE: return "device references cannot be serialised";
    case KA_E_TIMEOUT: return "timed out waiting for the response";
    case KA_E_UNSUPPORTED: return "unsupported option";
    case KA_E_INJECTED: return "injected failure (test hook)";
    case KA_E_WORKSPACE: return "workspace too small or not initialised";
    case KA_E_TOO_LARGE: return "size above the static-scratch limit (KA_STATIC_MAX_N entries)";
    default: return "unknown status";
    }
}

int32_t ka_version(void) { return 100; }

int32_t ka_last_cuda_error(void) { return g_last_cuda_error; }

ka_status ka_workspace_size(uint64_t capacity, const ka_tile *tile, uint64_t *bytes) {
    if (!bytes) return KA_E_ARG;
    if (capacity > 0xFFFFFFFFull) return KA_E_ARG;
    uint32_t te = 512;  // smallest supported tile: enough for every shape
    if (tile && tile->block && tile->ipt) {
        if (!tile_supported(tile->block, tile->ipt) && !tma_shape(tile->block, tile->ipt)) return KA_E_ARG;
        te = tile->block * tile->ipt;
    }
    *bytes = workspace_bytes_for_tiles(tiles_for(capacity, te) + 1);
    return KA_OK;
}

ka_status ka_workspace_init(void *d_ws, uint64_t bytes, void *stream) {
    if (!d_ws || bytes < kWsHeaderBytes) return KA_E_ARG;
    if ((reinterpret_cast<uintptr_t>(d_ws) & 255u) != 0) return KA_E_ARG;
    const uint64_t words = (bytes - kWsHeaderBytes) / 8;
    auto *h = static_cast<WsHeader *>(d_ws);
    auto *status = reinterpret_cast<uint64_t *>(static_cast<char *>(d_ws) + kWsHeaderBytes);
    uint64_t blocks = (words + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 1024) blocks = 1024;
    k_ws_init<<<unsigned(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(h, status, words);
    return cuda_status(cudaGetLastError());
}

ka_status ka_workspace_status(const void *d_ws, void *stream, ka_status *device_status) {
    if (!d_ws || !device_status) return KA_E_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ka_status s = cuda_status(cudaStreamSynchronize(st));
    if (s != KA_OK) return s;
    WsHeader h;
    s = cuda_status(cudaMemcpy(&h, d_ws, sizeof(h), cudaMemcpyDeviceToHost));
    if (s != KA_OK) return s;
    if (h.magic != kWsMagic) {
        *device_status = KA_E_WORKSPACE;
        return KA_OK;
    }
    *device_status = h.error == 0 ? KA_OK : -int32_t(h.error);
    return KA_OK;
}

ka_status ka_debug_pred_keep(int32_t pred, uint32_t param, uint32_t x, int32_t *keep) {
    if (!keep) return KA_E_ARG;
    PredDev p;
    const ka_status s = make_pred(pred, param, &p);
    if (s != KA_OK) return s;
    *keep = pred_keep(p, x) ? 1 : 0;
    return KA_OK;
}

ka_status ka_debug_device_cache(const int32_t *devices, const int32_t *values, uint32_t n, int32_t *out) {
    if (n && (!devices || !values || !out)) return KA_E_ARG;
    PerDeviceInt cache{};
    for (uint32_t i = 0; i < n; ++i) out[i] = per_device_value(cache, devices[i], [&] { return values[i]; });
    return KA_OK;
}

ka_status ka_workspace_set_spin_limit(void *d_ws, uint32_t polls, void *stream) {
    if (!d_ws || polls == 0) return KA_E_ARG;
    k_ws_set_spin<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<WsHeader *>(d_ws), polls);
    return cuda_status(cudaGetLastError());
}

}  // extern "C"
