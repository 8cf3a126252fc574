// Internal host-side declarations of libka (not part of the C ABI).
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ka.h"
#include "ka_dev.cuh"

namespace ka {

// Device properties of the current device, cached per ordinal.
struct DeviceInfo {
    int ordinal = -1;
    int sm_count = 0;
    int max_smem_optin = 0;
};
const DeviceInfo &device_info();

// A launch quantity (occupancy, resident grid size) cached per device
// ordinal: devices differ in SM count and resident slots, and a function
// attribute set with cudaFuncSetAttribute holds for the current device only.
constexpr int kMaxDevices = 64;
struct PerDeviceInt {
    std::atomic<int> slot[kMaxDevices];  // 0: not computed yet (static storage starts at zero)
};
// Ordinal of the calling thread's current device (-1 on error).
int current_device();
// The value for device `dev`: the cached one, else compute(), cached when it
// is positive (a value <= 0 reports an error and is not cached). Threads that
// race on a first use both compute the same value.
template <class F>
int per_device_value(PerDeviceInt &cache, int dev, F &&compute) {
    if (dev < 0 || dev >= kMaxDevices) return compute();
    const int v = cache.slot[dev].load(std::memory_order_acquire);
    if (v > 0) return v;
    const int w = compute();
    if (w > 0) cache.slot[dev].store(w, std::memory_order_release);
    return w;
}

// Status of a launch whose set-up (function attribute, occupancy) failed: the
// CUDA error behind it, or KA_E_UNSUPPORTED when the kernel cannot be
// resident on this device at all.
inline ka_status launch_setup_error();

// cudaError_t -> ka_status (records the CUDA error for ka_strerror detail).
ka_status cuda_status(cudaError_t e);

// Canonical device predicate for (kind, param). KA_E_ARG on an unknown kind
// or a zero modulus.
ka_status make_pred(int32_t kind, uint32_t param, PredDev *out);

// Supported tile shapes (block threads, items per thread); the list drives
// every templated launcher through KA_FOR_EACH_SHAPE(X), X(block, ipt).
#define KA_FOR_EACH_SHAPE(X) \
    X(128, 4) X(128, 8) X(128, 16) X(256, 4) X(256, 8) X(256, 16) X(512, 4) X(512, 8) X(512, 16) X(1024, 4) X(1024, 8)
constexpr uint32_t shape_key(uint32_t block, uint32_t ipt) { return block * 100 + ipt; }
bool tile_supported(uint32_t block, uint32_t ipt);
// Shapes of the warp-specialised TMA kernels (compaction, scan, batch):
// (256, 16), (512, 16) and (768, 16); the last exists for them only.
bool tma_shape(uint32_t block, uint32_t ipt);
// Shape of the TMA batch kernel: the TMA shapes and (704, 16).
bool batch_tma_shape(uint32_t block, uint32_t ipt);
// Shape valid for `kernel` (a KA_KERNEL_* id).
bool tile_supported_for(int32_t kernel, uint32_t block, uint32_t ipt);
// Shape to use for `kernel` at size n: explicit shape, else autotuned, else default.
ka_tile resolve_tile(int32_t kernel, uint64_t n, const ka_tile *requested);
// The batch kernel has one shape for every batch, stored under this size.
constexpr uint64_t kBatchTileKey = 1ull << 17;
ka_status autotune_batch(uint64_t total, const char *cache_path, ka_tile *best, float *best_us, void *stream);

// Workspace layout for single-pass kernels: the 256-byte header, then status
// entries of kStatusStride words. Room for two entries per tile: one per tile
// plus, for the round-robin kernel, one per iteration (never more than tiles).
constexpr uint64_t kWsHeaderBytes = 256;
constexpr uint64_t kStatusEntryBytes = 8 * kStatusStride;
inline uint64_t tiles_for(uint64_t n, uint32_t tile_elems) { return (n + tile_elems - 1) / tile_elems; }
inline uint64_t workspace_bytes_for_tiles(uint64_t tiles) {
    return kWsHeaderBytes + ((2 * tiles * kStatusEntryBytes + 255) / 256) * 256;
}
inline uint32_t status_capacity(uint64_t ws_bytes) {
    const uint64_t e = ws_bytes > kWsHeaderBytes ? (ws_bytes - kWsHeaderBytes) / kStatusEntryBytes : 0;
    return e > 0xFFFFFFFFull ? 0xFFFFFFFFu : uint32_t(e);
}

// Device ordinal and memory budget of an actor system (for the serving loop).
ka_status system_exec_info(ka_system *sys, int *device, uint64_t *budget);

// Launchers shared by the C ABI and the actor runtime. All asynchronous.
struct CompactLaunch {
    const uint32_t *in;
    uint32_t *out;
    const uint32_t *n_ptr;
    uint32_t *count;
    uint64_t n;  // live length, or capacity when n_ptr is set
    PredDev pred;
    uint32_t mul;  // 1, or the hash multiplier
    void *ws;
    uint64_t ws_bytes;
    ka_tile tile;
};
ka_status launch_compact(const CompactLaunch &L, cudaStream_t stream);
// The warp-specialised TMA kernel (the TMA shapes, any 4-byte-aligned input
// of up to 2^32 - 4 entries); launch_compact routes to it when eligible.
bool compact_tma_eligible(const CompactLaunch &L);
ka_status launch_compact_tma(const CompactLaunch &L, cudaStream_t stream);

// The warp-specialised TMA kernel in scan mode (TMA shapes).
ka_status launch_scan_tma(const uint32_t *in, uint64_t n, const uint32_t *n_ptr, uint32_t *out, uint32_t *total,
                          void *ws, uint64_t ws_bytes, ka_tile tile, cudaStream_t stream);
ka_status launch_exclusive_scan(const uint32_t *in, uint64_t n, const uint32_t *n_ptr, uint32_t *out,
                                uint32_t *total, void *ws, uint64_t ws_bytes, ka_tile tile,
                                cudaStream_t stream);
ka_status launch_scatter(const uint32_t *x, const uint32_t *flags, const uint32_t *offsets, uint64_t n,
                         const uint32_t *n_ptr, uint32_t *out, uint32_t *count_out, cudaStream_t stream);
ka_status launch_empty(cudaStream_t stream);
// Stores n words of src (src null: the one word `fixed`) and, if err is not
// null, *err into host-mapped pinned memory dst / dst_err; then, if dst_tag is
// not null (n <= 256), `tag` into dst_tag after a system-scope fence.
ka_status launch_publish(const uint32_t *src, uint32_t n, uint32_t fixed, const uint32_t *err, uint32_t *dst,
                         uint32_t *dst_err, cudaStream_t stream, uint32_t *dst_tag = nullptr, uint32_t tag = 0);
ka_status launch_mandelbrot(uint32_t *out, uint32_t width, uint32_t height, float re_min, float im_min, float re_max,
                            float im_max, uint32_t max_iter, uint32_t *n_out, cudaStream_t stream);
ka_status launch_generate(uint32_t *out, uint64_t n, uint64_t seed, uint32_t *n_out, cudaStream_t stream);
ka_status launch_map_hash(const uint32_t *in, uint64_t n, const uint32_t *n_ptr, uint32_t *out,
                          uint32_t *n_out, cudaStream_t stream);
ka_status launch_predicate(const uint32_t *x, uint64_t n, const uint32_t *n_ptr, const PredDev &pred,
                           uint32_t *flags, uint32_t *n_out, cudaStream_t stream);
ka_status launch_prepare_index(const uint32_t *a, const uint32_t *b, uint64_t k, const uint32_t *k_ptr,
                               uint32_t *index, uint32_t *n_out, cudaStream_t stream);
ka_status launch_copy_count(const uint32_t *n_ptr, uint64_t n, uint32_t *n_out, cudaStream_t stream);

// Workspace validation (host side): size and alignment.
ka_status check_workspace(const void *ws, uint64_t ws_bytes, uint64_t tiles_needed);

constexpr uint32_t kHashMul = 2654435761u;

inline ka_status launch_setup_error() {
    const cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? cuda_status(e) : KA_E_UNSUPPORTED;
}

}  // namespace ka
