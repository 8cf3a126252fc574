// Three-phase compaction in the manner of Billeter et al., the method the
// paper's fuseFillsLiterals step uses (Sec. 4.1, Listing 5): count the kept
// entries of each segment, exclusive-scan the segment counts, then move
// every kept entry to its segment's offset plus its rank inside the
// segment. The input is read twice (8N + 4K bytes plus the small count
// arrays), against 4N + 4K for the single pass and 28N + 4K for flag map,
// element scan and scatter.
//
// A segment is 512 entries, one warp's share, as in Billeter et al.: warps
// count and move their segments independently (no block barriers), each
// lane holding four 16-byte rows of the segment (entry r 128 + 4 lane + c).
// The move stages a segment's kept entries in the warp's own 2 KiB of shared
// memory and stores them 16 bytes at a time, realigned to the output.
//
// Workspace: first the workspace of the scan of the counts (its header is the
// workspace's header, so ka_workspace_status reports the scan's device-side
// failures), then segment counts [segments], segment offsets [segments] and
// the live segment count.
#include "ka_internal.h"
#include "ka_tma.cuh"

namespace ka {
namespace {

constexpr int kTpBlock = 256, kTpWarps = kTpBlock / 32;
constexpr int kTpSeg = 512;  // entries per segment
constexpr int kTpTile = kTpSeg;

struct TpLayout {
    uint32_t *counts;
    uint32_t *offsets;
    uint32_t *n_tiles;  // live segment count (device word; the scan's length)
    void *scan_ws;
    uint64_t scan_ws_bytes;
};

uint64_t r256(uint64_t b) { return (b + 255) / 256 * 256; }

// Scan workspace for `tiles` segment counts (sized for the smallest tile).
uint64_t tp_scan_bytes(uint64_t tiles) { return r256(workspace_bytes_for_tiles(tiles_for(tiles, 512) + 1)); }

TpLayout tp_layout(void *ws, uint64_t tiles) {
    TpLayout L;
    char *p = static_cast<char *>(ws);
    L.scan_ws = p;
    L.scan_ws_bytes = tp_scan_bytes(tiles);
    p += L.scan_ws_bytes;
    L.counts = reinterpret_cast<uint32_t *>(p);
    p += r256(tiles * 4);
    L.offsets = reinterpret_cast<uint32_t *>(p);
    p += r256(tiles * 4);
    L.n_tiles = reinterpret_cast<uint32_t *>(p);
    return L;
}

uint64_t tp_bytes(uint64_t capacity) {
    const uint64_t tiles = tiles_for(capacity ? capacity : 1, kTpTile);
    return tp_scan_bytes(tiles) + 2 * r256(tiles * 4) + 256;
}

__device__ __forceinline__ uint32_t tp_live(const uint32_t *n_ptr, uint32_t n) {
    if (!n_ptr) return n;
    const uint32_t d = *n_ptr;
    return d < n ? d : n;
}

// Segments of n entries (64-bit sum: n may be up to 2^32 - 1).
__device__ __forceinline__ uint32_t tp_segments(uint32_t n) {
    return uint32_t((uint64_t(n) + kTpSeg - 1) / kTpSeg);
}

// This lane's 16 entries of the segment at seg_in (valid entries: the first
// `valid`; the others read as 0 and are masked off), transformed by mul, and
// their keep mask (bit 4 r + c for entry r 128 + 4 lane + c).
// With `pre` (a full, 16-byte aligned segment) the rows come from q, loaded
// earlier by tp_prefetch.
__device__ __forceinline__ uint32_t tp_segment(const uint32_t *seg_in, uint32_t valid, bool pre, const uint4 q[4],
                                               uint32_t mul, const PredDev &pred, int lane, uint32_t v[16]) {
    uint32_t m = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const uint32_t e0 = uint32_t(r * 128 + lane * 4);
        if (pre) {
            v[4 * r] = q[r].x;
            v[4 * r + 1] = q[r].y;
            v[4 * r + 2] = q[r].z;
            v[4 * r + 3] = q[r].w;
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) v[4 * r + c] = e0 + c < valid ? seg_in[e0 + c] : 0u;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) v[4 * r + c] *= mul;
        uint32_t mk = pred_mask4(pred, v[4 * r], v[4 * r + 1], v[4 * r + 2], v[4 * r + 3]);
        const uint32_t left = valid > e0 ? valid - e0 : 0u;
        mk &= left >= 4 ? 0xFu : ((1u << left) - 1u);
        m |= mk << (4 * r);
    }
    return m;
}

// This lane's four rows of a full segment, when the input is 16-byte aligned.
__device__ __forceinline__ void tp_prefetch(const uint32_t *seg_in, int lane, uint4 q[4]) {
#pragma unroll
    for (int r = 0; r < 4; ++r) q[r] = ld_stream_v4(seg_in + r * 128 + lane * 4);
}

// Walks this warp's segments seg0, seg0 + stride, ... with the next full
// aligned segment's loads issued before the current one is processed;
// body(seg, base, valid, pre, q) processes one segment.
template <class Body>
__device__ __forceinline__ void tp_walk(const uint32_t *in, uint32_t n, bool vec, uint32_t seg0, uint32_t stride,
                                        int lane, Body body) {
    const uint32_t segs = tp_segments(n), full = n / kTpSeg;
    uint4 cur[4], nxt[4];
    if (vec && seg0 < full) tp_prefetch(in + size_t(seg0) * kTpSeg, lane, nxt);
    for (uint32_t seg = seg0; seg < segs; seg += stride) {
        const bool pre = vec && seg < full;
#pragma unroll
        for (int r = 0; r < 4; ++r) cur[r] = nxt[r];
        if (vec && seg + stride < full) tp_prefetch(in + size_t(seg + stride) * kTpSeg, lane, nxt);
        const uint32_t base = seg * uint32_t(kTpSeg);
        body(seg, base, min(n - base, uint32_t(kTpSeg)), pre, cur);
    }
}

// Phase 1: kept entries per segment, one warp per segment.
constexpr int kTpBlocksPerSm = 4;  // each warp keeps two segments' loads in flight
__global__ void __launch_bounds__(kTpBlock, kTpBlocksPerSm) k_tp_count(const uint32_t *in, uint32_t cap, const uint32_t *n_ptr,
                                                        PredDev pred, uint32_t mul, int vec, TpLayout L) {
    const uint32_t n = tp_live(n_ptr, cap);
    const uint32_t segs = tp_segments(n);
    if (blockIdx.x == 0 && threadIdx.x == 0) *L.n_tiles = segs;
    const int lane = threadIdx.x & 31;
    tp_walk(in, n, vec != 0, blockIdx.x * kTpWarps + (threadIdx.x >> 5), gridDim.x * kTpWarps, lane,
            [&](uint32_t seg, uint32_t base, uint32_t valid, bool pre, const uint4 q[4]) {
                uint32_t v[16];
                const uint32_t m = tp_segment(in + base, valid, pre, q, mul, pred, lane, v);
                const uint32_t c = warp_sum(uint32_t(__popc(m)));
                if (lane == 0) L.counts[seg] = c;
            });
}

// Phase 3: every kept entry of a segment to offsets[segment] + its rank.
__global__ void __launch_bounds__(kTpBlock, kTpBlocksPerSm) k_tp_move(const uint32_t *in, uint32_t cap, const uint32_t *n_ptr,
                                                       PredDev pred, uint32_t mul, int vec, TpLayout L,
                                                       uint32_t *out) {
    __shared__ __align__(16) uint32_t s_seg[kTpWarps][kTpSeg];
    const uint32_t n = tp_live(n_ptr, cap);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *const stage = s_seg[warp];
    tp_walk(in, n, vec != 0, blockIdx.x * kTpWarps + uint32_t(warp), gridDim.x * kTpWarps, lane,
            [&](uint32_t seg, uint32_t base, uint32_t valid, bool pre, const uint4 q[4]) {
        uint32_t v[16];
        const uint32_t m = tp_segment(in + base, valid, pre, q, mul, pred, lane, v);
        // rank of this lane's first kept entry of each row: row counts in
        // 8-bit fields (a row keeps at most 128), scanned across the warp
        uint32_t packed = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) packed += uint32_t(__popc((m >> (4 * r)) & 0xFu)) << (8 * r);
        const uint32_t incl = warp_incl_scan(packed, lane);
        const uint32_t excl = incl - packed;
        const uint32_t rows = __shfl_sync(kFull, incl, 31);
        uint32_t rowbase = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            uint32_t pos = rowbase + ((excl >> (8 * r)) & 0xFFu);
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if ((m >> (4 * r + c)) & 1u) stage[pos++] = v[4 * r + c];
            rowbase += (rows >> (8 * r)) & 0xFFu;
        }
        __syncwarp();
        if (rowbase) tma::warp_copy_out(stage, out + L.offsets[seg], rowbase, lane);
        __syncwarp();  // the stage is read before the next segment overwrites it
    });
}

// One wave of `per_sm` blocks per SM, each warp looping over segments.
unsigned tp_grid(uint64_t cap, int per_sm) {
    uint64_t g = tiles_for(tiles_for(cap ? cap : 1, kTpSeg), kTpWarps);
    const uint64_t lim = uint64_t(device_info().sm_count) * per_sm;
    return unsigned(g < lim ? g : lim);
}

}  // namespace
}  // namespace ka

using namespace ka;

extern "C" {

ka_status ka_three_phase_workspace_size(uint64_t capacity, uint64_t *bytes) {
    if (!bytes || capacity > 0xFFFFFFFFull) return KA_E_ARG;
    *bytes = tp_bytes(capacity);
    return KA_OK;
}

ka_status ka_compact_three_phase(const uint32_t *d_in, uint64_t n, const uint32_t *d_n, int32_t pred, uint32_t param,
                                 uint32_t xform, uint32_t *d_out, uint32_t *d_count, void *d_ws, uint64_t ws_bytes,
                                 void *stream) {
    if (n > 0xFFFFFFFFull || (n && (!d_in || !d_out)) || !d_count) return KA_E_ARG;
    if (d_n && d_n == d_count) return KA_E_ARG;
    if (xform != KA_XFORM_NONE && xform != KA_XFORM_HASH) return KA_E_ARG;
    if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255u) != 0) return KA_E_ARG;
    if (ws_bytes < tp_bytes(n)) return KA_E_WORKSPACE;
    PredDev p;
    ka_status s = make_pred(pred, param, &p);
    if (s != KA_OK) return s;
    const uint64_t tiles = tiles_for(n ? n : 1, kTpTile);
    const TpLayout L = tp_layout(d_ws, tiles);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t mul = xform == KA_XFORM_HASH ? kHashMul : 1u;
    const int vec = (reinterpret_cast<uintptr_t>(d_in) & 15u) == 0 ? 1 : 0;
    // the scan's workspace is the one ka_workspace_init prepared; its epoch
    // tags make later launches safe without clearing
    k_tp_count<<<tp_grid(n, kTpBlocksPerSm), kTpBlock, 0, st>>>(d_in, uint32_t(n), d_n, p, mul, vec, L);
    s = cuda_status(cudaGetLastError());
    if (s != KA_OK) return s;
    // phase 2: segment offsets; the total of the counts is the result length
    s = launch_exclusive_scan(L.counts, tiles, L.n_tiles, L.offsets, d_count, L.scan_ws, L.scan_ws_bytes,
                              resolve_tile(KA_KERNEL_SCAN, tiles, nullptr), st);
    if (s != KA_OK) return s;
    k_tp_move<<<tp_grid(n, kTpBlocksPerSm), kTpBlock, 0, st>>>(d_in, uint32_t(n), d_n, p, mul, vec, L, d_out);
    return cuda_status(cudaGetLastError());
}

}  // extern "C"
