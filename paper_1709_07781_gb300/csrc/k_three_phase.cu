// Three-phase compaction in the manner of Billeter et al., the method the
// paper's fuseFillsLiterals step uses (Sec. 4.1, Listing 5): count the kept
// entries of each tile, exclusive-scan the tile counts, then move every kept
// entry to its tile's offset plus its rank inside the tile. The input is read
// twice (8N + 4K bytes plus the small count arrays), against 4N + 4K for the
// single pass and 28N + 4K for flag map, element scan and scatter.
//
// Workspace: tile counts [tiles], tile offsets [tiles], the live tile count,
// then a workspace for the scan of the counts.
#include "ka_internal.h"
#include "ka_tma.cuh"

namespace ka {
namespace {

constexpr int kTpBlock = 256, kTpIpt = 16, kTpTile = kTpBlock * kTpIpt;  // 4096 entries per tile
constexpr int kTpWarps = kTpBlock / 32;

struct TpLayout {
    uint32_t *counts;
    uint32_t *offsets;
    uint32_t *n_tiles;  // live tile count (device word; the scan's length)
    void *scan_ws;
    uint64_t scan_ws_bytes;
};

uint64_t r256(uint64_t b) { return (b + 255) / 256 * 256; }

TpLayout tp_layout(void *ws, uint64_t tiles, uint64_t ws_bytes) {
    TpLayout L;
    char *p = static_cast<char *>(ws);
    L.counts = reinterpret_cast<uint32_t *>(p);
    p += r256(tiles * 4);
    L.offsets = reinterpret_cast<uint32_t *>(p);
    p += r256(tiles * 4);
    L.n_tiles = reinterpret_cast<uint32_t *>(p);
    p += 256;
    L.scan_ws = p;
    const uint64_t used = uint64_t(p - static_cast<char *>(ws));
    L.scan_ws_bytes = ws_bytes > used ? ws_bytes - used : 0;
    return L;
}

uint64_t tp_bytes(uint64_t capacity) {
    const uint64_t tiles = tiles_for(capacity ? capacity : 1, kTpTile);
    return 2 * r256(tiles * 4) + 256 + workspace_bytes_for_tiles(tiles_for(tiles, 512) + 1);
}

__device__ __forceinline__ uint32_t tp_live(const uint32_t *n_ptr, uint32_t n) {
    if (!n_ptr) return n;
    const uint32_t d = *n_ptr;
    return d < n ? d : n;
}

// Entry e (0..15) of thread t in a tile: rows of 4-entry vectors,
// entry = 4 (r kTpBlock + t) + c, so each warp load is one coalesced 512-byte run.
__device__ __forceinline__ void tp_load(const uint32_t *tile_in, uint32_t valid, bool vec, uint32_t mul,
                                        uint32_t v[kTpIpt]) {
    const int t = threadIdx.x;
#pragma unroll
    for (int r = 0; r < kTpIpt / 4; ++r) {
        const uint32_t e0 = uint32_t(r * kTpBlock + t) * 4;
        if (vec && e0 + 4 <= valid) {
            const uint4 q = ld_stream_v4(tile_in + e0);
            v[4 * r] = q.x;
            v[4 * r + 1] = q.y;
            v[4 * r + 2] = q.z;
            v[4 * r + 3] = q.w;
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) v[4 * r + c] = e0 + c < valid ? tile_in[e0 + c] : 0u;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) v[4 * r + c] *= mul;
    }
}

__device__ __forceinline__ uint32_t tp_mask(const PredDev &pred, const uint32_t v[kTpIpt], uint32_t valid) {
    const int t = threadIdx.x;
    uint32_t m = 0;
#pragma unroll
    for (int r = 0; r < kTpIpt / 4; ++r) {
        const uint32_t e0 = uint32_t(r * kTpBlock + t) * 4;
        uint32_t mk = pred_mask4(pred, v[4 * r], v[4 * r + 1], v[4 * r + 2], v[4 * r + 3]);
        const uint32_t left = valid > e0 ? valid - e0 : 0u;
        mk &= left >= 4 ? 0xFu : ((1u << left) - 1u);
        m |= mk << (4 * r);
    }
    return m;
}

// Phase 1: kept entries per tile.
__global__ void __launch_bounds__(kTpBlock) k_tp_count(const uint32_t *in, uint32_t cap, const uint32_t *n_ptr,
                                                        PredDev pred, uint32_t mul, int vec, TpLayout L) {
    __shared__ uint32_t s_w[kTpWarps];
    const uint32_t n = tp_live(n_ptr, cap);
    const uint32_t tiles = (n + kTpTile - 1) / kTpTile;
    if (blockIdx.x == 0 && threadIdx.x == 0) *L.n_tiles = tiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const uint32_t base = tile * uint32_t(kTpTile);
        const uint32_t valid = min(n - base, uint32_t(kTpTile));
        uint32_t v[kTpIpt];
        tp_load(in + base, valid, vec != 0, mul, v);
        const uint32_t c = warp_sum(uint32_t(__popc(tp_mask(pred, v, valid))));
        if (lane == 0) s_w[warp] = c;
        __syncthreads();
        if (warp == 0) {
            const uint32_t t = warp_sum(lane < kTpWarps ? s_w[lane] : 0u);
            if (lane == 0) L.counts[tile] = t;
        }
        __syncthreads();
    }
}

// Phase 3: every kept entry to offsets[tile] + its rank in the tile, staged
// in shared memory so the tile's run goes out as coalesced stores.
__global__ void __launch_bounds__(kTpBlock) k_tp_move(const uint32_t *in, uint32_t cap, const uint32_t *n_ptr,
                                                       PredDev pred, uint32_t mul, int vec, TpLayout L,
                                                       uint32_t *out) {
    __shared__ uint32_t s_out[kTpTile];
    __shared__ uint32_t s_w[kTpWarps];
    const uint32_t n = tp_live(n_ptr, cap);
    const uint32_t tiles = (n + kTpTile - 1) / kTpTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const uint32_t base = tile * uint32_t(kTpTile);
        const uint32_t valid = min(n - base, uint32_t(kTpTile));
        uint32_t v[kTpIpt];
        tp_load(in + base, valid, vec != 0, mul, v);
        const uint32_t m = tp_mask(pred, v, valid);
        // rank of this thread's first kept entry: the entries of thread t come
        // in rows, so the rank is taken row by row (8-bit row fields, 4 rows)
        uint32_t packed = 0;
#pragma unroll
        for (int r = 0; r < kTpIpt / 4; ++r) packed += uint32_t(__popc((m >> (4 * r)) & 0xFu)) << (8 * r);
        const uint32_t incl = warp_incl_scan(packed, lane);
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        // row r of the tile: warps in order; rows in order
        uint32_t row_base[kTpIpt / 4], warp_off[kTpIpt / 4];
        {
            uint32_t acc = 0;
#pragma unroll
            for (int r = 0; r < kTpIpt / 4; ++r) {
                uint32_t before = 0, total = 0;
#pragma unroll
                for (int w = 0; w < kTpWarps; ++w) {
                    const uint32_t f = (s_w[w] >> (8 * r)) & 0xFFu;
                    if (w < warp) before += f;
                    total += f;
                }
                row_base[r] = acc;
                warp_off[r] = before;
                acc += total;
            }
        }
        const uint32_t excl = incl - packed;
#pragma unroll
        for (int r = 0; r < kTpIpt / 4; ++r) {
            uint32_t pos = row_base[r] + warp_off[r] + ((excl >> (8 * r)) & 0xFFu);
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if ((m >> (4 * r + c)) & 1u) s_out[pos++] = v[4 * r + c];
        }
        __syncthreads();
        const uint32_t kept = L.counts[tile];
        uint32_t *dst = out + L.offsets[tile];
        for (uint32_t i = threadIdx.x; i < kept; i += kTpBlock) dst[i] = s_out[i];
        __syncthreads();
    }
}

// Phase 3 for a 16-byte aligned input: the same move, with the input tiles
// streamed into shared memory by bulk copies (thread 0 copies the block's
// next tile while the block moves this one, two buffers) and the tile's
// kept entries stored 16 bytes at a time, realigned to the output address.
// A tile's kept entries are staged in its own input buffer (every thread
// has its entries in registers by then), so a block needs 32 KiB of shared
// memory and five blocks fit on an SM (three or four buffers per block,
// with fewer blocks, measured slower). The last, partial tile is read with
// plain loads.
constexpr int kTpMoveBufs = 2;
constexpr int kTpMoveMinBlocks = 5;
constexpr size_t kTpMoveSmem = size_t(kTpMoveBufs) * kTpTile * 4;  // input buffers

__global__ void __launch_bounds__(kTpBlock, kTpMoveMinBlocks) k_tp_move_bulk(const uint32_t *in, uint32_t cap, const uint32_t *n_ptr,
                                                            PredDev pred, uint32_t mul, TpLayout L, uint32_t *out) {
    using namespace tma;
    extern __shared__ __align__(128) uint32_t tp_smem[];
    __shared__ __align__(8) uint64_t bar[kTpMoveBufs];
    __shared__ uint32_t s_w[kTpWarps];
    const uint32_t n = tp_live(n_ptr, cap);
    const uint32_t tiles = (n + kTpTile - 1) / kTpTile, full = n / kTpTile;
    const uint32_t G = gridDim.x;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    WsHeader *const err_ws = static_cast<WsHeader *>(L.scan_ws);
    if (t == 0) {
        for (int i = 0; i < kTpMoveBufs; ++i) mbar_init(&bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto fetch = [&](uint32_t tile, int buf) {  // thread 0: tile -> buffer buf
        fence_proxy_async();
        mbar_expect_tx(&bar[buf], uint32_t(kTpTile) * 4u);
        bulk_g2s(tp_smem + size_t(buf) * kTpTile, in + size_t(tile) * kTpTile, uint32_t(kTpTile) * 4u, &bar[buf]);
    };
    // tiles kTpMoveBufs - 1 ahead are in flight
    if (t == 0)
        for (int i = 0; i + 1 < kTpMoveBufs; ++i)
            if (blockIdx.x + uint32_t(i) * G < full) fetch(blockIdx.x + uint32_t(i) * G, i);
    uint32_t k = 0;
    for (uint32_t tile = blockIdx.x; tile < tiles; tile += G, ++k) {
        const int buf = int(k % kTpMoveBufs);
        // the buffer of tile k + B - 1 was last read in the previous trip (before its final barrier)
        const uint32_t ahead = tile + uint32_t(kTpMoveBufs - 1) * G;
        if (t == 0 && ahead < full) fetch(ahead, int((k + kTpMoveBufs - 1) % kTpMoveBufs));
        const uint32_t base = tile * uint32_t(kTpTile);
        const uint32_t valid = min(n - base, uint32_t(kTpTile));
        uint32_t v[kTpIpt];
        if (tile < full) {
            if (!mbar_wait(&bar[buf], (k / kTpMoveBufs) & 1u) && t == 0) record_error(err_ws, kDevErrTimeout, tile);
            const uint32_t *src = tp_smem + size_t(buf) * kTpTile;
#pragma unroll
            for (int r = 0; r < kTpIpt / 4; ++r) {
                const uint4 q = *reinterpret_cast<const uint4 *>(src + (r * kTpBlock + t) * 4);
                v[4 * r] = q.x * mul;
                v[4 * r + 1] = q.y * mul;
                v[4 * r + 2] = q.z * mul;
                v[4 * r + 3] = q.w * mul;
            }
        } else {
            tp_load(in + base, valid, true, mul, v);
        }
        const uint32_t m = tp_mask(pred, v, valid);
        uint32_t packed = 0;
#pragma unroll
        for (int r = 0; r < kTpIpt / 4; ++r) packed += uint32_t(__popc((m >> (4 * r)) & 0xFu)) << (8 * r);
        const uint32_t incl = warp_incl_scan(packed, lane);
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        uint32_t row_base[kTpIpt / 4], warp_off[kTpIpt / 4];
        {
            uint32_t acc = 0;
#pragma unroll
            for (int r = 0; r < kTpIpt / 4; ++r) {
                uint32_t before = 0, total = 0;
#pragma unroll
                for (int w = 0; w < kTpWarps; ++w) {
                    const uint32_t f = (s_w[w] >> (8 * r)) & 0xFFu;
                    if (w < warp) before += f;
                    total += f;
                }
                row_base[r] = acc;
                warp_off[r] = before;
                acc += total;
            }
        }
        const uint32_t excl = incl - packed;
        // (every thread read its entries before the barrier above)
        uint32_t *const s_out = tp_smem + size_t(buf) * kTpTile;
#pragma unroll
        for (int r = 0; r < kTpIpt / 4; ++r) {
            uint32_t pos = row_base[r] + warp_off[r] + ((excl >> (8 * r)) & 0xFFu);
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if ((m >> (4 * r + c)) & 1u) s_out[pos++] = v[4 * r + c];
        }
        __syncthreads();
        // the tile's kept entries: single entries up to the output's next
        // 16-byte boundary, 16-byte chunks (each from two aligned shared
        // loads; index <= 1023 since kept <= 4096), then single entries
        const uint32_t kept = L.counts[tile];
        uint32_t *dst = out + L.offsets[tile];
        const uint32_t to16 = uint32_t((16u - (reinterpret_cast<uintptr_t>(dst) & 15u)) & 15u) >> 2;
        const uint32_t head = to16 < kept ? to16 : kept;
        const uint32_t body = (kept - head) >> 2, t0 = head + 4 * body;
        if (uint32_t(t) < head) dst[t] = s_out[t];
        const uint4 *s4 = reinterpret_cast<const uint4 *>(s_out);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst + head);
        for (uint32_t i = uint32_t(t); i < body; i += kTpBlock) {
            const uint4 x = s4[i];
            if (head == 0) {
                d4[i] = x;
            } else {
                const uint4 y = s4[i + 1];
                d4[i] = head == 1 ? make_uint4(x.y, x.z, x.w, y.x)
                        : head == 2 ? make_uint4(x.z, x.w, y.x, y.y)
                                    : make_uint4(x.w, y.x, y.y, y.z);
            }
        }
        if (uint32_t(t) < kept - t0) dst[t0 + t] = s_out[t0 + t];
        __syncthreads();
    }
}

unsigned tp_grid(uint64_t cap) {
    uint64_t g = tiles_for(cap ? cap : 1, kTpTile);
    const uint64_t lim = uint64_t(device_info().sm_count) * 8;
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
    const TpLayout L = tp_layout(d_ws, tiles, ws_bytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t mul = xform == KA_XFORM_HASH ? kHashMul : 1u;
    const int vec = (reinterpret_cast<uintptr_t>(d_in) & 15u) == 0 ? 1 : 0;
    const unsigned grid = tp_grid(n);
    // the scan's workspace starts zeroed on the first use of this workspace;
    // its epoch tags make later launches safe without clearing
    k_tp_count<<<grid, kTpBlock, 0, st>>>(d_in, uint32_t(n), d_n, p, mul, vec, L);
    s = cuda_status(cudaGetLastError());
    if (s != KA_OK) return s;
    // phase 2: tile offsets; the total of the counts is the result length
    s = launch_exclusive_scan(L.counts, tiles, L.n_tiles, L.offsets, d_count, L.scan_ws, L.scan_ws_bytes,
                              resolve_tile(KA_KERNEL_SCAN, tiles, nullptr), st);
    if (s != KA_OK) return s;
    if (vec) {
        static bool attr_set = false;
        if (!attr_set) {
            if (cudaFuncSetAttribute(k_tp_move_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(kTpMoveSmem)) != cudaSuccess)
                return cuda_status(cudaGetLastError());
            attr_set = true;
        }
        // one wave of resident blocks (each loops over its tiles)
        const uint64_t resident = uint64_t(device_info().sm_count) * kTpMoveMinBlocks;
        const unsigned mgrid = unsigned(std::min<uint64_t>(tiles_for(n ? n : 1, kTpTile), resident));
        k_tp_move_bulk<<<mgrid, kTpBlock, kTpMoveSmem, st>>>(d_in, uint32_t(n), d_n, p, mul, L, d_out);
    } else {
        k_tp_move<<<grid, kTpBlock, 0, st>>>(d_in, uint32_t(n), d_n, p, mul, vec, L, d_out);
    }
    return cuda_status(cudaGetLastError());
}

}  // extern "C"
