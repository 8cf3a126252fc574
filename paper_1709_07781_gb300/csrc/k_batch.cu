// Batched compaction: many independent instances in one persistent launch,
// and batched seeded generation.
//
// Compaction plan kernel (one block per 256 items, chained by a decoupled
// look-back): for every item, the live length (read once, so a count word
// may alias its length word), the canonical predicate, its tile count, and an
// exclusive scan of tile counts -> per-item first tile in one flattened tile
// space; for the TMA kernel, also the map words of small items' tiles.
//
// Register persistent kernel: blocks take flattened tiles by ticket, find
// the owning item with a warp-wide search (first a 32-item window after the
// block's previous item, then a 32-ary search; tickets only grow within a
// block), and run the fused tile body with a look-back that stops at the
// item's first tile. Every status word is indexed by flattened tile, so each
// item owns a contiguous run of the status array.
//
// Generation plan kernel (one block, passes of 4096 items: thread t reads
// items t, t + 1024, t + 2048, t + 3072 of a pass, coalesced, and the tile
// counts go through shared memory so that thread t then scans items
// 4t .. 4t + 3), then a grid-stride generation kernel. Running tile totals
// are 64-bit and saturate at 2^32 - 1 in the stored offsets, above every
// status capacity (the kernels then stop with the workspace error).
#include "ka_batch.cuh"
#include "ka_tile.cuh"

namespace ka {

constexpr int kPlanBlock = 1024;  // the generation plan
constexpr int kPlanIpt = 4;       // items per thread in a pass of it

// A 64-bit tile total stored in a 32-bit offset word: past 2^32 - 1 it stays
// there, above every status capacity (batch_layout keeps that below 2^32 - 1).
__device__ __forceinline__ uint32_t sat32(uint64_t v) { return v > 0xFFFFFFFFull ? 0xFFFFFFFFu : uint32_t(v); }

// Exclusive block scan of v over kPlanBlock threads; *total = block sum.
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t *s_warp, uint64_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint64_t w = s_warp[lane];  // kPlanBlock / 32 == 32 warp sums
        uint64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += y;
        }
        s_warp[lane] = wi - w;
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    const uint64_t r = s_warp[warp] + incl - v;
    *total = s_warp[32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Compaction plan: one block per 256 items, one item per thread. Blocks take
// their index from the workspace ticket, so every lower-numbered block has
// started (the chained scan below waits only on those). A block plans its
// items (live length, canonical predicate, tile count; with `shift`, an
// item's tiles cover its input shifted back to a 16-byte boundary, as the
// TMA kernel copies it), scans their tile counts, and gets the tiles of all
// blocks before it by a decoupled look-back over one status word per block:
// word 0 of status entry p, under the plan's own epoch (the compaction
// kernel that follows draws the next one, and rewrites those words). It then
// writes its items' first tiles and, with `map`, the map word of each tile of
// an item of at most kMapMaxTiles tiles (the item's own thread, one store per
// tile; tagged with the epoch the compaction kernel will draw): the TMA
// kernel's producer finds the items of other tiles by search, which small
// items would defeat. A total past 2^32 - 1 saturates there,
// above every status capacity.
constexpr int kBatchPlanBlock = 256;
constexpr uint32_t kMapMaxTiles = 8;

__device__ __forceinline__ uint32_t sat_add(uint32_t x, uint32_t y) {
    const uint32_t r = x + y;
    return r < x ? 0xFFFFFFFFu : r;
}

__global__ void __launch_bounds__(kBatchPlanBlock) k_batch_plan(const ka_batch_item *items, uint32_t n_items,
                                                                 uint32_t T, BatchLayout L, WsHeader *ws, bool shift,
                                                                 bool map) {
    constexpr int NW = kBatchPlanBlock / 32;
    __shared__ uint32_t s_warp[NW + 1];
    __shared__ uint32_t s_p, s_epoch, s_spin, s_prefix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        uint32_t ep;
        bool last;
        s_p = take_ticket(ws, 0u, &ep, &last);  // the last block starts the next epoch
        s_epoch = ep;
        const uint32_t sl = ws->spin_limit;
        s_spin = sl ? sl : kDefaultSpinLimit;
    }
    __syncthreads();
    const uint32_t p = s_p, epoch = s_epoch, spin = s_spin;
    const uint64_t i = uint64_t(p) * kBatchPlanBlock + uint32_t(tid);
    uint32_t tiles = 0;  // (an item holds at most 2^23 + 1 tiles: 256 items stay below 2^32)
    if (i < n_items) {
        const ka_batch_item it = items[i];
        uint32_t n = it.n;
        if (it.n_ptr) {
            const uint32_t d = *it.n_ptr;
            n = d < n ? d : n;
        }
        ItemPlan pl;
        const bool ok = pred_canon(it.pred, it.param, &pl.pred) == 0 && it.xform <= 1u;
        if (!ok) {
            record_error(ws, 1u, uint32_t(i));  // -KA_E_ARG
            n = 0;
        }
        pl.mul = it.xform == 1u ? kHashMul : 1u;
        pl.n = n;
        const uint32_t lead = shift && n ? uint32_t(reinterpret_cast<uintptr_t>(it.in) & 15u) / 4u : 0u;
        tiles = uint32_t((uint64_t(n) + lead + T - 1) / T);
        pl.tiles = tiles;
        L.plans[i] = pl;
        if (n == 0 && it.count) *it.count = 0u;
    }
    const uint32_t incl = warp_incl_scan(tiles, lane);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = lane < NW ? s_warp[lane] : 0u;
        const uint32_t vi = warp_incl_scan(v, lane);
        if (lane < NW) s_warp[lane] = vi - v;
        if (lane == NW - 1) s_warp[NW] = vi;
    }
    __syncthreads();
    const uint32_t excl = s_warp[warp] + incl - tiles, total = s_warp[NW];
    if (warp == 0) {
        // tiles of the blocks before this one
        uint32_t prefix = 0;
        bool failed = false;
        if (p == 0) {
            if (lane == 0) st_relaxed_u64(status_at(L.status, 0), pack_status(epoch, kFlagInclusive, total));
        } else {
            if (lane == 0) st_relaxed_u64(status_at(L.status, p), pack_status(epoch, kFlagAggregate, total));
            const uint32_t want = epoch & kEpochMask;
            uint32_t hi = p, polls = 0, sleep_ns = 0;  // blocks below hi still to add
            for (;;) {
                // lane l: block hi - 1 - l (none below block 0: an inclusive 0)
                const bool valid = uint32_t(lane) < hi;
                const uint64_t w = valid ? ld_relaxed_u64(status_at(L.status, hi - 1u - uint32_t(lane))) : 0ull;
                const uint32_t f = !valid ? kFlagInclusive
                                          : uint32_t(w >> 34) == want ? uint32_t(w >> 32) & 3u : kFlagInvalid;
                const uint32_t incl_lanes = __ballot_sync(kFull, f == kFlagInclusive);
                const uint32_t ready = __ballot_sync(kFull, f != kFlagInvalid);
                // the nearest inclusive word and every word nearer than it
                const uint32_t upto = incl_lanes ? uint32_t(__ffs(incl_lanes)) - 1u : 31u;
                const uint32_t need = 0xFFFFFFFFu >> (31u - upto);
                if ((ready & need) == need) {
                    uint64_t add = valid && uint32_t(lane) <= upto ? uint32_t(w) : 0u;
#pragma unroll
                    for (int d = 16; d > 0; d >>= 1) add += __shfl_xor_sync(kFull, add, d);
                    prefix = sat_add(prefix, add > 0xFFFFFFFFull ? 0xFFFFFFFFu : uint32_t(add));
                    if (incl_lanes) break;
                    hi -= 32u;
                    continue;
                }
                if (++polls >= spin) {
                    failed = true;
                    if (lane == 0) record_error(ws, kDevErrTimeout, p);
                    break;
                }
                if (polls > 2) {
                    __nanosleep(sleep_ns);
                    sleep_ns = sleep_ns < 256 ? sleep_ns * 2 + 32 : 256;
                }
            }
            // a failed block saturates its successors: the compaction then stops
            if (failed) prefix = 0xFFFFFFFFu;
            if (lane == 0)
                st_relaxed_u64(status_at(L.status, p), pack_status(epoch, kFlagInclusive, sat_add(prefix, total)));
        }
        if (lane == 0) s_prefix = prefix;
    }
    __syncthreads();
    const uint32_t prefix = s_prefix, end = sat_add(prefix, total);
    if (i < n_items) L.tile_off[i] = sat_add(prefix, excl);
    if (i + 1 == n_items) {
        L.tile_off[n_items] = end;
        if (end > L.status_cap) record_error(ws, kDevErrWorkspace, 0);
    }
    if (map && end <= L.status_cap && i < n_items && tiles <= kMapMaxTiles) {
        const uint32_t first = prefix + excl;
        for (uint32_t x = 0; x < tiles; ++x)
            st_relaxed_u64(tile_map_at(L.status, first + x), (uint64_t(epoch + 1u) << 32) | uint32_t(i));
    }
}

template <int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK) k_compact_batch(const BatchArgs a) {
    constexpr int T = BLOCK * IPT;
    __shared__ CompactSmem<BLOCK, IPT> sm;
    __shared__ uint32_t s_ticket, s_epoch, s_total, s_spin, s_item;
    __shared__ const uint32_t *s_in;
    __shared__ uint32_t *s_outp, *s_count;
    __shared__ ItemPlan s_plan;
    __shared__ uint32_t s_first;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    if (tid == 0) {
        s_total = a.L.tile_off[a.n_items];
        const uint32_t sl = a.ws->spin_limit;
        s_spin = sl ? sl : kDefaultSpinLimit;
        s_item = 0;
    }
    __syncthreads();
    const uint32_t total = s_total;
    const uint32_t spin = s_spin;
    if (total > a.L.status_cap) return;

    for (;;) {
        if (tid == 0) {
            uint32_t ep;
            bool last;
            s_ticket = take_ticket(a.ws, total, &ep, &last);
            s_epoch = ep;
        }
        __syncthreads();
        const uint32_t ticket = s_ticket;
        const uint32_t epoch = s_epoch;
        if (ticket >= total) break;
        if (warp == 0) {
            const uint32_t item = find_item(a.L.tile_off, a.n_items, s_item, ticket);
            if ((tid & 31) == 0) {
                s_item = item;
                const ka_batch_item *it = a.items + item;
                s_in = it->in;
                s_outp = it->out;
                s_count = it->count;
                s_plan = a.L.plans[item];
                s_first = a.L.tile_off[item];
            }
        }
        __syncthreads();
        const ItemPlan pl = s_plan;
        const uint32_t first = s_first;
        const uint32_t local = ticket - first;
        const uint32_t base = local * uint32_t(T);
        const uint32_t valid = (pl.n - base) < uint32_t(T) ? (pl.n - base) : uint32_t(T);
        const uint32_t *in = s_in;
        const bool vec_ok = (reinterpret_cast<uintptr_t>(in) & 15u) == 0;
        compact_tile<BLOCK, IPT>(sm, in + base, s_outp, valid, vec_ok, pl.mul, pl.pred, a.L.status, ticket, first,
                                 epoch, spin, a.ws, local == pl.tiles - 1 ? s_count : nullptr);
    }
}

template <int BLOCK, int IPT>
static ka_status launch_batch_shape(const BatchArgs &a, uint32_t grid, cudaStream_t stream) {
    static PerDeviceInt occ_cache;
    const int occupancy = per_device_value(occ_cache, current_device(), [] {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_compact_batch<BLOCK, IPT>, BLOCK, 0);
        return occ > 0 ? occ : 1;
    });
    const uint64_t resident = uint64_t(device_info().sm_count) * occupancy;
    uint64_t g = grid ? grid : resident;
    if (g > resident) g = resident;  // every block resident: tickets need no more
    k_compact_batch<BLOCK, IPT><<<unsigned(g), BLOCK, 0, stream>>>(a);
    return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Batched generation: same plan, fixed 4096-entry tiles, static grid-stride
// over flattened tiles (no ordering between tiles is needed).
constexpr uint32_t kGenTile = 4096;
constexpr int kGenBlock = 256;

__global__ void __launch_bounds__(kPlanBlock) k_gen_plan(const ka_gen_item *items, uint32_t n_items,
                                                          BatchLayout L, WsHeader *ws) {
    __shared__ uint64_t s_warp[33];
    __shared__ uint32_t s_tiles[kPlanBlock * kPlanIpt];
    uint64_t carry = 0;
    for (uint64_t base = 0; base < n_items; base += uint64_t(kPlanBlock) * kPlanIpt) {
        uint32_t nk[kPlanIpt];
#pragma unroll
        for (int k = 0; k < kPlanIpt; ++k) {
            const uint64_t i = base + uint64_t(k) * kPlanBlock + threadIdx.x;
            nk[k] = i < n_items ? items[i].n : 0u;
        }
#pragma unroll
        for (int k = 0; k < kPlanIpt; ++k)
            s_tiles[k * kPlanBlock + threadIdx.x] = uint32_t((uint64_t(nk[k]) + kGenTile - 1) / kGenTile);
        __syncthreads();
        uint32_t v[kPlanIpt];
        uint64_t sum = 0;
#pragma unroll
        for (int k = 0; k < kPlanIpt; ++k) {
            v[k] = s_tiles[threadIdx.x * kPlanIpt + k];
            sum += v[k];
        }
        uint64_t block_total;
        uint64_t off = carry + block_excl_scan(sum, s_warp, &block_total);  // (synchronises: s_tiles reusable)
#pragma unroll
        for (int k = 0; k < kPlanIpt; ++k) {
            const uint64_t i = base + uint64_t(threadIdx.x) * kPlanIpt + k;
            if (i < n_items) L.tile_off[i] = sat32(off);
            off += v[k];
        }
        carry += block_total;
    }
    if (threadIdx.x == 0) {
        L.tile_off[n_items] = sat32(carry);
        if (carry >= 0xFFFFFFFFull) record_error(ws, kDevErrWorkspace, 0);
    }
}

__device__ __forceinline__ uint64_t splitmix64_b(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void __launch_bounds__(kGenBlock) k_generate_batch(const ka_gen_item *items, uint32_t n_items,
                                                               const uint32_t *tile_off) {
    __shared__ uint32_t s_item;
    const uint32_t total = tile_off[n_items];
    if (total == 0xFFFFFFFFu) return;  // the plan kernel has recorded the error
    uint32_t item = 0;
    for (uint32_t t = blockIdx.x; t < total; t += gridDim.x) {
        if (threadIdx.x < 32) {
            const uint32_t f = find_item(tile_off, n_items, item, t);
            if (threadIdx.x == 0) s_item = f;
        }
        __syncthreads();
        item = s_item;
        const ka_gen_item it = items[item];
        // 64-bit positions: an item may hold up to 2^32 - 1 entries
        const uint64_t base = uint64_t(t - tile_off[item]) * kGenTile;
        const uint64_t end = it.n - base < kGenTile ? uint64_t(it.n) : base + kGenTile;
        for (uint64_t e = base + threadIdx.x; e < end; e += kGenBlock)
            it.out[e] = uint32_t(splitmix64_b(it.seed, e) >> 32);
        __syncthreads();
    }
}

}  // namespace ka

using namespace ka;

extern "C" {

ka_status ka_batch_workspace_size(uint32_t max_items, uint64_t total_capacity, const ka_tile *tile,
                                  uint64_t *bytes) {
    if (!bytes || max_items == 0) return KA_E_ARG;
    uint32_t te = 512;
    if (tile && tile->block && tile->ipt) {
        if (!tile_supported_for(KA_KERNEL_BATCH, tile->block, tile->ipt)) return KA_E_ARG;
        te = tile->block * tile->ipt;
    }
    // + 3 entries per item: the TMA shapes shift each item back to a 16-byte boundary
    const uint64_t tiles = tiles_for(total_capacity + 3ull * max_items, te) + max_items + 1;
    *bytes = batch_fixed_bytes(max_items) + round256(tiles * kStatusEntryBytes);
    return KA_OK;
}

ka_status ka_compact_batch(const ka_batch_item *d_items, uint32_t n_items, uint32_t max_items, void *d_ws,
                           uint64_t ws_bytes, const ka_tile *tile, uint32_t grid, void *stream) {
    if (n_items > max_items || max_items == 0) return KA_E_ARG;
    if (n_items && !d_items) return KA_E_ARG;
    if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255u) != 0) return KA_E_ARG;
    if (ws_bytes < batch_fixed_bytes(max_items) + kStatusEntryBytes) return KA_E_WORKSPACE;
    if (n_items == 0) return KA_OK;
    const ka_tile t = resolve_tile(KA_KERNEL_BATCH, kBatchTileKey, tile);
    if (!tile_supported_for(KA_KERNEL_BATCH, t.block, t.ipt)) return KA_E_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    BatchArgs a;
    a.items = d_items;
    a.n_items = n_items;
    a.L = batch_layout(d_ws, ws_bytes, max_items);
    a.ws = static_cast<WsHeader *>(d_ws);
    const bool tma = batch_tma_shape(t.block, t.ipt);
    // one plan block per 256 items, each with a status word of its own
    const uint32_t plan_blocks = (n_items + kBatchPlanBlock - 1) / kBatchPlanBlock;
    if (plan_blocks > a.L.status_cap) return KA_E_WORKSPACE;
    k_batch_plan<<<plan_blocks, kBatchPlanBlock, 0, st>>>(d_items, n_items, t.block * t.ipt, a.L, a.ws, tma, tma);
    ka_status s = cuda_status(cudaGetLastError());
    if (s != KA_OK) return s;
    if (tma) return launch_batch_tma(a, t, grid, st);
    switch (shape_key(t.block, t.ipt)) {
#define KA_CASE(B, I) \
    case shape_key(B, I): return launch_batch_shape<B, I>(a, grid, st);
        KA_FOR_EACH_SHAPE(KA_CASE)
#undef KA_CASE
    default: return KA_E_ARG;
    }
}

ka_status ka_generate_batch(const ka_gen_item *d_items, uint32_t n_items, uint32_t max_items, void *d_ws,
                            uint64_t ws_bytes, void *stream) {
    if (n_items > max_items || max_items == 0) return KA_E_ARG;
    if (n_items && !d_items) return KA_E_ARG;
    if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255u) != 0) return KA_E_ARG;
    if (ws_bytes < batch_fixed_bytes(max_items)) return KA_E_WORKSPACE;
    if (n_items == 0) return KA_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const BatchLayout L = batch_layout(d_ws, ws_bytes, max_items);
    k_gen_plan<<<1, kPlanBlock, 0, st>>>(d_items, n_items, L, static_cast<WsHeader *>(d_ws));
    ka_status s = cuda_status(cudaGetLastError());
    if (s != KA_OK) return s;
    const unsigned grid = unsigned(device_info().sm_count) * 8;
    k_generate_batch<<<grid, kGenBlock, 0, st>>>(d_items, n_items, L.tile_off);
    return cuda_status(cudaGetLastError());
}

}  // extern "C"
