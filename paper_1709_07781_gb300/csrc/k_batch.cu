// Batched compaction: many independent instances in one persistent launch,
// and batched seeded generation.
//
// Plan kernel (one block): for every item, the live length (read once, so a
// count word may alias its length word), the canonical predicate, its tile
// count, and an exclusive scan of tile counts -> per-item first tile in one
// flattened tile space. Persistent kernel: blocks take flattened tiles by
// ticket, find the owning item with a warp-wide search (first a 32-item window
// after the block's previous item, then a 32-ary search; tickets only grow
// within a block), and run the fused tile body with a look-back that stops at
// the item's first tile. Every status word is indexed by flattened tile, so
// each item owns a contiguous segment of the status array.
#include "ka_batch.cuh"
#include "ka_tile.cuh"

namespace ka {

constexpr int kPlanBlock = 1024;

// Exclusive block scan of v over kPlanBlock threads; *total = block sum.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_warp, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t incl = warp_incl_scan(v, lane);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = s_warp[lane];
        const uint32_t wi = warp_incl_scan(w, lane);
        s_warp[lane] = wi - w;
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    const uint32_t r = s_warp[warp] + incl - v;
    *total = s_warp[32];
    __syncthreads();
    return r;
}

// With `shift`, an item's tiles cover its input shifted back to a 16-byte
// boundary (the TMA kernel), so its lead entries count in its tile count.
__global__ void __launch_bounds__(kPlanBlock) k_batch_plan(const ka_batch_item *items, uint32_t n_items,
                                                            uint32_t T, BatchLayout L, WsHeader *ws, bool shift) {
    __shared__ uint32_t s_warp[33];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < n_items; base += kPlanBlock) {
        const uint32_t i = base + threadIdx.x;
        uint32_t tiles = 0;
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
                record_error(ws, 1u, i);  // -KA_E_ARG
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
        uint32_t block_total;
        const uint32_t excl = block_excl_scan(tiles, s_warp, &block_total);
        if (i < n_items) L.tile_off[i] = carry + excl;
        carry += block_total;
    }
    if (threadIdx.x == 0) {
        L.tile_off[n_items] = carry;
        if (carry > L.status_cap) record_error(ws, kDevErrWorkspace, 0);
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
    __shared__ uint32_t s_warp[33];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < n_items; base += kPlanBlock) {
        const uint32_t i = base + threadIdx.x;
        uint32_t tiles = 0;
        if (i < n_items) tiles = uint32_t((uint64_t(items[i].n) + kGenTile - 1) / kGenTile);
        uint32_t block_total;
        const uint32_t excl = block_excl_scan(tiles, s_warp, &block_total);
        if (i < n_items) L.tile_off[i] = carry + excl;
        carry += block_total;
    }
    if (threadIdx.x == 0) L.tile_off[n_items] = carry;
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

namespace ka {
namespace {
// Each flattened tile's item, into the spare word of the tile's status entry
// (the TMA batch kernel's producer reads it ahead of time); one warp per item.
__global__ void k_batch_tile_items(uint32_t n_items, BatchLayout L) {
    const uint32_t total = L.tile_off[n_items];
    if (total > L.status_cap) return;  // the plan kernel has recorded the error
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t stride = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n_items; i += stride) {
        const uint32_t t1 = L.tile_off[i + 1];
        for (uint32_t t = L.tile_off[i] + lane; t < t1; t += 32) *tile_item_at(L.status, t) = i;
    }
}
}  // namespace
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
    const bool tma = tma_shape(t.block, t.ipt);
    k_batch_plan<<<1, kPlanBlock, 0, st>>>(d_items, n_items, t.block * t.ipt, a.L, a.ws, tma);
    ka_status s = cuda_status(cudaGetLastError());
    if (s != KA_OK) return s;
    if (tma) {
        const uint64_t warps_needed = n_items, per_block = kPlanBlock / 32;
        const uint64_t lim = uint64_t(device_info().sm_count) * 8;
        const unsigned g = unsigned(std::min<uint64_t>((warps_needed + per_block - 1) / per_block, lim));
        k_batch_tile_items<<<g, kPlanBlock, 0, st>>>(n_items, a.L);
        s = cuda_status(cudaGetLastError());
        if (s != KA_OK) return s;
        return launch_batch_tma(a, t, grid, st);
    }
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
