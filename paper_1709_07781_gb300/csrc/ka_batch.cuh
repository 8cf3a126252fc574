// Layout shared by the batched compaction kernels: per-item plan records,
// the flattened tile space (item i owns tiles tile_off[i] .. tile_off[i+1]-1),
// the status array indexed by flattened tile, and the warp-wide search for
// the item that owns a tile.
#pragma once

#include "ka_internal.h"

namespace ka {

struct ItemPlan {  // 32 bytes
    PredDev pred;
    uint32_t mul;
    uint32_t n;
    uint32_t tiles;
};
static_assert(sizeof(ItemPlan) == 32, "plan record is 32 bytes");

struct BatchLayout {
    uint32_t *tile_off;  // [max_items + 1]
    ItemPlan *plans;     // [max_items]
    uint64_t *status;    // [status_cap]
    uint32_t status_cap;
};

inline uint64_t round256(uint64_t b) { return (b + 255) / 256 * 256; }

inline uint64_t batch_fixed_bytes(uint32_t max_items) {
    return kWsHeaderBytes + round256((uint64_t(max_items) + 1) * 4) + round256(uint64_t(max_items) * 32);
}

inline BatchLayout batch_layout(void *ws, uint64_t ws_bytes, uint32_t max_items) {
    BatchLayout L;
    char *p = static_cast<char *>(ws) + kWsHeaderBytes;
    L.tile_off = reinterpret_cast<uint32_t *>(p);
    p += round256((uint64_t(max_items) + 1) * 4);
    L.plans = reinterpret_cast<ItemPlan *>(p);
    p += round256(uint64_t(max_items) * 32);
    L.status = reinterpret_cast<uint64_t *>(p);
    const uint64_t fixed = batch_fixed_bytes(max_items);
    const uint64_t entries = ws_bytes > fixed ? (ws_bytes - fixed) / kStatusEntryBytes : 0;
    // below 2^32 - 1: a saturated tile total (the plan's overflow mark) exceeds it
    L.status_cap = entries > 0xFFFFFFFEull ? 0xFFFFFFFEu : uint32_t(entries);
    return L;
}

// Item owning flattened tile `ticket`: the largest i with tile_off[i] <= ticket.
// Precondition: tile_off[lo] <= ticket < tile_off[n_items]. Called by a full warp.
__device__ __forceinline__ uint32_t find_item(const uint32_t *tile_off, uint32_t n_items, uint32_t lo,
                                              uint32_t ticket) {
    const int lane = threadIdx.x & 31;
    {
        const uint32_t j = lo + 1 + lane;
        const uint32_t v = j <= n_items ? tile_off[j] : 0xFFFFFFFFu;
        const uint32_t b = __ballot_sync(kFull, v > ticket);
        if (b) return lo + __ffs(b) - 1;
    }
    lo += 32;
    uint32_t hi = n_items;
    while (hi - lo > 1) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint64_t jj = uint64_t(lo) + uint64_t(lane + 1) * step;
        const uint32_t j = jj < hi ? uint32_t(jj) : hi;
        const uint32_t v = tile_off[j];
        const uint32_t b = __ballot_sync(kFull, v > ticket);
        const uint32_t f = __ffs(b) - 1;
        const uint64_t nh = uint64_t(lo) + uint64_t(f + 1) * step;
        const uint32_t new_hi = nh < hi ? uint32_t(nh) : hi;
        lo = f == 0 ? lo : lo + f * step;
        hi = new_hi;
    }
    return lo;
}

#ifdef __CUDACC__
// Map word of flattened tile t: (plan epoch << 32) | item, in the spare
// second word of the tile's status entry (the first is the tile's status).
// The plan kernel writes it for the tiles of small items; the TMA batch
// kernel's producer reads it ahead and trusts it only under the plan epoch
// of the same call.
__device__ __forceinline__ uint64_t *tile_map_at(uint64_t *status, uint32_t t) {
    return status + uint64_t(t) * 4u + 1u;
}
#endif

struct BatchArgs {
    const ka_batch_item *items;
    uint32_t n_items;
    BatchLayout L;
    WsHeader *ws;
};

// The TMA batch kernel (tile shapes (256, 16), (512, 16), (768, 16)); the plan
// must have been made with the lead shift (plan_shift = true).
ka_status launch_batch_tma(const BatchArgs &a, ka_tile tile, uint32_t grid, cudaStream_t stream);

}  // namespace ka
