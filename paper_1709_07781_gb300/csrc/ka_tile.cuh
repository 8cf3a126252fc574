// One tile of the fused single-pass compaction, shared by the single-array
// kernel (k_compact.cu) and the batched persistent kernel (k_batch.cu).
//
// One tile = BLOCK threads x IPT entries:
//   1. 16-byte streaming loads in row-major stripes (row r, thread t holds
//      entries [4 (r BLOCK + t), +4)), so every warp load is fully coalesced;
//   2. the keep-test gives a 4-bit mask per row; per-row counts are packed
//      into one 32-bit word (8 bits per row, at most 128 per warp) and scanned
//      across the warp with five shuffles for all rows at once;
//   3. warp 0 scans the per-warp totals (16-bit fields), publishes the tile's
//      count and runs the decoupled look-back for the tile's output offset;
//   4. kept entries go to shared memory at their tile-local offset, then the
//      block writes the contiguous run out[offset, offset + count) with
//      consecutive threads on consecutive words.
#pragma once

#include "ka_dev.cuh"

namespace ka {

template <int BLOCK, int IPT>
struct CompactSmem {
    static constexpr int T = BLOCK * IPT;
    static constexpr int WARPS = BLOCK / 32;
    uint32_t out[T];
    uint32_t wtot[WARPS];
    uint64_t wexcl[WARPS];
    uint64_t tot;
    uint32_t prefix;
    uint32_t err;
};

__device__ __forceinline__ uint32_t sum16x4(uint64_t t) {
    return uint32_t(t & 0xFFFFu) + uint32_t((t >> 16) & 0xFFFFu) + uint32_t((t >> 32) & 0xFFFFu) +
           uint32_t(t >> 48);
}

// Compacts the `valid` entries at tile_in (the tile's first entry) into
// out[prefix ...], where prefix is found by look-back over status[first_tile,
// tile). If count_last is not null this is the last tile of its array and the
// total length is written there. Called by every thread of the block; starts
// and ends with the block's shared memory free for the next tile (the caller
// places a barrier before the next call).
template <int BLOCK, int IPT>
__device__ __forceinline__ void compact_tile(CompactSmem<BLOCK, IPT> &sm, const uint32_t *tile_in, uint32_t *out,
                                             uint32_t valid, bool vec_ok, uint32_t mul, const PredDev &pred,
                                             uint64_t *status, uint32_t tile, uint32_t first_tile, uint32_t epoch,
                                             uint32_t spin, WsHeader *ws, uint32_t *count_last) {
    constexpr int T = BLOCK * IPT;
    constexpr int ROWS = IPT / 4;
    constexpr int WARPS = BLOCK / 32;
    static_assert(ROWS >= 1 && ROWS <= 4, "8-bit row fields hold at most 4 rows");
    static_assert(WARPS <= 32, "16-bit block fields hold at most 32 warps x 128 (and one warp scans them)");
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;

    uint32_t v[ROWS][4];
    uint32_t m[ROWS];
    if (valid == uint32_t(T) && vec_ok) {
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const uint4 q = ld_stream_v4(tile_in + (r * BLOCK + tid) * 4);
            v[r][0] = q.x * mul;
            v[r][1] = q.y * mul;
            v[r][2] = q.z * mul;
            v[r][3] = q.w * mul;
        }
    } else {
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t idx = uint32_t(r * BLOCK + tid) * 4 + j;
                v[r][j] = idx < valid ? ld_stream_u32(tile_in + idx) * mul : 0u;
            }
        }
    }
    uint32_t packed = 0;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        uint32_t mk = pred_mask4(pred, v[r][0], v[r][1], v[r][2], v[r][3]);
        if (valid != uint32_t(T)) {
            const uint32_t idx0 = uint32_t(r * BLOCK + tid) * 4;
            const uint32_t left = valid > idx0 ? valid - idx0 : 0u;
            mk &= left >= 4 ? 0xFu : ((1u << left) - 1u);
        }
        m[r] = mk;
        packed += __popc(mk) << (8 * r);
    }
    const uint32_t incl = warp_incl_scan(packed, lane);
    const uint32_t lane_excl = incl - packed;
    if (lane == 31) sm.wtot[warp] = incl;
    __syncthreads();

    if (warp == 0) {
        const uint64_t wt = lane < WARPS ? spread8to16(sm.wtot[lane]) : 0ull;
        const uint64_t wincl = warp_incl_scan64(wt, lane, WARPS);
        if (lane < WARPS) sm.wexcl[lane] = wincl - wt;
        const uint64_t tot = __shfl_sync(kFull, wincl, WARPS - 1);
        const uint32_t agg = sum16x4(tot);
        bool err;
        const uint32_t prefix = lookback_warp(status, tile, first_tile, epoch, agg, spin, ws, &err);
        if (lane == 0) {
            sm.tot = tot;
            sm.prefix = prefix;
            sm.err = err ? 1u : 0u;
            if (!err && count_last) *count_last = prefix + agg;
        }
    }
    __syncthreads();
    const uint64_t tot = sm.tot;
    const uint32_t prefix = sm.prefix;
    const bool err = sm.err != 0u;
    if (!err) {
        const uint64_t wex = sm.wexcl[warp];
        uint32_t rowbase = 0;
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            uint32_t off = rowbase + uint32_t((wex >> (16 * r)) & 0xFFFFu) + ((lane_excl >> (8 * r)) & 0xFFu);
            const uint32_t mk = m[r];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if ((mk >> j) & 1u) {
                    sm.out[off] = v[r][j];
                    ++off;
                }
            }
            rowbase += uint32_t((tot >> (16 * r)) & 0xFFFFu);
        }
    }
    __syncthreads();
    if (!err) {
        const uint32_t agg = sum16x4(tot);
        uint32_t *dst = out + prefix;
        for (uint32_t k = tid; k < agg; k += BLOCK) dst[k] = sm.out[k];
    }
}

}  // namespace ka
