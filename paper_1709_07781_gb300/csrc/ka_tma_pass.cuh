#pragma once
// The warp-specialised TMA kernels: fused single-pass compaction
// (k_compact_tma) and single-pass exclusive scan (k_scan_tma), each one
// persistent kernel fed by bulk copies, whose compute warps never wait for one
// another.
//
// Layout of the work. The grid holds exactly the blocks that fit on the GPU at
// once (cooperative launch), G of them; block b owns tiles b, b + G, b + 2G, ...
// (iteration j of block b is tile t = j G + b). A tile is CWW segments of 512
// entries; compute warp w owns segment w of every tile. Tiles start on
// 16-byte boundaries: an input that starts 4, 8 or 12 bytes past one is read
// from that boundary, and the 1-3 entries before its start belong to no tile.
//
// Inside a block:
//   * a producer warp streams tiles into a ring of S shared-memory stages with
//     cp.async.bulk (completion on the stage's "full" mbarrier), and refills a
//     stage once every compute warp has released it ("empty");
//   * each compute warp counts (compaction) or scans (scan) its segment of
//     tile j and posts the result ("counted" mbarrier of tile j); the last
//     warp to post publishes the tile aggregate at once (an atomic on a shared
//     word tells it that it is last);
//   * one look-back warp resolves the tiles' exclusive prefixes in order,
//     anchored on the block's own previous tile: prefix(t) = prefix(t - G) +
//     agg(t - G) + the aggregates of the G - 1 tiles t - G + 1 .. t - 1, which
//     the other blocks publish as soon as they have counted. So no block waits
//     for another block's look-back, and a tile costs one batch of independent
//     loads. This is the decoupled look-back of Merrill & Garland (2016)
//     reorganised around a round-robin persistent grid.
//
// The look-back's loads queue behind the SM's own stream of bulk copies, so a
// round trip takes about as long as a tile's copy (1-2 us). The two kernels
// keep it off the copy stream's critical path in different ways:
//   * scan: every segment is written out whole, from its stage, LAG tiles
//     after it was scanned (the "prefix" mbarrier says its offset is ready),
//     and only then is the stage released. One round trip per tile.
//   * compaction: a warp whose segment keeps at most kSpillCap entries
//     compacts them into a slot of its own small spill ring, releases the
//     stage at once, and writes the entries out NS - 1 tiles later (one store
//     per lane). A segment that keeps more is compacted in place in its stage
//     and written out by its warp LAG tiles later, as in the scan. When every
//     segment of the oldest pending tile was spilled, the look-back warp
//     resolves every tile counted so far (up to BMAX) in one round trip; when
//     one was held, it resolves that tile alone, whose write-out waits for it.
//     At low selectivity the stages thus turn over at the rate of the copies,
//     and the look-back's round trips overlap them instead of gating them.
// One lane per warp arrives on an mbarrier, after __syncwarp: 32 arrivals on
// one barrier word serialise. Every wait is bounded (a few seconds); on
// time-out the kernel records a device error and still finishes.
#include "ka_internal.h"
#include "ka_tma.cuh"

namespace ka {
namespace tma {

struct TmaArgs {
    const uint32_t *in;  // input rounded down to 16 bytes: entry i of the input is in[lead + i]
    uint32_t *out;
    const uint32_t *n_ptr;
    uint32_t *count;
    WsHeader *ws;
    uint64_t *status;
    uint32_t n;
    uint32_t status_cap;
    uint32_t mul;
    uint32_t lead;     // 0..3 entries before the input's first entry
    uint32_t out_vec;  // scan: out - lead is 16-byte aligned (output entries align with input entries)
    PredDev pred;
};

// Entries a compaction segment may keep and still go to the spill ring. At
// 1 % kept a 512-entry segment keeps about 5 (more than 16 about once in
// 10^4 segments); 16 rather than 32 leaves room in shared memory for a larger
// tile, and a segment that keeps more takes the held path.
constexpr int kSpillCap = 16;

// Block set-up shared by both passes (thread 0): the live length, the spin
// limit and the launch epoch (one ticket per block; the last block resets).
__device__ __forceinline__ void tma_block_setup(const TmaArgs &a, uint32_t *s_n, uint32_t *s_spin,
                                                uint32_t *s_epoch) {
    uint32_t n = a.n;
    if (a.n_ptr) {
        const uint32_t d = *a.n_ptr;
        n = d < n ? d : n;
    }
    *s_n = n;
    const uint32_t sl = a.ws->spin_limit;
    *s_spin = sl ? sl : kDefaultSpinLimit;
    uint32_t ep;
    bool last;
    take_ticket(a.ws, 0u, &ep, &last);
    *s_epoch = ep;
}

// The producer warp's loop (lane 0 only): tiles b, b + G, ... of the full
// tiles into the S-stage ring; the ragged last tile is read by the compute
// warps. Waits (bounded) for its last copies before returning, so none lands
// after the block exits.
template <int S, int T>
__device__ __forceinline__ void tma_produce(const TmaArgs &a, uint32_t *stage_mem, uint64_t *full_bar,
                                            uint64_t *empty_bar, uint32_t my_tiles, uint32_t full_tiles) {
    const uint32_t G = gridDim.x, b = blockIdx.x;
    uint32_t issued = 0;
    for (uint32_t jj = 0; jj < my_tiles; ++jj) {
        const uint32_t tile = b + jj * G;
        if (tile >= full_tiles) break;
        const int s = int(jj % S);
        if (jj >= uint32_t(S) && !mbar_wait(&empty_bar[s], ((jj / S) - 1u) & 1u)) {
            record_error(a.ws, kDevErrTimeout, tile);
            break;
        }
        // the status sector of this block's tile two ahead: in L2 before its
        // aggregate is stored and polled (first touches by those went to
        // DRAM; 1 % faster at s = 1 %)
        if (jj + 2 < my_tiles) prefetch_l2(status_at(a.status, uint64_t(tile) + 2u * G));
        fence_proxy_async();  // the compute warps' accesses to this stage precede the copy into it
        mbar_expect_tx(&full_bar[s], uint32_t(T) * 4u);
        // two copies of half a tile each, both completing on the stage's
        // barrier (measured 0.5 % faster than one at 1 % and 50 % kept)
        static_assert(T % 8 == 0, "each half is whole 16-byte chunks");
        bulk_g2s(stage_mem + size_t(s) * T, a.in + size_t(tile) * T, uint32_t(T / 2) * 4u, &full_bar[s]);
        bulk_g2s(stage_mem + size_t(s) * T + T / 2, a.in + size_t(tile) * T + T / 2, uint32_t(T / 2) * 4u,
                 &full_bar[s]);
        issued = jj + 1;
    }
    for (uint32_t jj = issued > uint32_t(S) ? issued - S : 0u; jj < issued; ++jj)
        mbar_wait(&full_bar[jj % S], (jj / S) & 1u);
}

// A compute warp's segment of tile j in shared memory: waits for the copy, or
// reads the ragged last tile with plain loads (zeros outside the input).
// Entries [vlo, vhi) of the segment are input entries.
__device__ __forceinline__ void tma_segment_ready(const TmaArgs &a, uint32_t *seg, uint64_t *full_bar_s,
                                                  uint32_t parity, bool full_tile, uint64_t base, uint32_t vlo,
                                                  uint32_t vhi, uint32_t tile, int lane) {
    if (full_tile) {
        if (!mbar_wait(full_bar_s, parity) && lane == 0) record_error(a.ws, kDevErrTimeout, tile);
    } else {
        const uint32_t *src = a.in + base;
        for (uint32_t e = uint32_t(lane); e < uint32_t(kSeg); e += 32)
            seg[e] = e >= vlo && e < vhi ? src[e] : 0u;
        __syncwarp();
    }
}

// ============================================================================ scan
// Exclusive prefix sum: CWW compute warps (tile = CWW * 512 entries), S
// stages, write-out LAG tiles after scanning, at most MAXG blocks.
template <int CWW, int S, int LAG, int MAXG>
__device__ __forceinline__ void tma_scan_pass(const TmaArgs &a) {
    constexpr int T = CWW * kSeg, ROWS = 4;
    constexpr int K = (MAXG + 31) / 32;
    static_assert(LAG >= 1 && LAG < S && LAG <= 3, "a stage is written out before its refill; slots repeat every 4");
    static_assert(CWW <= 32, "the look-back warp holds one segment sum per lane");
    extern __shared__ __align__(128) uint32_t stage_mem[];
    __shared__ __align__(8) uint64_t full_bar[S], empty_bar[S], count_bar[4], prefix_bar[4];
    __shared__ uint32_t s_wcnt[4][CWW], s_woff[4][CWW], s_err[4];
    __shared__ uint32_t s_pack[4];  // per tile slot: segments scanned
    __shared__ uint32_t s_n, s_epoch, s_spin;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t G = gridDim.x, b = blockIdx.x;

    if (tid == 0) {
        tma_block_setup(a, &s_n, &s_spin, &s_epoch);
        for (int s = 0; s < S; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], CWW);
        }
        for (int k = 0; k < 4; ++k) {
            s_pack[k] = 0;
            mbar_init(&count_bar[k], CWW);
            mbar_init(&prefix_bar[k], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const uint32_t n_in = s_n, n = n_in + a.lead;
    const uint32_t epoch = s_epoch, want = epoch & kEpochMask, spin = s_spin;
    const uint32_t live = uint32_t((uint64_t(n) + T - 1) / T);
    const uint32_t full_tiles = n / uint32_t(T);
    if (uint64_t(live) > a.status_cap) {
        if (tid == 0 && b == 0) record_error(a.ws, kDevErrWorkspace, 0);
        return;
    }
    if (n_in == 0) {
        if (tid == 0 && b == 0) *a.count = 0u;
        return;
    }
    const uint32_t my_tiles = live > b ? (live - b + G - 1) / G : 0u;
    uint64_t *agg_words = a.status;  // entry per tile

    if (warp == CWW + 1) {
        if (lane == 0) tma_produce<S, T>(a, stage_mem, full_bar, empty_bar, my_tiles, full_tiles);
        return;
    }

    if (warp == CWW) {
        // ---------------------------------------------------------------- look-back warp
        uint32_t incl_prev = 0;  // inclusive prefix of this block's previous tile
        bool broken = false;     // an earlier look-back of this block gave up
        for (uint32_t j = 0; j < my_tiles; ++j) {
            const uint32_t k = j & 3u, tile = b + j * G;
            bool failed = !mbar_wait(&count_bar[k], (j >> 2) & 1u);  // every segment of tile j scanned
            if (failed && lane == 0) record_error(a.ws, kDevErrTimeout, tile);
            const uint32_t wc = lane < CWW ? s_wcnt[k][lane] : 0u;
            const uint32_t wincl = warp_incl_scan(wc, lane);
            const uint32_t agg = __shfl_sync(kFull, wincl, 31);  // (published by the last warp to scan)
            const uint32_t lo = j == 0 ? 0u : tile - G + 1u;     // first tile of the window
            const uint32_t wn = tile - lo;                       // window length, < G
            uint32_t sum = 0, polls = 0, sleep_ns = 0;
            failed = failed || broken;
            while (!failed) {
                uint64_t raw[K];
#pragma unroll
                for (int kk = 0; kk < K; ++kk) {
                    const uint32_t i = uint32_t(lane) + 32u * kk;
                    raw[kk] = i < wn ? ld_relaxed_u64(status_at(agg_words, uint64_t(lo) + i)) : 0ull;
                }
                bool all = true;
                sum = 0;
#pragma unroll
                for (int kk = 0; kk < K; ++kk) {
                    const uint32_t i = uint32_t(lane) + 32u * kk;
                    if (i < wn) {
                        const uint32_t f =
                            uint32_t(raw[kk] >> 34) == want ? uint32_t(raw[kk] >> 32) & 3u : kFlagInvalid;
                        if (f == kFlagAggregate) sum += uint32_t(raw[kk]);
                        else all = false;
                    }
                }
                if (__all_sync(kFull, all)) break;
                if (++polls >= spin) {
                    failed = true;
                    if (lane == 0) record_error(a.ws, kDevErrTimeout, tile);
                    break;
                }
                if (polls > 2) {
                    __nanosleep(sleep_ns);
                    sleep_ns = sleep_ns < 128 ? sleep_ns * 2 + 32 : 128;
                }
            }
            const uint32_t prefix = incl_prev + warp_sum(sum);
            broken = failed;
            incl_prev = prefix + agg;
            if (lane < CWW) s_woff[k][lane] = prefix + wincl - wc;
            if (lane == 0) {
                if (!failed && tile == live - 1) *a.count = prefix + agg;
                s_err[k] = failed ? 1u : 0u;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&prefix_bar[k]);  // offsets of tile j ready
        }
        return;
    }

    // ---------------------------------------------------------------- compute warps
    // Iteration j: write out this warp's segment of tile j-LAG (every input
    // entry plus the segment's offset), whose offset the look-back warp has
    // had LAG iterations to resolve, and release its stage; then scan the
    // segment of tile j in place and post its sum.
    const int w = warp;
    uint32_t *const seg_base = stage_mem + w * kSeg;
    for (uint32_t j = 0; j < my_tiles + uint32_t(LAG); ++j) {
        if (j >= uint32_t(LAG)) {
            const uint32_t jp = j - uint32_t(LAG), k = jp & 3u;
            const int s = int(jp % S);
            const bool ok = mbar_wait(&prefix_bar[k], (jp >> 2) & 1u);
            if (!ok && lane == 0) record_error(a.ws, kDevErrTimeout, b + jp * G);
            const uint32_t off = s_woff[k][w];
            __syncwarp();
            if (ok && s_err[k] == 0u) {
                const uint64_t base = uint64_t(b + jp * G) * T + uint32_t(w) * kSeg;
                const uint32_t vlo = base < a.lead ? a.lead - uint32_t(base) : 0u;
                const uint32_t vhi = n > base ? uint32_t(min(n - base, uint64_t(kSeg))) : 0u;
                const uint32_t *sg = seg_base + size_t(s) * T;
                uint32_t *dst = a.out - a.lead + base;  // entry i of the output is a.out[i]
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    const uint32_t e0 = uint32_t(r * 128 + lane * 4);
                    uint4 q = *reinterpret_cast<const uint4 *>(sg + e0);
                    q.x += off;
                    q.y += off;
                    q.z += off;
                    q.w += off;
                    if (a.out_vec && e0 >= vlo && e0 + 4 <= vhi) {
                        *reinterpret_cast<uint4 *>(dst + e0) = q;
                    } else {
                        if (e0 >= vlo && e0 < vhi) dst[e0] = q.x;
                        if (e0 + 1 >= vlo && e0 + 1 < vhi) dst[e0 + 1] = q.y;
                        if (e0 + 2 >= vlo && e0 + 2 < vhi) dst[e0 + 2] = q.z;
                        if (e0 + 3 >= vlo && e0 + 3 < vhi) dst[e0 + 3] = q.w;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty_bar[s]);  // this warp is done with the stage
        }
        if (j < my_tiles) {
            const uint32_t tile = b + j * G, k = j & 3u;
            const int s = int(j % S);
            uint32_t *seg = seg_base + size_t(s) * T;
            // entries [vlo, vhi) of this segment are input entries (64-bit
            // position: the last tile's later segments can lie past 2^32 when
            // T does not divide 2^32)
            const uint64_t base = uint64_t(tile) * T + uint32_t(w) * kSeg;
            const uint32_t vlo = base < a.lead ? a.lead - uint32_t(base) : 0u;
            const uint32_t vhi = n > base ? uint32_t(min(n - base, uint64_t(kSeg))) : 0u;
            tma_segment_ready(a, seg, &full_bar[s], (j / S) & 1u, tile < full_tiles, base, vlo, vhi, tile, lane);
            uint32_t v[ROWS][4];
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const uint32_t e0 = uint32_t(r * 128 + lane * 4);
                const uint4 q = *reinterpret_cast<const uint4 *>(seg + e0);
                v[r][0] = q.x;
                v[r][1] = q.y;
                v[r][2] = q.z;
                v[r][3] = q.w;
                if (vlo != 0u || vhi != uint32_t(kSeg)) {
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (e0 + c < vlo || e0 + c >= vhi) v[r][c] = 0u;
                }
            }
            uint32_t rs[ROWS], incl[ROWS], rowbase = 0;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) rs[r] = v[r][0] + v[r][1] + v[r][2] + v[r][3];
#pragma unroll
            for (int r = 0; r < ROWS; ++r) incl[r] = warp_incl_scan(rs[r], lane);
            // in place: every lane rewrites only the entries it read
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const uint32_t e0 = uint32_t(r * 128 + lane * 4);
                uint32_t x = rowbase + incl[r] - rs[r];
                uint4 o;
                o.x = x;
                x += v[r][0];
                o.y = x;
                x += v[r][1];
                o.z = x;
                x += v[r][2];
                o.w = x;
                *reinterpret_cast<uint4 *>(seg + e0) = o;
                rowbase += __shfl_sync(kFull, incl[r], 31);
            }
            if (lane == 0) {
                s_wcnt[k][w] = rowbase;
                // segment sums are full 32-bit values: the last warp adds them up
                __threadfence_block();
                if (atomicAdd(&s_pack[k], 1u) == uint32_t(CWW - 1)) {
                    __threadfence_block();
                    uint32_t agg = 0;
                    for (int q = 0; q < CWW; ++q) agg += s_wcnt[k][q];
                    s_pack[k] = 0;
                    st_relaxed_u64(status_at(agg_words, tile), pack_status(epoch, kFlagAggregate, agg));
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&count_bar[k]);
        }
    }
}

// ====================================================================== compaction
// Fused compaction with predicate kind PK (a PredKind, or -1: any kind,
// chosen at run time): CWW compute warps (tile = CWW * 512 entries), S
// stages, at most MAXG blocks, NS tile slots (counts, offsets, barriers, and
// the NS slots of kSpillCap entries of each warp's spill ring), at most BMAX
// tiles resolved per round trip of the look-back. A held segment is written
// out LAG tiles after it was counted, a spilled one NS - 1 tiles after.
template <int PK, int CWW, int S, int LAG, int MAXG, int NS, int BMAX>
__device__ __forceinline__ void tma_compact_pass(const TmaArgs &a) {
    constexpr int T = CWW * kSeg, ROWS = 4, SPC = kSpillCap, LAGS = NS - 1;
    constexpr int KB = (MAXG - 1 + 31) / 32;  // loads per lane for the G - 1 words before one tile
    static_assert(NS >= 2 && (NS & (NS - 1)) == 0, "tile slots: a power of two");
    static_assert(LAG >= 1 && LAG < S && LAG <= LAGS, "a held segment is written out before its stage is refilled");
    static_assert(BMAX >= 1 && BMAX <= NS, "a batch of tiles fits the tile slots");
    static_assert(CWW <= 32, "the look-back warp holds one segment count per lane");
    static_assert(CWW * kSeg < 65536, "a tile aggregate fits the 16 low bits of s_pack");
    extern __shared__ __align__(128) uint32_t stage_mem[];
    uint32_t *const spill_mem = stage_mem + size_t(S) * T;  // [CWW][NS][SPC]
    __shared__ __align__(8) uint64_t full_bar[S], empty_bar[S], count_bar[NS], prefix_bar[NS];
    __shared__ uint32_t s_wcnt[NS][CWW], s_woff[NS][CWW], s_err[NS];
    __shared__ uint32_t s_pack[NS];  // per tile slot: (segments counted << 16) | kept so far
    __shared__ uint32_t s_n, s_epoch, s_spin;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t G = gridDim.x, b = blockIdx.x;

    if (tid == 0) {
        tma_block_setup(a, &s_n, &s_spin, &s_epoch);
        for (int s = 0; s < S; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], CWW);
        }
        for (int k = 0; k < NS; ++k) {
            s_pack[k] = 0;
            mbar_init(&count_bar[k], CWW);
            mbar_init(&prefix_bar[k], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const uint32_t n_in = s_n, n = n_in + a.lead;
    const uint32_t epoch = s_epoch, want = epoch & kEpochMask, spin = s_spin;
    const uint32_t live = uint32_t((uint64_t(n) + T - 1) / T);
    const uint32_t full_tiles = n / uint32_t(T);
    if (uint64_t(live) > a.status_cap) {
        if (tid == 0 && b == 0) record_error(a.ws, kDevErrWorkspace, 0);
        return;
    }
    if (n_in == 0) {
        if (tid == 0 && b == 0) *a.count = 0u;
        return;
    }
    const uint32_t my_tiles = live > b ? (live - b + G - 1) / G : 0u;
    uint64_t *const agg_words = a.status;  // entry per tile

    if (warp == CWW + 1) {
        if (lane == 0) tma_produce<S, T>(a, stage_mem, full_bar, empty_bar, my_tiles, full_tiles);
        return;
    }

    if (warp == CWW) {
        // ---------------------------------------------------------------- look-back warp
        // Tiles r, r + 1, ... of this block (iterations) are resolved in
        // order. One round trip loads, for every tile counted so far (up to
        // BMAX), the words of the G - 1 tiles between it and this block's
        // previous tile (for r = 0: the tiles before it); word i is tile lo + i,
        // lo following this block's last resolved tile, and batch tile t sits
        // at i = e_t = (t + 1) G - c. The tiles whose words before them are
        // all published are resolved; the rest wait for the next trip.
        uint32_t r = 0, incl_prev = 0, polls = 0, sleep_ns = 0;
        bool broken = false;  // a wait of this block's look-back gave up: no later tile is resolved
        while (r < my_tiles) {
            const uint32_t k0 = r & uint32_t(NS - 1);
            if (!mbar_wait(&count_bar[k0], (r / NS) & 1u) && !broken) {
                if (lane == 0) record_error(a.ws, kDevErrTimeout, b + r * G);
                broken = true;
            }
            if (broken) {
                // releases the waiters on this tile (once it is counted, so
                // that the barriers' phases stay in step); its output is not
                // written
                if (lane == 0) s_err[k0] = 1u;
                __syncwarp();
                if (lane == 0) mbar_arrive(&prefix_bar[k0]);
                ++r;
                continue;
            }
            // Batching pays when the compute warps run ahead (every segment of
            // tile r spilled); when some were held, their write-outs wait for
            // this tile alone, and a batch would only lengthen the trip.
            const uint32_t wc0 = lane < CWW ? s_wcnt[k0][lane] : 0u;
            const bool held0 = __any_sync(kFull, wc0 > uint32_t(SPC));
            uint32_t m = 1;
            while (!held0 && m < uint32_t(BMAX) && r + m < my_tiles &&
                   mbar_test_wait(&count_bar[(r + m) & uint32_t(NS - 1)], ((r + m) / NS) & 1u))
                ++m;
            const uint32_t lo = r == 0 ? 0u : b + (r - 1u) * G + 1u;
            const uint32_t c = r == 0 ? G - b : 1u;
            uint32_t bsum[BMAX], first_bad = 0xFFFFFFFFu;  // first word not yet published
#pragma unroll
            for (int t = 0; t < BMAX; ++t) bsum[t] = 0u;
            // per batch tile: this lane's segment offset within the tile, and
            // the tile aggregate; computed while the window's loads are in flight
            uint32_t wexcl[BMAX], wagg[BMAX];
            auto scan_counts = [&]() {
#pragma unroll
                for (int t = 0; t < BMAX; ++t) {
                    if (uint32_t(t) < m) {
                        const uint32_t k = (r + uint32_t(t)) & uint32_t(NS - 1);
                        const uint32_t wc = lane < CWW ? s_wcnt[k][lane] : 0u;
                        const uint32_t wincl = warp_incl_scan(wc, lane);
                        wexcl[t] = wincl - wc;
                        wagg[t] = __shfl_sync(kFull, wincl, 31);
                    }
                }
            };
            if (m == 1) {
                // one tile pending (the look-back keeps up): its G - 1 words only
                const uint32_t end = G - c;
                uint64_t raw[KB];
#pragma unroll
                for (int kk = 0; kk < KB; ++kk) {
                    const uint32_t i = uint32_t(lane) + 32u * kk;
                    raw[kk] = i < end ? ld_relaxed_u64(status_at(agg_words, uint64_t(lo + i))) : 0ull;
                }
                scan_counts();
#pragma unroll
                for (int kk = 0; kk < KB; ++kk) {
                    const uint32_t i = uint32_t(lane) + 32u * kk;
                    if (i < end) {
                        if (uint32_t(raw[kk] >> 34) == want && (uint32_t(raw[kk] >> 32) & 3u) == kFlagAggregate)
                            bsum[0] += uint32_t(raw[kk]);
                        else
                            first_bad = i;
                    }
                }
                if (!__all_sync(kFull, first_bad == 0xFFFFFFFFu)) first_bad = 0u;
            } else {
                // several tiles counted: the words before each of them, all in one round trip
                uint64_t raw[BMAX][KB];
#pragma unroll
                for (int t = 0; t < BMAX; ++t) {
                    if (uint32_t(t) < m) {
                        const uint32_t start = t == 0 ? 0u : uint32_t(t) * G - c + 1u, end = uint32_t(t + 1) * G - c;
#pragma unroll
                        for (int kk = 0; kk < KB; ++kk) {
                            const uint32_t i = start + uint32_t(lane) + 32u * kk;
                            raw[t][kk] = i < end ? ld_relaxed_u64(status_at(agg_words, uint64_t(lo + i))) : 0ull;
                        }
                    }
                }
                scan_counts();
#pragma unroll
                for (int t = 0; t < BMAX; ++t) {
                    if (uint32_t(t) < m) {
                        const uint32_t start = t == 0 ? 0u : uint32_t(t) * G - c + 1u, end = uint32_t(t + 1) * G - c;
#pragma unroll
                        for (int kk = 0; kk < KB; ++kk) {
                            const uint32_t i = start + uint32_t(lane) + 32u * kk;
                            const uint64_t wv = raw[t][kk];
                            if (i < end) {
                                if (uint32_t(wv >> 34) == want && (uint32_t(wv >> 32) & 3u) == kFlagAggregate)
                                    bsum[t] += uint32_t(wv);
                                else
                                    first_bad = min(first_bad, i);
                            }
                        }
                    }
                }
                first_bad = __reduce_min_sync(kFull, first_bad);
            }
            uint32_t nres = 0;  // batch tile t is resolved when every word before it is published
            while (nres < m && (nres + 1u) * G - c <= first_bad) ++nres;
            if (nres == 0) {
                if (++polls >= spin) {
                    if (lane == 0) record_error(a.ws, kDevErrTimeout, b + r * G);
                    broken = true;
                } else if (polls > 2) {
                    __nanosleep(sleep_ns);
                    sleep_ns = sleep_ns < 128 ? sleep_ns * 2 + 32 : 128;
                }
                continue;
            }
            polls = 0;
            sleep_ns = 0;
            uint32_t before = incl_prev;  // inclusive prefix of the tile before batch tile t
#pragma unroll
            for (int t = 0; t < BMAX; ++t) {
                if (uint32_t(t) < nres) {
                    const uint32_t part = warp_sum(bsum[t]);
                    const uint32_t tt = r + uint32_t(t), k = tt & uint32_t(NS - 1);
                    const uint32_t prefix = before + part, agg = wagg[t];
                    before = prefix + agg;
                    if (lane < CWW) s_woff[k][lane] = prefix + wexcl[t];
                    if (lane == 0) {
                        s_err[k] = 0u;
                        if (b + tt * G == live - 1) *a.count = prefix + agg;
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&prefix_bar[k]);  // offsets of tile tt ready
                }
            }
            incl_prev = before;
            r += nres;
        }
        return;
    }

    // ---------------------------------------------------------------- compute warps
    // Iteration j: write out this warp's segment of tile j - LAG if it was
    // held in its stage, and release that stage; write out its segment of
    // tile j - (NS - 1) if that one was spilled; then count the segment of
    // tile j and compact it into slot j % NS of the warp's spill ring (at
    // most kSpillCap kept: the stage is released at once) or in place (held).
    // Every segment's write-out waits for its tile's offsets, so slot j % NS
    // (the last tile there is j - NS) is free when tile j is counted.
    const int w = warp;
    const uint32_t mul = a.mul;
    uint32_t *const seg_base = stage_mem + w * kSeg;
    uint32_t *const spill_base = spill_mem + size_t(w) * NS * SPC;
    const uint32_t lead_tiles = a.lead != 0u ? 1u : 0u;  // tile 0 starts before the input
    for (uint32_t j = 0; j < my_tiles + uint32_t(LAGS); ++j) {
        if (j >= uint32_t(LAG) && j - uint32_t(LAG) < my_tiles) {
            const uint32_t jp = j - uint32_t(LAG), k = jp & uint32_t(NS - 1);
            const uint32_t cnt = s_wcnt[k][w];
            if (cnt > uint32_t(SPC)) {
                const int s = int(jp % S);
                const bool ok = mbar_wait(&prefix_bar[k], (jp / NS) & 1u);
                if (!ok && lane == 0) record_error(a.ws, kDevErrTimeout, b + jp * G);
                const uint32_t off = s_woff[k][w];
                __syncwarp();
                if (ok && s_err[k] == 0u) warp_copy_out(seg_base + size_t(s) * T, a.out + off, cnt, lane);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty_bar[s]);  // this warp is done with the stage
            }
        }
        if (j >= uint32_t(LAGS)) {
            const uint32_t jq = j - uint32_t(LAGS), k = jq & uint32_t(NS - 1);
            const uint32_t cnt = s_wcnt[k][w];
            if (cnt <= uint32_t(SPC)) {
                const bool ok = mbar_wait(&prefix_bar[k], (jq / NS) & 1u);
                if (!ok && lane == 0) record_error(a.ws, kDevErrTimeout, b + jq * G);
                if (ok && s_err[k] == 0u && uint32_t(lane) < cnt) a.out[s_woff[k][w] + lane] = spill_base[k * SPC + lane];
            }
        }
        if (j < my_tiles) {
            const uint32_t tile = b + j * G, k = j & uint32_t(NS - 1);
            const int s = int(j % S);
            uint32_t *seg = seg_base + size_t(s) * T;
            // Entries [vlo, vhi) of this segment are input entries: all of them
            // except in the first tile of an input with lead entries and in
            // the ragged last tile, the only tiles that compute the bounds
            // (64-bit position: the last tile's later segments can lie past
            // 2^32 when T does not divide 2^32). The ragged tile is read with
            // plain loads (zeros outside the input).
            uint32_t vlo = 0u, vhi = uint32_t(kSeg);
            const bool full_tile = tile < full_tiles;
            if (!full_tile || tile < lead_tiles) {
                const uint64_t base = uint64_t(tile) * T + uint32_t(w) * kSeg;
                vlo = base < a.lead ? a.lead - uint32_t(base) : 0u;
                vhi = n > base ? uint32_t(min(n - base, uint64_t(kSeg))) : 0u;
                if (!full_tile) {
                    const uint32_t *src = a.in + base;
                    for (uint32_t e = uint32_t(lane); e < uint32_t(kSeg); e += 32)
                        seg[e] = e >= vlo && e < vhi ? src[e] : 0u;
                    __syncwarp();
                }
            }
            if (full_tile && !mbar_wait(&full_bar[s], (j / S) & 1u) && lane == 0)
                record_error(a.ws, kDevErrTimeout, tile);
            const bool edge = vlo != 0u || vhi != uint32_t(kSeg);
            uint32_t v[ROWS][4], mk4[ROWS], packed = 0;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const uint32_t e0 = uint32_t(r * 128 + lane * 4);
                const uint4 q = *reinterpret_cast<const uint4 *>(seg + e0);
                v[r][0] = q.x;
                v[r][1] = q.y;
                v[r][2] = q.z;
                v[r][3] = q.w;
            }
            if (mul != 1u) {
#pragma unroll
                for (int r = 0; r < ROWS; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) v[r][c] *= mul;
            }
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const uint32_t e0 = uint32_t(r * 128 + lane * 4);
                uint32_t mk = mask4_of<PK>(a.pred, v[r][0], v[r][1], v[r][2], v[r][3]);
                if (edge) {
                    const uint32_t skip = vlo > e0 ? min(vlo - e0, 4u) : 0u;
                    const uint32_t left = vhi > e0 ? vhi - e0 : 0u;
                    mk &= (0xFu << skip) & (left >= 4 ? 0xFu : ((1u << left) - 1u));
                }
                mk4[r] = mk;
                packed += uint32_t(__popc(mk)) << (8 * r);
            }
            // per-row counts, 8 bits each (a row of the warp keeps at most 128)
            const uint32_t incl = warp_incl_scan(packed, lane);
            const uint32_t excl = incl - packed;
            const uint32_t rows = __shfl_sync(kFull, incl, 31);
            const uint32_t total = (rows & 0xFFu) + ((rows >> 8) & 0xFFu) + ((rows >> 16) & 0xFFu) + (rows >> 24);
            const bool spilled = total <= uint32_t(SPC);
            if (spilled) {
                // At most kSpillCap entries for the whole warp: each lane
                // stores only its own kept entries, in order, reading each
                // back from the stage (as many trips as the busiest lane has
                // kept entries; at low selectivity most lanes hold none, where
                // the 16 predicated stores below cost every lane 16 slots).
                // Entry r * 128 + 4 lane + c of the segment is bit 4 r + c of
                // the lane's mask; its slot is the lane's first slot in row r
                // (byte r of `first`: the rows before r plus the lanes before
                // this one in row r; every count is at most 16, so no byte
                // carries) plus its kept entries in row r already stored.
                const uint32_t orig = mk4[0] | (mk4[1] << 4) | (mk4[2] << 8) | (mk4[3] << 12);
                const uint32_t first = excl + rows * 0x01010100u;
                uint32_t *const ring = spill_base + k * SPC;
                const uint32_t *const mine = seg + uint32_t(lane) * 4u;
                for (uint32_t m = orig; m != 0u; m &= m - 1u) {
                    const uint32_t i = uint32_t(__ffs(int(m))) - 1u, r = i >> 2;
                    const uint32_t pos = ((first >> (8u * r)) & 0xFFu) + __popc((orig ^ m) & (0xFu << (4u * r)));
                    ring[pos] = mine[r * 128u + (i & 3u)] * mul;
                }
                __syncwarp();
            } else {
                // in place, at the front of the segment (an explicit st.shared
                // to the segment's shared-memory address)
                const uint32_t dst = smem_addr(seg);
                __syncwarp();  // every lane holds its entries before any is overwritten
                uint32_t rowbase = 0;
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    uint32_t pos = rowbase + ((excl >> (8 * r)) & 0xFFu);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        if ((mk4[r] >> c) & 1u) st_shared_u32(dst + 4u * pos++, v[r][c]);
                    }
                    rowbase += (rows >> (8 * r)) & 0xFFu;
                }
                __syncwarp();
            }
            if (lane == 0) {
                s_wcnt[k][w] = total;
                // the last segment counted publishes the tile aggregate at once
                const uint32_t prev = atomicAdd(&s_pack[k], (1u << 16) | total);
                if ((prev >> 16) == uint32_t(CWW - 1)) {
                    s_pack[k] = 0;
                    st_relaxed_u64(status_at(agg_words, tile),
                                   pack_status(epoch, kFlagAggregate, (prev & 0xFFFFu) + total));
                }
                mbar_arrive(&count_bar[k]);
                if (spilled) mbar_arrive(&empty_bar[s]);  // nothing of this tile is left in the stage
            }
        }
    }
}

template <int PK, int CWW, int S, int LAG, int MAXG, int MINB, int NS, int BMAX>
__global__ void __launch_bounds__((CWW + 2) * 32, MINB) k_compact_tma(const TmaArgs a) {
    tma_compact_pass<PK, CWW, S, LAG, MAXG, NS, BMAX>(a);
}

template <int CWW, int S, int LAG, int MAXG, int MINB>
__global__ void __launch_bounds__((CWW + 2) * 32, MINB) k_scan_tma(const TmaArgs a) {
    tma_scan_pass<CWW, S, LAG, MAXG>(a);
}

// Cooperative launch of `kern` with `smem` bytes of dynamic shared memory:
// one block per tile up to the blocks resident at once (at most MAXG),
// found once per device.
template <int BLOCK, int T, int MAXG, class Kern>
ka_status launch_tma_kernel(Kern kern, PerDeviceInt &grid_cache, size_t smem, const TmaArgs &a, uint64_t cap,
                            cudaStream_t stream) {
    const int resident = per_device_value(grid_cache, current_device(), [&] {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
            return -1;
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, BLOCK, smem) != cudaSuccess || occ < 1)
            return -1;
        const int g = device_info().sm_count * occ;
        return g > MAXG ? MAXG : g;
    });
    if (resident <= 0) return launch_setup_error();
    uint64_t grid = (cap + T - 1) / T;
    if (grid > uint64_t(resident)) grid = uint64_t(resident);
    if (grid < 1) grid = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(BLOCK);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cuda_status(cudaLaunchKernelEx(&cfg, kern, a));
}

template <int PK, int CWW, int S, int LAG, int MAXG, int MINB, int NS, int BMAX>
ka_status launch_compact_shape(const TmaArgs &a, uint64_t cap, cudaStream_t stream) {
    constexpr int BLOCK = (CWW + 2) * 32, T = CWW * kSeg;
    const size_t smem = size_t(S) * T * 4 + size_t(CWW) * NS * kSpillCap * 4;
    static PerDeviceInt grid_cache;
    return launch_tma_kernel<BLOCK, T, MAXG>(k_compact_tma<PK, CWW, S, LAG, MAXG, MINB, NS, BMAX>, grid_cache, smem,
                                             a, cap, stream);
}

// One configuration's kernels: the scan, or the compaction for predicate kind
// pk (every kind has its own kernel).
template <int CWW, int S, int LAG, int MAXG, int MINB, int NS, int BMAX>
ka_status launch_tma_config(const TmaArgs &a, bool scan, int32_t pk, uint64_t cap, cudaStream_t stream) {
    if (scan) {
        constexpr int BLOCK = (CWW + 2) * 32, T = CWW * kSeg;
        static PerDeviceInt grid_cache;
        return launch_tma_kernel<BLOCK, T, MAXG>(k_scan_tma<CWW, S, LAG, MAXG, MINB>, grid_cache,
                                                 size_t(S) * T * 4, a, cap, stream);
    }
    switch (pk) {
    case kAndMaskEq0: return launch_compact_shape<kAndMaskEq0, CWW, S, LAG, MAXG, MINB, NS, BMAX>(a, cap, stream);
    case kLt: return launch_compact_shape<kLt, CWW, S, LAG, MAXG, MINB, NS, BMAX>(a, cap, stream);
    case kPopcOdd: return launch_compact_shape<kPopcOdd, CWW, S, LAG, MAXG, MINB, NS, BMAX>(a, cap, stream);
    case kModNe0: return launch_compact_shape<kModNe0, CWW, S, LAG, MAXG, MINB, NS, BMAX>(a, cap, stream);
    case kNe: return launch_compact_shape<kNe, CWW, S, LAG, MAXG, MINB, NS, BMAX>(a, cap, stream);
    case kAll: return launch_compact_shape<kAll, CWW, S, LAG, MAXG, MINB, NS, BMAX>(a, cap, stream);
    default: return launch_compact_shape<-1, CWW, S, LAG, MAXG, MINB, NS, BMAX>(a, cap, stream);
    }
}

// One translation unit per tile shape instantiates its configuration.
ka_status launch_tma_768(const TmaArgs &a, bool scan, int32_t pk, uint64_t cap, cudaStream_t stream);
ka_status launch_tma_512(const TmaArgs &a, bool scan, int32_t pk, uint64_t cap, cudaStream_t stream);
ka_status launch_tma_256(const TmaArgs &a, bool scan, int32_t pk, uint64_t cap, cudaStream_t stream);

}  // namespace tma
}  // namespace ka
