#pragma once
// The warp-specialised TMA kernel: fused single-pass compaction, and
// single-pass exclusive scan, as one
// persistent, warp-specialised kernel fed by TMA bulk copies, whose compute
// warps never wait for one another. The scan (k_scan_tma) differs only in
// what a compute warp does with its segment: it scans it in place and later
// writes every entry plus the segment's offset (below, "count" and "kept"
// read "sum").
//
// Layout of the work. The grid holds exactly the blocks that fit on the GPU at
// once (cooperative launch), G of them; block b owns tiles b, b + G, b + 2G, ...
// (iteration j of block b is tile t = j G + b). A tile is CWW segments of 512
// entries; compute warp w owns segment w of every tile. Tiles start on
// 16-byte boundaries: an input that starts 4, 8 or 12 bytes past one is read
// from that boundary, and the 1-3 entries before its start belong to no tile.
//
// Inside a block:
//   * a producer warp streams tiles into a ring of S shared-memory stages
//     with cp.async.bulk (completion on the stage's "full" mbarrier), and
//     refills a stage once every compute warp has released it ("empty");
//   * each compute warp counts the kept entries of its segment of tile j,
//     compacts them in place at the front of the segment (a warp-local
//     operation) and posts its count ("counted" mbarrier of tile j); the
//     last warp to post publishes the tile aggregate at once (an atomic on a
//     shared word tells it that it is last). LAG iterations later the warp
//     copies its compacted segment to the output at the offset the look-back
//     warp left for it ("prefix" mbarrier) and releases the stage;
//   * one look-back warp resolves the tiles' exclusive prefixes in order.
//     The prefix of tile t is anchored on the block's own previous tile,
//     prefix(t) = prefix(t - G) + agg(t - G) + the aggregates of the G - 1
//     tiles t - G + 1 .. t - 1, so a tile costs one batch of independent
//     loads of aggregates, which the other blocks publish as soon as they
//     have counted, and no block waits for another block's look-back.
// This is the decoupled look-back of Merrill & Garland (2016) reorganised
// around a round-robin persistent grid. The look-back's loads queue behind
// the SM's own stream of copies, so its round trip is about a microsecond;
// the LAG tiles between counting and writing out hide it, and large tiles
// (one 24-warp block per SM) keep the number of round trips low.
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

// One pass of the warp-specialised kernel. SCAN = false: fused compaction
// with predicate kind PK (a PredKind, or -1: any kind, chosen at run time)
// (count, compact in place, write out the kept entries). SCAN = true:
// exclusive prefix sum (scan each segment in place, write every entry plus
// its offset; a.count receives the total). CWW compute warps (tile = CWW *
// 512 entries), S stages, write-out LAG tiles after counting, at most MAXG
// blocks.
template <bool SCAN, int PK, int CWW, int S, int LAG, int MAXG>
__device__ __forceinline__ void tma_pass(const TmaArgs &a) {
    constexpr int T = CWW * kSeg, ROWS = 4;
    constexpr int K = (MAXG + 31) / 32;
    static_assert(LAG >= 1 && LAG < S && LAG <= 3, "a stage is written out before its refill; slots repeat every 4");
    static_assert(CWW <= 32, "the look-back warp holds one segment count per lane");
    static_assert(CWW * kSeg < 65536, "a tile aggregate fits the 16 low bits of s_pack");
    extern __shared__ __align__(128) uint32_t stage_mem[];
    __shared__ __align__(8) uint64_t full_bar[S], empty_bar[S], count_bar[4], prefix_bar[4];
    __shared__ uint32_t s_wcnt[4][CWW], s_woff[4][CWW], s_err[4];
    __shared__ uint32_t s_pack[4];  // per tile slot: (segments counted << 16) | kept so far
    __shared__ uint32_t s_n, s_epoch, s_spin;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t G = gridDim.x, b = blockIdx.x;

    if (tid == 0) {
        uint32_t n = a.n;
        if (a.n_ptr) {
            const uint32_t d = *a.n_ptr;
            n = d < n ? d : n;
        }
        s_n = n;
        const uint32_t sl = a.ws->spin_limit;
        s_spin = sl ? sl : kDefaultSpinLimit;
        uint32_t ep;
        bool last;
        take_ticket(a.ws, 0u, &ep, &last);  // one ticket per block: the epoch; the last block resets
        s_epoch = ep;
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
    // Tiles cover the input shifted by `lead` entries, so that every tile
    // starts on a 16-byte boundary; the lead entries belong to no tile.
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
        // ------------------------------------------------------------------ producer warp
        if (lane != 0) return;
        uint32_t issued = 0;
        for (uint32_t jj = 0; jj < my_tiles; ++jj) {
            const uint32_t tile = b + jj * G;
            if (tile >= full_tiles) break;  // the ragged last tile is read by the compute warps
            const int s = int(jj % S);
            if (jj >= uint32_t(S) && !mbar_wait(&empty_bar[s], ((jj / S) - 1u) & 1u)) {
                record_error(a.ws, kDevErrTimeout, tile);
                break;
            }
            fence_proxy_async();  // the compute warps' writes to this stage precede the copy into it
            mbar_expect_tx(&full_bar[s], uint32_t(T) * 4u);
            bulk_g2s(stage_mem + size_t(s) * T, a.in + size_t(tile) * T, uint32_t(T) * 4u, &full_bar[s]);
            issued = jj + 1;
        }
        // Every copy has been consumed unless a wait gave up; wait (bounded)
        // for the last one on each stage so none lands after the block exits.
        for (uint32_t jj = issued > uint32_t(S) ? issued - S : 0u; jj < issued; ++jj)
            mbar_wait(&full_bar[jj % S], (jj / S) & 1u);
        return;
    }

    if (warp == CWW) {
        // ---------------------------------------------------------------- look-back warp
        // The prefix of tile t = j G + b is anchored on this block's own
        // previous tile: prefix(t) = prefix(t - G) + agg(t - G) + the
        // aggregates of the G - 1 tiles in between, t - G + 1 .. t - 1 (for
        // j = 0: the aggregates of tiles 0 .. t - 1). The anchor is a
        // register, so a tile costs one batch of independent loads of
        // aggregates, which other blocks publish as soon as they have counted,
        // and no block waits for another block's look-back.
        uint32_t incl_prev = 0;  // inclusive prefix of this block's previous tile
        bool broken = false;     // an earlier look-back of this block gave up
        for (uint32_t j = 0; j < my_tiles; ++j) {
            const uint32_t k = j & 3u, tile = b + j * G;
            bool failed = !mbar_wait(&count_bar[k], (j >> 2) & 1u);  // every segment of tile j counted
            if (failed && lane == 0) record_error(a.ws, kDevErrTimeout, tile);
            const uint32_t wc = lane < CWW ? s_wcnt[k][lane] : 0u;
            const uint32_t wincl = warp_incl_scan(wc, lane);
            const uint32_t agg = __shfl_sync(kFull, wincl, 31);  // (published by the last warp to count)
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
    // Iteration j: write out this warp's segment of tile j-LAG, whose offsets
    // the look-back warp has had LAG iterations to resolve, and release its
    // stage; then count the segment of tile j, compact it in place and post
    // the count.
    const int w = warp;
    const uint32_t mul = a.mul;
    uint32_t *const seg_base = stage_mem + w * kSeg;
    for (uint32_t j = 0; j < my_tiles + uint32_t(LAG); ++j) {
        if (j >= uint32_t(LAG)) {
            const uint32_t jp = j - uint32_t(LAG), k = jp & 3u;
            const int s = int(jp % S);
            const bool ok = mbar_wait(&prefix_bar[k], (jp >> 2) & 1u);
            if (!ok && lane == 0) record_error(a.ws, kDevErrTimeout, b + jp * G);
            const uint32_t cnt = s_wcnt[k][w];
            const uint32_t off = s_woff[k][w];
            __syncwarp();
            if constexpr (!SCAN) {
                if (ok && s_err[k] == 0u && cnt != 0u)
                    warp_copy_out(seg_base + size_t(s) * T, a.out + off, cnt, lane);
            } else if (ok && s_err[k] == 0u) {
                // every input entry of the segment, plus the segment's offset, at its own index
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
            if (tile < full_tiles) {
                if (!mbar_wait(&full_bar[s], (j / S) & 1u) && lane == 0) record_error(a.ws, kDevErrTimeout, tile);
            } else {
                // ragged last tile: plain loads of this segment, zeros outside the input
                const uint32_t *src = a.in + base;
                for (uint32_t e = uint32_t(lane); e < uint32_t(kSeg); e += 32)
                    seg[e] = e >= vlo && e < vhi ? src[e] : 0u;
                __syncwarp();
            }
            uint32_t rowbase = 0;  // kept entries (compaction) or sum (scan) of this segment
            if constexpr (SCAN) {
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
                uint32_t rs[ROWS], incl[ROWS];
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
            } else {
                uint32_t v[ROWS][4], m[ROWS], packed = 0;
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
                    if (vlo != 0u || vhi != uint32_t(kSeg)) {
                        const uint32_t skip = vlo > e0 ? min(vlo - e0, 4u) : 0u;
                        const uint32_t left = vhi > e0 ? vhi - e0 : 0u;
                        mk &= (0xFu << skip) & (left >= 4 ? 0xFu : ((1u << left) - 1u));
                    }
                    m[r] = mk;
                    packed += uint32_t(__popc(mk)) << (8 * r);
                }
                // per-row counts, 8 bits each (a row of the warp keeps at most 128)
                const uint32_t incl = warp_incl_scan(packed, lane);
                const uint32_t excl = incl - packed;
                const uint32_t rows = __shfl_sync(kFull, incl, 31);
                __syncwarp();  // every lane holds its entries before any is overwritten
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    uint32_t pos = rowbase + ((excl >> (8 * r)) & 0xFFu);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        if ((m[r] >> c) & 1u) seg[pos++] = v[r][c];
                    }
                    rowbase += (rows >> (8 * r)) & 0xFFu;
                }
            }
            if (lane == 0) {
                s_wcnt[k][w] = rowbase;
                // the last segment counted publishes the tile aggregate at once
                if constexpr (!SCAN) {
                    const uint32_t prev = atomicAdd(&s_pack[k], (1u << 16) | rowbase);
                    if ((prev >> 16) == uint32_t(CWW - 1)) {
                        s_pack[k] = 0;
                        st_relaxed_u64(status_at(agg_words, tile),
                                       pack_status(epoch, kFlagAggregate, (prev & 0xFFFFu) + rowbase));
                    }
                } else {  // segment sums are full 32-bit values: the last warp adds them up
                    __threadfence_block();
                    if (atomicAdd(&s_pack[k], 1u) == uint32_t(CWW - 1)) {
                        __threadfence_block();
                        uint32_t agg = 0;
                        for (int q = 0; q < CWW; ++q) agg += s_wcnt[k][q];
                        s_pack[k] = 0;
                        st_relaxed_u64(status_at(agg_words, tile), pack_status(epoch, kFlagAggregate, agg));
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&count_bar[k]);
        }
    }
}

template <int PK, int CWW, int S, int LAG, int MAXG, int MINB>
__global__ void __launch_bounds__((CWW + 2) * 32, MINB) k_compact_tma(const TmaArgs a) {
    tma_pass<false, PK, CWW, S, LAG, MAXG>(a);
}

template <int CWW, int S, int LAG, int MAXG, int MINB>
__global__ void __launch_bounds__((CWW + 2) * 32, MINB) k_scan_tma(const TmaArgs a) {
    tma_pass<true, kAll, CWW, S, LAG, MAXG>(a);
}

template <bool SCAN, int PK, int CWW, int S, int LAG, int MAXG, int MINB>
ka_status launch_tma_shape(const TmaArgs &a, uint64_t cap, cudaStream_t stream) {
    constexpr int BLOCK = (CWW + 2) * 32, T = CWW * kSeg;
    const size_t smem = size_t(S) * T * 4;
    auto kern = SCAN ? k_scan_tma<CWW, S, LAG, MAXG, MINB> : k_compact_tma<PK, CWW, S, LAG, MAXG, MINB>;
    static int grid_cached = 0;
    if (grid_cached == 0) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
            return cuda_status(cudaGetLastError());
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, BLOCK, smem) != cudaSuccess || occ < 1)
            return cuda_status(cudaGetLastError());
        int g = device_info().sm_count * occ;
        grid_cached = g > MAXG ? MAXG : g;
    }
    uint64_t grid = (cap + T - 1) / T;
    if (grid > uint64_t(grid_cached)) grid = grid_cached;
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

// One configuration's kernels: the scan, or the compaction for predicate kind
// pk (every kind has its own kernel).
template <int CWW, int S, int LAG, int MAXG, int MINB>
ka_status launch_tma_config(const TmaArgs &a, bool scan, int32_t pk, uint64_t cap, cudaStream_t stream) {
    if (scan) return launch_tma_shape<true, kAll, CWW, S, LAG, MAXG, MINB>(a, cap, stream);
    switch (pk) {
    case kAndMaskEq0: return launch_tma_shape<false, kAndMaskEq0, CWW, S, LAG, MAXG, MINB>(a, cap, stream);
    case kLt: return launch_tma_shape<false, kLt, CWW, S, LAG, MAXG, MINB>(a, cap, stream);
    case kPopcOdd: return launch_tma_shape<false, kPopcOdd, CWW, S, LAG, MAXG, MINB>(a, cap, stream);
    case kModNe0: return launch_tma_shape<false, kModNe0, CWW, S, LAG, MAXG, MINB>(a, cap, stream);
    case kNe: return launch_tma_shape<false, kNe, CWW, S, LAG, MAXG, MINB>(a, cap, stream);
    case kAll: return launch_tma_shape<false, kAll, CWW, S, LAG, MAXG, MINB>(a, cap, stream);
    default: return launch_tma_shape<false, -1, CWW, S, LAG, MAXG, MINB>(a, cap, stream);
    }
}

// One translation unit per tile shape instantiates its configuration.
ka_status launch_tma_768(const TmaArgs &a, bool scan, int32_t pk, uint64_t cap, cudaStream_t stream);
ka_status launch_tma_512(const TmaArgs &a, bool scan, int32_t pk, uint64_t cap, cudaStream_t stream);
ka_status launch_tma_256(const TmaArgs &a, bool scan, int32_t pk, uint64_t cap, cudaStream_t stream);

}  // namespace tma
}  // namespace ka
