// Batched compaction on the warp-specialised TMA design: many independent
// instances in one persistent launch.
//
// The plan kernel has laid every item's tiles out in one flattened tile
// space (item i owns tiles tile_off[i] .. tile_off[i+1]-1, each item shifted
// back to a 16-byte boundary as in the single-array kernel). Block b of the G
// resident blocks takes flattened tiles b, b + G, b + 2G, ... The roles are
// those of the single-array kernel:
//   * the producer warp finds the item of each of its tiles (the plan's map
//     word for a tile of a small item, else a warp-wide search starting at
//     the item of its previous tile; both two tiles ahead, so that no load
//     waits between two copies), records the item's
//     output, count word, predicate and the tile's valid range in the
//     stage's slot, and copies the tile with cp.async.bulk; a partial last
//     tile is copied rounded up to 16 bytes (the extra entries lie in the
//     same 16-byte chunk as the item's last entry and are masked);
//   * compute warps count, compact in place and write out their segments
//     with the stage's item parameters;
//   * the look-back warp resolves the tile's prefix within its item: if the
//     block's previous tile (t - G) belongs to the same item, it anchors on
//     that tile's inclusive prefix and adds the G - 1 aggregates in between;
//     otherwise it adds the aggregates from the item's first tile to t - 1
//     (fewer than G). The look-back writes the item's count at its last tile.
#include "ka_batch.cuh"
#include "ka_tma.cuh"

namespace ka {
namespace {

using namespace tma;

struct TileInfo {  // one per stage
    uint32_t *out;    // item output
    uint32_t *count;  // item count word
    PredDev pred;
    uint32_t mul;
    uint32_t first;  // item's first flattened tile
    uint32_t last;   // item's last flattened tile
    uint32_t vlo;    // entries before the item's start at the front of this tile
    uint32_t vhi;    // entries of this tile, from its start, up to the item's end
};

}  // namespace

template <int CWW, int S, int LAG, int MAXG, int MINB>
__global__ void __launch_bounds__((CWW + 2) * 32, MINB) k_batch_tma(const BatchArgs a) {
    constexpr int T = CWW * kSeg;
    constexpr int K = (MAXG + 31) / 32;
    static_assert(LAG >= 1 && LAG < S && LAG <= 3, "a stage is written out before its refill; slots repeat every 4");
    static_assert(CWW <= 32, "the look-back warp holds one segment count per lane");
    static_assert(CWW * kSeg < 65536, "a tile aggregate fits the 16 low bits of s_pack");
    extern __shared__ __align__(128) uint32_t stage_mem[];
    __shared__ __align__(8) uint64_t full_bar[S], empty_bar[S], count_bar[4], prefix_bar[4];
    __shared__ TileInfo s_info[S];
    __shared__ uint32_t s_wcnt[4][CWW], s_woff[4][CWW], s_err[4];
    __shared__ uint32_t s_pack[4];
    __shared__ uint32_t s_total, s_epoch, s_spin;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t G = gridDim.x, b = blockIdx.x;
    const BatchLayout &L = a.L;

    if (tid == 0) {
        s_total = L.tile_off[a.n_items];
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
    const uint32_t total = s_total, epoch = s_epoch, want = epoch & kEpochMask, spin = s_spin;
    if (total > L.status_cap) return;  // the plan kernel has recorded the error
    const uint32_t my_tiles = total > b ? (total - b + G - 1) / G : 0u;
    uint64_t *agg_words = L.status;  // entry per flattened tile

    if (warp == CWW + 1) {
        // ------------------------------------------------------------------ producer warp
        // Tiles b, b + G, ... lie in non-decreasing items. The item of tile
        // jj + 2 is found while tile jj is issued: its map word (read three
        // tiles ahead, which also brings the tile's status sector into L2
        // before its aggregate is stored and polled), written by the plan for
        // tiles of small items, or else ballots over the window
        // tile_off[i + 1 .. i + 128] after the item i of tile jj + 1, loaded
        // one tile earlier (a 32-ary search from there when the window ends
        // first; G tiles of items that are not small span fewer items).
        // Tile jj + 1's item and plan records are loaded then as well, one
        // word per lane: lanes 0-11 the item (48 bytes), 12-19 the plan (32
        // bytes), 20 the item's first tile. So no dependent load sits between
        // two copies. A map word is a hint: a tile outside its item's tiles
        // (a word left by another use of the workspace) is found by search.
        constexpr int kWin = 4;  // window words per lane
        struct Window {
            uint32_t v[kWin];
        };
        uint32_t issued = 0;
        bool stop = false;
        auto window = [&](uint32_t i) -> Window {  // this lane's words of the window after item i
            Window w;
#pragma unroll
            for (int k = 0; k < kWin; ++k) {
                const uint32_t j = i + 1u + uint32_t(lane) + 32u * k;
                w.v[k] = j <= a.n_items && j > i ? L.tile_off[j] : 0xFFFFFFFFu;
            }
            return w;
        };
        auto resolve = [&](const Window &w, uint32_t i, uint32_t jj) -> uint32_t {  // item of tile jj (every lane)
            if (jj >= my_tiles) return i;
            const uint32_t t = b + jj * G;
#pragma unroll
            for (int k = 0; k < kWin; ++k) {
                const uint32_t bal = __ballot_sync(kFull, w.v[k] > t);
                if (bal) return i + 32u * k + uint32_t(__ffs(bal)) - 1u;
            }
            return find_item(L.tile_off, a.n_items, i + 32u * kWin, t);
        };
        auto record = [&](uint32_t i) -> uint32_t {  // this lane's word of item i's records
            i = i < a.n_items ? i : 0u;
            if (lane < 12) return reinterpret_cast<const uint32_t *>(a.items + i)[lane];
            if (lane < 20) return reinterpret_cast<const uint32_t *>(L.plans + i)[lane - 12];
            return lane == 20 ? L.tile_off[i] : 0u;
        };
        const uint32_t map_tag = epoch;  // the plan's epoch plus one: this launch's
        auto map_of = [&](uint32_t jj) -> uint64_t {  // tile jj's map word (every lane)
            return jj < my_tiles ? ld_relaxed_u64(tile_map_at(L.status, b + jj * G)) : 0ull;
        };
        auto mapped = [&](uint64_t m) { return uint32_t(m >> 32) == map_tag; };
        const uint64_t m0 = map_of(0), m1 = map_of(1);
        uint64_t m2 = map_of(2);
        const uint32_t it0 = !my_tiles ? 0u : mapped(m0) ? uint32_t(m0) : find_item(L.tile_off, a.n_items, 0u, b);
        uint32_t it1 = mapped(m1) ? uint32_t(m1) : resolve(window(it0), it0, 1u);  // item of tile jj + 1
        Window win = window(it1);                                                // window after it
        uint32_t rec = record(it0);
        for (uint32_t jj = 0; jj < my_tiles && !stop; ++jj) {
            const uint32_t tile = b + jj * G;
            const uint32_t it2 = mapped(m2) ? uint32_t(m2) : resolve(win, it1, jj + 2u);
            m2 = map_of(jj + 3u);
            const uint32_t rec_next = jj + 1 < my_tiles ? record(it1) : 0u;
            if (jj + 2 < my_tiles) win = window(it2);
            // a hint that does not hold: the item by search
            if (tile - __shfl_sync(kFull, rec, 20) >= __shfl_sync(kFull, rec, 19))
                rec = record(find_item(L.tile_off, a.n_items, 0u, tile));
            // tile jj's records from the lanes that hold them
            auto w = [&](int l) { return __shfl_sync(kFull, rec, l); };
            const uint64_t in_u = uint64_t(w(0)) | (uint64_t(w(1)) << 32);
            const uint64_t out_u = uint64_t(w(2)) | (uint64_t(w(3)) << 32);
            const uint64_t cnt_u = uint64_t(w(6)) | (uint64_t(w(7)) << 32);
            ItemPlan pl;
            pl.pred.kind = int32_t(w(12));
            pl.pred.a = w(13);
            pl.pred.b = w(14);
            pl.pred.c = w(15);
            pl.pred.d = w(16);
            pl.mul = w(17);
            pl.n = w(18);
            pl.tiles = w(19);
            const uint32_t first = w(20);
            if (lane == 0) {
                const uint32_t *in = reinterpret_cast<const uint32_t *>(in_u);
                const uint32_t lead = uint32_t(in_u & 15u) / 4u;
                const uint32_t local = tile - first;
                // 64-bit: an item of up to 2^32 - 1 entries plus its lead
                const uint64_t nv = uint64_t(pl.n) + lead, start = uint64_t(local) * T;
                TileInfo ti;
                ti.out = reinterpret_cast<uint32_t *>(out_u);
                ti.count = reinterpret_cast<uint32_t *>(cnt_u);
                ti.pred = pl.pred;
                ti.mul = pl.mul;
                ti.first = first;
                ti.last = first + pl.tiles - 1;
                ti.vlo = local == 0 ? lead : 0u;
                ti.vhi = uint32_t(min(nv - start, uint64_t(T)));
                const uint32_t *src = in - lead + start;
                const uint32_t bytes = (ti.vhi * 4u + 15u) & ~15u;
                const int s = int(jj % S);
                if (jj >= uint32_t(S) && !mbar_wait(&empty_bar[s], ((jj / S) - 1u) & 1u)) {
                    record_error(a.ws, kDevErrTimeout, tile);
                    stop = true;
                } else {
                    s_info[s] = ti;
                    fence_proxy_async();  // the compute warps' writes to this stage precede the copy into it
                    mbar_expect_tx(&full_bar[s], bytes);
                    bulk_g2s(stage_mem + size_t(s) * T, src, bytes, &full_bar[s]);
                    issued = jj + 1;
                }
            }
            stop = __shfl_sync(kFull, stop ? 1u : 0u, 0) != 0u;
            rec = rec_next;
            it1 = it2;
        }
        // Every copy has been consumed unless a wait gave up; wait (bounded)
        // for the last one on each stage so none lands after the block exits.
        if (lane == 0)
            for (uint32_t jj = issued > uint32_t(S) ? issued - S : 0u; jj < issued; ++jj)
                mbar_wait(&full_bar[jj % S], (jj / S) & 1u);
        return;
    }

    if (warp == CWW) {
        // ---------------------------------------------------------------- look-back warp
        uint32_t incl_prev = 0;  // inclusive prefix (within its item) of this block's previous tile
        bool broken = false;     // the look-back of that tile gave up
        for (uint32_t j = 0; j < my_tiles; ++j) {
            const uint32_t k = j & 3u, tile = b + j * G;
            const int s = int(j % S);
            bool failed = !mbar_wait(&count_bar[k], (j >> 2) & 1u);  // every segment of tile j counted
            if (failed && lane == 0) record_error(a.ws, kDevErrTimeout, tile);
            const uint32_t first = s_info[s].first, last = s_info[s].last;
            uint32_t *const count = s_info[s].count;
            const uint32_t wc = lane < CWW ? s_wcnt[k][lane] : 0u;
            const uint32_t wincl = warp_incl_scan(wc, lane);
            const uint32_t agg = __shfl_sync(kFull, wincl, 31);
            const bool anchored = tile - first >= G;  // the block's previous tile is in the same item
            const uint32_t lo = anchored ? tile - G + 1u : first;
            const uint32_t wn = tile - lo;  // window length, < G
            uint32_t sum = 0, polls = 0, sleep_ns = 0;
            failed = failed || (anchored && broken);
            while (!failed && wn) {
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
            const uint32_t prefix = (anchored ? incl_prev : 0u) + warp_sum(sum);
            broken = failed;
            incl_prev = prefix + agg;
            if (lane < CWW) s_woff[k][lane] = prefix + wincl - wc;
            if (lane == 0) {
                if (!failed && tile == last) *count = prefix + agg;
                s_err[k] = failed ? 1u : 0u;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&prefix_bar[k]);  // offsets of tile j ready
        }
        return;
    }

    // ---------------------------------------------------------------- compute warps
    const int w = warp;
    uint32_t *const seg_base = stage_mem + w * kSeg;
    for (uint32_t j = 0; j < my_tiles + uint32_t(LAG); ++j) {
        if (j >= uint32_t(LAG)) {
            const uint32_t jp = j - uint32_t(LAG), k = jp & 3u;
            const int s = int(jp % S);
            const bool ok = mbar_wait(&prefix_bar[k], (jp >> 2) & 1u);
            if (!ok && lane == 0) record_error(a.ws, kDevErrTimeout, b + jp * G);
            const uint32_t cnt = s_wcnt[k][w];
            const uint32_t off = s_woff[k][w];
            uint32_t *const out = s_info[s].out;
            __syncwarp();
            if (ok && s_err[k] == 0u && cnt != 0u) warp_copy_out(seg_base + size_t(s) * T, out + off, cnt, lane);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty_bar[s]);  // this warp is done with the stage
        }
        if (j < my_tiles) {
            const uint32_t tile = b + j * G, k = j & 3u;
            const int s = int(j % S);
            uint32_t *seg = seg_base + size_t(s) * T;
            if (!mbar_wait(&full_bar[s], (j / S) & 1u) && lane == 0) record_error(a.ws, kDevErrTimeout, tile);
            const TileInfo &ti = s_info[s];
            const uint32_t mul = ti.mul;
            // entries [vlo, vhi) of this segment are the item's entries
            const uint32_t base = uint32_t(w) * kSeg;
            const uint32_t vlo = ti.vlo > base ? ti.vlo - base : 0u;
            const uint32_t vhi = ti.vhi > base ? min(ti.vhi - base, uint32_t(kSeg)) : 0u;
            uint32_t rowbase = 0;
            if (vhi > vlo) {
                // the tile's item fixes the predicate: one branch per tile into
                // a count loop made for that predicate kind
                switch (ti.pred.kind) {
                case kAndMaskEq0: rowbase = compact_segment<kAndMaskEq0>(seg, ti.pred, mul, vlo, vhi, lane); break;
                case kLt: rowbase = compact_segment<kLt>(seg, ti.pred, mul, vlo, vhi, lane); break;
                case kPopcOdd: rowbase = compact_segment<kPopcOdd>(seg, ti.pred, mul, vlo, vhi, lane); break;
                case kModNe0: rowbase = compact_segment<kModNe0>(seg, ti.pred, mul, vlo, vhi, lane); break;
                case kNe: rowbase = compact_segment<kNe>(seg, ti.pred, mul, vlo, vhi, lane); break;
                default: rowbase = compact_segment<kAll>(seg, ti.pred, mul, vlo, vhi, lane); break;
                }
            }
            if (lane == 0) {
                s_wcnt[k][w] = rowbase;
                const uint32_t prev = atomicAdd(&s_pack[k], (1u << 16) | rowbase);
                if ((prev >> 16) == uint32_t(CWW - 1)) {
                    s_pack[k] = 0;
                    st_relaxed_u64(status_at(agg_words, tile),
                                   pack_status(epoch, kFlagAggregate, (prev & 0xFFFFu) + rowbase));
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&count_bar[k]);
        }
    }
}

namespace {

template <int CWW, int S, int LAG, int MAXG, int MINB>
ka_status launch_batch_tma_shape(const BatchArgs &a, uint32_t grid, cudaStream_t stream) {
    constexpr int BLOCK = (CWW + 2) * 32, T = CWW * kSeg;
    const size_t smem = size_t(S) * T * 4;
    auto kern = k_batch_tma<CWW, S, LAG, MAXG, MINB>;
    // per device: the shared-memory attribute holds for the current device only
    static PerDeviceInt grid_cache;
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
    const uint32_t g = grid && grid < uint32_t(resident) ? grid : uint32_t(resident);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g);
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

}  // namespace

bool batch_tma_shape(uint32_t block, uint32_t ipt) {
    return ipt == 16 && (block == 256 || block == 512 || block == 704 || block == 768);
}

ka_status launch_batch_tma(const BatchArgs &a, ka_tile tile, uint32_t grid, cudaStream_t stream) {
    // (704, 16): 22 compute warps and five stages of 44 KiB (220 KiB), the
    // largest tile with five stages in shared memory. With a write-out 3
    // tiles after counting, two stages are in flight at once: 0.89 of HBM on
    // 4096 log-uniform instances, against 0.81-0.83 for the four- and
    // three-stage shapes, which keep one in flight.
    if (tile.block == 704) return launch_batch_tma_shape<22, 5, 3, 160, 1>(a, grid, stream);
    if (tile.block == 768) return launch_batch_tma_shape<24, 4, 3, 160, 1>(a, grid, stream);
    if (tile.block == 512) return launch_batch_tma_shape<16, 3, 2, 320, 2>(a, grid, stream);
    return launch_batch_tma_shape<8, 4, 2, 480, 3>(a, grid, stream);
}

}  // namespace ka
