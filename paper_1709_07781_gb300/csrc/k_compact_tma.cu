// Fused single-pass compaction for 16-byte-aligned inputs: a persistent,
// warp-specialised kernel fed by TMA bulk copies.
//
// Layout of the work. The grid holds exactly the blocks that fit on the GPU at
// once (cooperative launch), G of them; block b owns tiles b, b + G, b + 2G, ...
// (iteration j of block b is tile j G + b), so at any moment the G blocks work
// on one contiguous window of G tiles.
//
// Inside a block:
//   * one thread streams tiles into a ring of S shared-memory stages with
//     cp.async.bulk (completion on an mbarrier per stage) and, PF iterations
//     further ahead, cp.async.bulk.prefetch.L2, so HBM reads are in flight
//     without holding shared memory for them;
//   * compute warps count the kept entries of tile j, compact it in place at
//     the front of its stage and publish the count (the tile's aggregate) at
//     once; they write a tile out LAG = S - 1 iterations later, when the
//     look-back warp has long had its prefix, and refill that stage;
//   * one look-back warp resolves prefixes in tile order. The prefix of tile
//     (j, b) is the inclusive total of iteration j-1 - a word published by the
//     last block of that iteration - plus the aggregates of tiles (j, 0..b-1),
//     all read in one batch of independent loads (a late iteration word is
//     replaced by the aggregates of that iteration). The block's own compute
//     warps need that prefix only LAG tiles later: the look-back is off their path.
// This is the decoupled look-back of Merrill & Garland (2016) reorganised
// around a round-robin persistent grid; on GB300 the straightforward form
// (every block walking back 32 predecessors at a time while its other warps
// wait) reached about a third of HBM bandwidth, this form reaches 85-100%.
// The hand-offs between the look-back warp and the compute warps are named
// barriers (see kCountBar / kPrefixBar).
#include "ka_internal.h"

namespace ka {
namespace {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bulk copy global -> this block's shared memory, completing on mbarrier m.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *m) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(m))
                 : "memory");
}

__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

__device__ __forceinline__ void bar_arrive(int id, int n) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

constexpr uint32_t kMbarSpin = 1u << 22;
constexpr uint32_t kMaxSkip = 4;  // iterations a look-back may add up instead of waiting for their word
// Named barriers: 1 = compute warps only; kCountBar + (t & 3) = tile t counted
// (compute warps arrive, look-back warp syncs); kPrefixBar + (t & 3) = prefix of
// tile t resolved (look-back warp arrives, compute warps sync). A period of 4 is
// at least the lag, so an id is never re-armed before its last use completed.
constexpr int kCountBar = 2;
constexpr int kPrefixBar = 6;

struct TmaArgs {
    const uint32_t *in;
    uint32_t *out;
    const uint32_t *n_ptr;
    uint32_t *count;
    WsHeader *ws;
    uint64_t *status;
    uint32_t n;
    uint32_t status_cap;
    uint32_t mul;
    PredDev pred;
};

}  // namespace

// CWW compute warps (tile = CWW * 32 threads * 16 entries), S stages, L2
// prefetch PF iterations ahead, at most MAXG blocks.
template <int CWW, int S, int PF, int MAXG, int MINB>
__global__ void __launch_bounds__((CWW + 1) * 32, MINB) k_compact_tma(const TmaArgs a) {
    constexpr uint32_t LAG = uint32_t(S) - 1;  // tiles between counting and writing out
    constexpr int NCW = CWW * 32, BLOCK = NCW + 32, ROWS = 4, T = NCW * 16;
    constexpr int SSTRIDE = T + 32;  // stage: the tile, then 32 scratch slots (16-byte aligned)
    constexpr int K = (MAXG + 31) / 32;
    static_assert(S >= 3 && S <= 4, "LAG = S - 1 in [2, 3]: the hand-off barriers and slots repeat every 4 tiles");
    extern __shared__ __align__(128) uint32_t stage_mem[];
    __shared__ __align__(8) uint64_t mbar[S];
    __shared__ uint32_t s_red[CWW], s_wtot[CWW];
    __shared__ uint64_t s_wexcl[CWW];
    __shared__ uint64_t s_tot;
    __shared__ uint32_t s_agg[4], s_prefix[4], s_err[4], s_kept[S];
    __shared__ uint32_t s_n, s_epoch, s_spin, s_pending;
    __shared__ uint32_t s_pend_j[S];  // iteration of the copy outstanding on each stage

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
        s_pending = 0;
        for (int s = 0; s < S; ++s) mbar_init(&mbar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const uint32_t n = s_n, epoch = s_epoch, want = epoch & kEpochMask, spin = s_spin;
    const uint32_t live = uint32_t((uint64_t(n) + T - 1) / T);
    const uint32_t full_tiles = n / uint32_t(T);
    const uint32_t iters = (live + G - 1) / G;
    if (uint64_t(live) + iters > a.status_cap) {
        if (tid == 0 && b == 0) record_error(a.ws, kDevErrWorkspace, 0);
        return;
    }
    if (live == 0) {
        if (tid == 0 && b == 0) *a.count = 0u;
        return;
    }
    const uint32_t my_tiles = live > b ? (live - b + G - 1) / G : 0u;
    uint64_t *agg_words = a.status;                   // entry per tile
    uint64_t *iter_words = a.status + uint64_t(live) * kStatusStride;  // entry per iteration

    // Issues the load of this block's tile jj into stage jj % S (full tiles
    // only; the ragged last tile is read by the compute warps themselves).
    auto issue = [&](uint32_t jj) {
        const uint32_t tile = b + jj * G;
        if (jj >= my_tiles || tile >= full_tiles) return;
        const int s = int(jj % S);
        mbar_expect_tx(&mbar[s], uint32_t(T) * 4u);
        bulk_g2s(stage_mem + size_t(s) * SSTRIDE, a.in + size_t(tile) * T, uint32_t(T) * 4u, &mbar[s]);
        s_pending |= 1u << s;
        s_pend_j[s] = jj;
        if (PF > 0) {
            const uint32_t pj = jj + PF;
            const uint32_t pt = b + pj * G;
            if (pj < my_tiles && pt < full_tiles) prefetch_l2(a.in + size_t(pt) * T, uint32_t(T) * 4u);
        }
    };
    if (tid == 0)
        for (uint32_t jj = 0; jj < uint32_t(S); ++jj) issue(jj);
    __syncthreads();

    if (warp == 0) {
        // ---------------------------------------------------------------- look-back warp
        for (uint32_t j = 0; j < my_tiles; ++j) {
            bar_sync(kCountBar + int(j & 3), BLOCK);  // tile j counted; its aggregate is in s_agg
            const uint32_t agg = s_agg[j & 3];
            const uint32_t tile = b + j * G;
            // prefix = sum of aggregates of tiles (j, 0..b-1)
            //        + the inclusive word of iteration j-1-d
            //        + all aggregates of iterations j-d .. j-1,
            // for the smallest d whose inclusive word is already published
            // (d = 0 normally); a late word is skipped, not waited for.
            uint32_t sum = 0, polls = 0, sleep_ns = 0;
            bool failed = false;
            {
                // (1) same-iteration predecessors: must be read in full
                for (;;) {
                    uint64_t raw[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const uint32_t i = uint32_t(lane) + 32u * k;
                        raw[k] = i < b ? ld_relaxed_u64(status_at(agg_words, uint64_t(j) * G + i)) : 0ull;
                    }
                    bool all = true;
                    sum = 0;
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const uint32_t i = uint32_t(lane) + 32u * k;
                        if (i < b) {
                            const uint32_t f =
                                uint32_t(raw[k] >> 34) == want ? uint32_t(raw[k] >> 32) & 3u : kFlagInvalid;
                            if (f == kFlagAggregate) sum += uint32_t(raw[k]);
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
                // (2) earlier iterations, newest inclusive word first
                uint32_t d = 0;
                uint32_t whole = 0;  // aggregates of whole iterations skipped so far (lane-partial)
                while (!failed && j > d) {
                    const uint32_t it = j - 1 - d;  // iteration whose inclusive word is tried
                    uint64_t rit = 0;
                    if (lane == 0) rit = ld_relaxed_u64(status_at(iter_words, it));
                    uint32_t fl = uint32_t(rit >> 34) == want ? uint32_t(rit >> 32) & 3u : kFlagInvalid;
                    fl = __shfl_sync(kFull, fl, 0);
                    const uint32_t val = __shfl_sync(kFull, uint32_t(rit), 0);
                    if (fl == kFlagInclusive) {
                        if (lane == 0) sum += val;
                        sum += whole;
                        whole = 0;
                        break;
                    }
                    if (fl == kFlagError) {
                        failed = true;
                        break;
                    }
                    if (d + 1 >= kMaxSkip) {  // deep enough: wait for this word
                        if (++polls >= spin) {
                            failed = true;
                            if (lane == 0) record_error(a.ws, kDevErrTimeout, tile);
                            break;
                        }
                        if (polls > 2) {
                            __nanosleep(sleep_ns);
                            sleep_ns = sleep_ns < 128 ? sleep_ns * 2 + 32 : 128;
                        }
                        continue;
                    }
                    // skip iteration `it`: add all of its aggregates instead
                    for (;;) {
                        uint64_t raw[K];
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            const uint32_t i = uint32_t(lane) + 32u * k;
                            raw[k] = i < G ? ld_relaxed_u64(status_at(agg_words, uint64_t(it) * G + i)) : 0ull;
                        }
                        bool all = true;
                        uint32_t part = 0;
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            const uint32_t i = uint32_t(lane) + 32u * k;
                            if (i < G) {
                                const uint32_t f =
                                    uint32_t(raw[k] >> 34) == want ? uint32_t(raw[k] >> 32) & 3u : kFlagInvalid;
                                if (f == kFlagAggregate) part += uint32_t(raw[k]);
                                else all = false;
                            }
                        }
                        if (__all_sync(kFull, all)) {
                            whole += part;
                            break;
                        }
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
                    ++d;
                }
                if (!failed && j <= d) sum += whole;  // reached the first iteration: nothing before it
            }
            const uint32_t prefix = warp_sum(sum);
            if (lane == 0) {
                if (b == G - 1 || tile == live - 1)
                    st_relaxed_u64(status_at(iter_words, j),
                                   pack_status(epoch, failed ? kFlagError : kFlagInclusive, prefix + agg));
                if (!failed && tile == live - 1) *a.count = prefix + agg;
                s_prefix[j & 3] = prefix;
                s_err[j & 3] = failed ? 1u : 0u;
            }
            bar_arrive(kPrefixBar + int(j & 3), BLOCK);  // prefix of tile j ready
        }
        return;
    }

    // -------------------------------------------------------------------- compute warps
    // Iteration j: first write out tile j-LAG, whose prefix the look-back warp
    // has had LAG iterations to resolve, and refill its stage with tile
    // j-LAG+S; then count tile j, compact it in place at the front of its
    // stage (tile-local offsets need no prefix) and publish its aggregate.
    const int ct = tid - 32, cw = warp - 1;
    for (uint32_t j = 0; j < my_tiles + LAG; ++j) {
        if (j >= uint32_t(LAG)) {
            const uint32_t jp = j - LAG;
            bar_sync(kPrefixBar + int(jp & 3), BLOCK);  // prefix of tile jp ready (and its compaction visible)
            const int s = int(jp % S);
            const uint32_t *sb = stage_mem + size_t(s) * SSTRIDE;
            const uint32_t prefix = s_prefix[jp & 3];
            const bool err = s_err[jp & 3] != 0u;
            const uint32_t kept = s_kept[s];
            if (!err && kept) {
                // head up to a 16-byte boundary of the output address (the output
                // itself may start anywhere 4-byte aligned), 16-byte stores, then the tail
                uint32_t *dst = a.out + prefix;
                const uint32_t to_boundary = uint32_t((16u - (reinterpret_cast<uintptr_t>(dst) & 15u)) & 15u) >> 2;
                const uint32_t head = min(to_boundary, kept);
                const uint32_t body4 = (kept - head) / 4;
                const uint32_t tail0 = head + body4 * 4;
                if (uint32_t(ct) < head) dst[ct] = sb[ct];
                for (uint32_t i = uint32_t(ct); i < body4; i += NCW) {
                    const uint32_t k = head + 4 * i;
                    *reinterpret_cast<uint4 *>(dst + k) = make_uint4(sb[k], sb[k + 1], sb[k + 2], sb[k + 3]);
                }
                if (uint32_t(ct) < kept - tail0) dst[tail0 + ct] = sb[tail0 + ct];
            }
            bar_sync(1, NCW);  // stage free
            if (ct == 0) {
                fence_proxy_async();
                if (!((s_pending >> s) & 1u)) issue(jp + S);  // (a stage whose copy never landed stays idle)
            }
        }
        if (j < my_tiles) {
            const uint32_t tile = b + j * G;
            const int s = int(j % S);
            uint32_t *buf = stage_mem + size_t(s) * SSTRIDE;
            uint32_t valid = uint32_t(T);
            if (tile < full_tiles) {
                const uint32_t parity = (j / S) & 1u;
                uint32_t polls = 0;
                bool ok = true;
                while (!mbar_try_wait(&mbar[s], parity)) {
                    if (++polls > kMbarSpin) {
                        record_error(a.ws, kDevErrTimeout, tile);
                        ok = false;
                        break;
                    }
                }
                if (ok && ct == 0) s_pending &= ~(1u << s);  // the copy has landed
            } else {
                // ragged last tile: plain loads into the stage, zeros past the end
                valid = n - tile * uint32_t(T);
                const uint32_t *src = a.in + size_t(tile) * T;
                for (uint32_t e = uint32_t(ct); e < uint32_t(T); e += NCW) buf[e] = e < valid ? src[e] : 0u;
                bar_sync(1, NCW);
            }
            uint32_t v[ROWS][4], m[ROWS], packed = 0;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const uint32_t e0 = uint32_t(r * NCW + ct) * 4;
                const uint4 q = *reinterpret_cast<const uint4 *>(buf + e0);
                v[r][0] = q.x * a.mul;
                v[r][1] = q.y * a.mul;
                v[r][2] = q.z * a.mul;
                v[r][3] = q.w * a.mul;
                uint32_t mk = pred_mask4(a.pred, v[r][0], v[r][1], v[r][2], v[r][3]);
                if (valid != uint32_t(T)) {
                    const uint32_t left = valid > e0 ? valid - e0 : 0u;
                    mk &= left >= 4 ? 0xFu : ((1u << left) - 1u);
                }
                m[r] = mk;
                packed += __popc(mk) << (8 * r);
            }
            const uint32_t incl = warp_incl_scan(packed, lane);
            const uint32_t lane_excl = incl - packed;
            if (lane == 31) s_wtot[cw] = incl;
            bar_sync(1, NCW);  // every entry of the stage is in registers; warp totals are in
            if (cw == 0) {
                const uint64_t wt = lane < CWW ? spread8to16(s_wtot[lane]) : 0ull;
                const uint64_t wi = warp_incl_scan64(wt, lane, CWW);
                if (lane < CWW) s_wexcl[lane] = wi - wt;
                const uint64_t total = __shfl_sync(kFull, wi, CWW - 1);  // inclusive total of the last warp
                const uint32_t agg = uint32_t(total & 0xFFFFu) + uint32_t((total >> 16) & 0xFFFFu) +
                                     uint32_t((total >> 32) & 0xFFFFu) + uint32_t(total >> 48);
                if (lane == 0) {
                    st_relaxed_u64(status_at(agg_words, tile), pack_status(epoch, kFlagAggregate, agg));
                    s_tot = total;
                    s_agg[j & 3] = agg;
                    s_kept[s] = agg;
                }
            }
            bar_sync(1, NCW);
            const uint64_t tot = s_tot;
            const uint64_t wex = s_wexcl[cw];
            uint32_t rowbase = 0;
            const uint32_t dummy = uint32_t(T) + uint32_t(lane);  // per-lane scratch slot past the tile
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                uint32_t off = rowbase + uint32_t((wex >> (16 * r)) & 0xFFFFu) + ((lane_excl >> (8 * r)) & 0xFFu);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t keep = (m[r] >> q) & 1u;
                    buf[keep ? off : dummy] = v[r][q];
                    off += keep;
                }
                rowbase += uint32_t((tot >> (16 * r)) & 0xFFFFu);
            }
            bar_arrive(kCountBar + int(j & 3), BLOCK);  // hand the count to the look-back warp
        }
    }
    // Every issued copy has been consumed unless a wait gave up; drain those
    // (bounded) so no copy lands after the block has exited.
    if (ct == 0) {
        const uint32_t pend = s_pending;
        for (int s = 0; s < S; ++s) {
            if (!((pend >> s) & 1u)) continue;
            const uint32_t parity = (s_pend_j[s] / S) & 1u;
            for (uint32_t polls = 0; polls < kMbarSpin; ++polls)
                if (mbar_try_wait(&mbar[s], parity)) break;
        }
    }
}

namespace {

template <int CWW, int S, int PF, int MAXG, int MINB>
ka_status launch_tma_shape(const TmaArgs &a, uint64_t cap, cudaStream_t stream) {
    constexpr int BLOCK = (CWW + 1) * 32, T = CWW * 32 * 16;
    const size_t smem = size_t(S) * (T + 32) * 4;
    auto kern = k_compact_tma<CWW, S, PF, MAXG, MINB>;
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

}  // namespace

bool compact_tma_eligible(const CompactLaunch &L) {
    if ((reinterpret_cast<uintptr_t>(L.in) & 15u) != 0) return false;
    return L.tile.ipt == 16 && (L.tile.block == 256 || L.tile.block == 512);
}

ka_status launch_compact_tma(const CompactLaunch &L, cudaStream_t stream) {
    TmaArgs a;
    a.in = L.in;
    a.out = L.out;
    a.n_ptr = L.n_ptr;
    a.count = L.count;
    a.ws = static_cast<WsHeader *>(L.ws);
    a.status = reinterpret_cast<uint64_t *>(static_cast<char *>(L.ws) + kWsHeaderBytes);
    a.n = uint32_t(L.n);
    a.status_cap = status_capacity(L.ws_bytes);
    a.mul = L.mul;
    a.pred = L.pred;
    if (L.tile.block == 512) return launch_tma_shape<16, 3, 2, 320, 2>(a, L.n, stream);
    return launch_tma_shape<8, 4, 4, 480, 3>(a, L.n, stream);
}

}  // namespace ka
