// Fused single-pass stream compaction (Sec. 4.1's flag, prefix-sum and move
// phases in one kernel; the paper's own OpenCL version fuses only the last
// two, and Sec. 3.6 names "several kernels inside one actor" as the way to
// avoid inter-stage traffic).
//
// One tile = BLOCK threads x IPT entries. Per tile:
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
// Blocks are persistent (grid = resident blocks) and take tiles by ticket.
// Output offsets never exceed input positions, so out == in is safe: a tile
// writes only after all its predecessors have loaded their input.
#include "ka_internal.h"

namespace ka {

struct CompactArgs {
    const uint32_t *in;
    uint32_t *out;
    const uint32_t *n_ptr;
    uint32_t *count;
    WsHeader *ws;
    uint64_t *status;
    uint32_t n;
    uint32_t status_cap;
    uint32_t mul;
    uint32_t vec_ok;
    PredDev pred;
};

template <int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK) k_compact_fused(const CompactArgs a) {
    constexpr int T = BLOCK * IPT;
    constexpr int ROWS = IPT / 4;
    constexpr int WARPS = BLOCK / 32;
    static_assert(ROWS >= 1 && ROWS <= 4, "8-bit row fields hold at most 4 rows");
    static_assert(WARPS <= 16, "16-bit block fields hold at most 16 warps x 128");

    __shared__ uint32_t s_out[T];
    __shared__ uint32_t s_wtot[WARPS];
    __shared__ uint64_t s_wexcl[WARPS];
    __shared__ uint64_t s_tot;
    __shared__ uint32_t s_ticket, s_epoch, s_prefix, s_n, s_err, s_spin;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;

    if (tid == 0) {
        uint32_t n = a.n;
        if (a.n_ptr) {
            const uint32_t d = *a.n_ptr;
            n = d < n ? d : n;
        }
        s_n = n;
        const uint32_t sl = a.ws->spin_limit;
        s_spin = sl ? sl : kDefaultSpinLimit;
    }
    __syncthreads();
    const uint32_t n = s_n;
    const uint32_t live_tiles = uint32_t((uint64_t(n) + T - 1) / T);
    if (live_tiles > a.status_cap) {
        if (tid == 0 && blockIdx.x == 0) record_error(a.ws, kDevErrWorkspace, 0);
        return;
    }

    for (;;) {
        if (tid == 0) {
            uint32_t ep;
            bool last;
            const uint32_t t = take_ticket(a.ws, live_tiles, &ep, &last);
            if (last && live_tiles == 0) *a.count = 0u;
            s_ticket = t;
            s_epoch = ep;
        }
        __syncthreads();
        const uint32_t tile = s_ticket;
        const uint32_t epoch = s_epoch;
        if (tile >= live_tiles) break;
        const uint32_t base = tile * uint32_t(T);
        const uint32_t valid = (n - base) < uint32_t(T) ? (n - base) : uint32_t(T);

        uint32_t v[ROWS][4];
        uint32_t m[ROWS];
        if (valid == uint32_t(T) && a.vec_ok) {
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const uint4 q = ld_stream_v4(a.in + base + (r * BLOCK + tid) * 4);
                v[r][0] = q.x * a.mul;
                v[r][1] = q.y * a.mul;
                v[r][2] = q.z * a.mul;
                v[r][3] = q.w * a.mul;
            }
        } else {
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t idx = uint32_t(r * BLOCK + tid) * 4 + j;
                    v[r][j] = idx < valid ? ld_stream_u32(a.in + base + idx) * a.mul : 0u;
                }
            }
        }
        uint32_t packed = 0;
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            uint32_t mk = pred_mask4(a.pred, v[r][0], v[r][1], v[r][2], v[r][3]);
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
        if (lane == 31) s_wtot[warp] = incl;
        __syncthreads();

        if (warp == 0) {
            const uint64_t wt = lane < WARPS ? spread8to16(s_wtot[lane]) : 0ull;
            const uint64_t wincl = warp_incl_scan64(wt, lane, WARPS);
            if (lane < WARPS) s_wexcl[lane] = wincl - wt;
            const uint64_t tot = __shfl_sync(kFull, wincl, WARPS - 1);
            const uint32_t agg = uint32_t(tot & 0xFFFFu) + uint32_t((tot >> 16) & 0xFFFFu) +
                                 uint32_t((tot >> 32) & 0xFFFFu) + uint32_t(tot >> 48);
            bool err;
            const uint32_t prefix = lookback_warp(a.status, tile, 0u, epoch, agg, s_spin, a.ws, &err);
            if (lane == 0) {
                s_tot = tot;
                s_prefix = prefix;
                s_err = err ? 1u : 0u;
                if (!err && tile == live_tiles - 1) *a.count = prefix + agg;
            }
        }
        __syncthreads();
        const uint64_t tot = s_tot;
        const uint32_t prefix = s_prefix;
        const bool err = s_err != 0u;
        if (!err) {
            const uint64_t wex = s_wexcl[warp];
            uint32_t rowbase = 0;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                uint32_t off = rowbase + uint32_t((wex >> (16 * r)) & 0xFFFFu) + ((lane_excl >> (8 * r)) & 0xFFu);
                const uint32_t mk = m[r];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if ((mk >> j) & 1u) {
                        s_out[off] = v[r][j];
                        ++off;
                    }
                }
                rowbase += uint32_t((tot >> (16 * r)) & 0xFFFFu);
            }
        }
        __syncthreads();
        if (!err) {
            const uint32_t agg = uint32_t(tot & 0xFFFFu) + uint32_t((tot >> 16) & 0xFFFFu) +
                                 uint32_t((tot >> 32) & 0xFFFFu) + uint32_t(tot >> 48);
            uint32_t *dst = a.out + prefix;
            for (uint32_t k = tid; k < agg; k += BLOCK) dst[k] = s_out[k];
        }
    }
}

template <int BLOCK, int IPT>
static ka_status launch_shape(const CompactArgs &a, uint64_t cap, cudaStream_t stream) {
    constexpr int T = BLOCK * IPT;
    static int occupancy = 0;
    if (occupancy == 0) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_compact_fused<BLOCK, IPT>, BLOCK, 0);
        occupancy = occ > 0 ? occ : 1;
    }
    uint64_t grid = (cap + T - 1) / T;
    const uint64_t resident = uint64_t(device_info().sm_count) * occupancy;
    if (grid > resident) grid = resident;
    if (grid < 1) grid = 1;
    k_compact_fused<BLOCK, IPT><<<unsigned(grid), BLOCK, 0, stream>>>(a);
    return cuda_status(cudaGetLastError());
}

ka_status launch_compact(const CompactLaunch &L, cudaStream_t stream) {
    if (L.n > 0xFFFFFFFFull) return KA_E_ARG;
    if (L.n && (!L.in || !L.out)) return KA_E_ARG;
    if (!L.count) return KA_E_ARG;
    if (L.n_ptr && L.n_ptr == L.count) return KA_E_ARG;
    const ka_tile t = L.tile;
    if (!tile_supported(t.block, t.ipt)) return KA_E_ARG;
    const uint64_t tiles = tiles_for(L.n, t.block * t.ipt);
    const ka_status ws_ok = check_workspace(L.ws, L.ws_bytes, tiles);
    if (ws_ok != KA_OK) return ws_ok;
    CompactArgs a;
    a.in = L.in;
    a.out = L.out;
    a.n_ptr = L.n_ptr;
    a.count = L.count;
    a.ws = static_cast<WsHeader *>(L.ws);
    a.status = reinterpret_cast<uint64_t *>(static_cast<char *>(L.ws) + kWsHeaderBytes);
    a.n = uint32_t(L.n);
    const uint64_t cap_words = (L.ws_bytes - kWsHeaderBytes) / 8;
    a.status_cap = cap_words > 0xFFFFFFFFull ? 0xFFFFFFFFu : uint32_t(cap_words);
    a.mul = L.mul;
    a.vec_ok = (reinterpret_cast<uintptr_t>(L.in) & 15u) == 0 ? 1u : 0u;
    a.pred = L.pred;
    switch (t.block * 100 + t.ipt) {
    case 12804: return launch_shape<128, 4>(a, L.n, stream);
    case 12808: return launch_shape<128, 8>(a, L.n, stream);
    case 12816: return launch_shape<128, 16>(a, L.n, stream);
    case 25604: return launch_shape<256, 4>(a, L.n, stream);
    case 25608: return launch_shape<256, 8>(a, L.n, stream);
    case 25616: return launch_shape<256, 16>(a, L.n, stream);
    case 51204: return launch_shape<512, 4>(a, L.n, stream);
    case 51208: return launch_shape<512, 8>(a, L.n, stream);
    default: return KA_E_ARG;
    }
}

}  // namespace ka

using namespace ka;

extern "C" ka_status ka_compact(const uint32_t *d_in, uint64_t n, const uint32_t *d_n, int32_t pred, uint32_t param,
                                uint32_t xform, uint32_t *d_out, uint32_t *d_count, void *d_ws, uint64_t ws_bytes,
                                const ka_tile *tile, void *stream) {
    CompactLaunch L;
    const ka_status s = make_pred(pred, param, &L.pred);
    if (s != KA_OK) return s;
    if (xform != KA_XFORM_NONE && xform != KA_XFORM_HASH) return KA_E_ARG;
    L.in = d_in;
    L.out = d_out;
    L.n_ptr = d_n;
    L.count = d_count;
    L.n = n;
    L.mul = xform == KA_XFORM_HASH ? kHashMul : 1u;
    L.ws = d_ws;
    L.ws_bytes = ws_bytes;
    L.tile = resolve_tile(KA_KERNEL_COMPACT, n, tile);
    return launch_compact(L, static_cast<cudaStream_t>(stream));
}
