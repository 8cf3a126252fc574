// Single-pass exclusive prefix sum of uint32 values (phase 2 of the
// compaction of Sec. 4.1: "prefix sum" of the flags), mod 2^32, with
// decoupled look-back between tiles.
//
// Layout as in the fused compaction: row r, thread t holds the 16-byte vector
// [4 (r BLOCK + t), +4). Each row is scanned separately across the warp
// (shuffles), warp 0 scans the per-warp row totals and runs the look-back,
// then every thread writes its four exclusive sums back as one 16-byte store
// in the same coalesced layout. Blocks are persistent and take tiles by
// ticket. out == in is allowed (each tile reads its own range before writing).
#include "ka_internal.h"

namespace ka {

struct ScanArgs {
    const uint32_t *in;
    uint32_t *out;
    const uint32_t *n_ptr;
    uint32_t *total;
    WsHeader *ws;
    uint64_t *status;
    uint32_t n;
    uint32_t status_cap;
    uint32_t vec_ok;
};

template <int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK) k_exclusive_scan(const ScanArgs a) {
    constexpr int T = BLOCK * IPT;
    constexpr int ROWS = IPT / 4;
    constexpr int WARPS = BLOCK / 32;

    __shared__ uint32_t s_wt[ROWS][WARPS];
    __shared__ uint32_t s_wx[ROWS][WARPS];
    __shared__ uint32_t s_rowbase[ROWS];
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
            if (last && live_tiles == 0) *a.total = 0u;
            s_ticket = t;
            s_epoch = ep;
        }
        __syncthreads();
        const uint32_t tile = s_ticket;
        const uint32_t epoch = s_epoch;
        if (tile >= live_tiles) break;
        const uint32_t base = tile * uint32_t(T);
        const uint32_t valid = (n - base) < uint32_t(T) ? (n - base) : uint32_t(T);
        const bool full = valid == uint32_t(T) && a.vec_ok;

        uint32_t v[ROWS][4];
        if (full) {
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const uint4 q = ld_stream_v4(a.in + base + (r * BLOCK + tid) * 4);
                v[r][0] = q.x;
                v[r][1] = q.y;
                v[r][2] = q.z;
                v[r][3] = q.w;
            }
        } else {
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t idx = uint32_t(r * BLOCK + tid) * 4 + j;
                    v[r][j] = idx < valid ? a.in[base + idx] : 0u;
                }
            }
        }
        uint32_t lane_excl[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const uint32_t s = v[r][0] + v[r][1] + v[r][2] + v[r][3];
            const uint32_t incl = warp_incl_scan(s, lane);
            lane_excl[r] = incl - s;
            if (lane == 31) s_wt[r][warp] = incl;
        }
        __syncthreads();

        if (warp == 0) {
            uint32_t agg = 0;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const uint32_t wt = lane < WARPS ? s_wt[r][lane] : 0u;
                const uint32_t wi = warp_incl_scan(wt, lane);
                if (lane < WARPS) s_wx[r][lane] = wi - wt;
                if (lane == 0) s_rowbase[r] = agg;
                agg += __shfl_sync(kFull, wi, 31);
            }
            bool err;
            const uint32_t prefix = lookback_warp(a.status, tile, 0u, epoch, agg, s_spin, a.ws, &err);
            if (lane == 0) {
                s_prefix = prefix;
                s_err = err ? 1u : 0u;
                if (!err && tile == live_tiles - 1) *a.total = prefix + agg;
            }
        }
        __syncthreads();
        if (s_err == 0u) {
            const uint32_t prefix = s_prefix;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const uint32_t e0 = prefix + s_rowbase[r] + s_wx[r][warp] + lane_excl[r];
                const uint32_t e1 = e0 + v[r][0];
                const uint32_t e2 = e1 + v[r][1];
                const uint32_t e3 = e2 + v[r][2];
                const uint32_t idx = uint32_t(r * BLOCK + tid) * 4;
                if (full) {
                    *reinterpret_cast<uint4 *>(a.out + base + idx) = make_uint4(e0, e1, e2, e3);
                } else {
                    if (idx + 0 < valid) a.out[base + idx + 0] = e0;
                    if (idx + 1 < valid) a.out[base + idx + 1] = e1;
                    if (idx + 2 < valid) a.out[base + idx + 2] = e2;
                    if (idx + 3 < valid) a.out[base + idx + 3] = e3;
                }
            }
        }
        // s_wx / s_rowbase are rewritten in the next tile only after the
        // ticket barrier, which every thread passes after these reads.
    }
}

template <int BLOCK, int IPT>
static ka_status launch_scan_shape(const ScanArgs &a, uint64_t cap, cudaStream_t stream) {
    constexpr int T = BLOCK * IPT;
    static PerDeviceInt occ_cache;
    const int occupancy = per_device_value(occ_cache, current_device(), [] {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_exclusive_scan<BLOCK, IPT>, BLOCK, 0);
        return occ > 0 ? occ : 1;
    });
    uint64_t grid = (cap + T - 1) / T;
    const uint64_t resident = uint64_t(device_info().sm_count) * occupancy;
    if (grid > resident) grid = resident;
    if (grid < 1) grid = 1;
    k_exclusive_scan<BLOCK, IPT><<<unsigned(grid), BLOCK, 0, stream>>>(a);
    return cuda_status(cudaGetLastError());
}

ka_status launch_exclusive_scan(const uint32_t *in, uint64_t n, const uint32_t *n_ptr, uint32_t *out,
                                uint32_t *total, void *ws, uint64_t ws_bytes, ka_tile t, cudaStream_t stream) {
    if (n > 0xFFFFFFFFull || (n && (!in || !out)) || !total) return KA_E_ARG;
    if (n_ptr && n_ptr == total) return KA_E_ARG;
    if (!tile_supported_for(KA_KERNEL_SCAN, t.block, t.ipt)) return KA_E_ARG;
    const ka_status ws_ok = check_workspace(ws, ws_bytes, tiles_for(n, t.block * t.ipt));
    if (ws_ok != KA_OK) return ws_ok;
    if (tma_shape(t.block, t.ipt) && n <= 0xFFFFFFFCull)
        return launch_scan_tma(in, n, n_ptr, out, total, ws, ws_bytes, t, stream);
    if (!tile_supported(t.block, t.ipt)) return KA_E_ARG;  // a TMA-only shape beyond its size limit
    ScanArgs a;
    a.in = in;
    a.out = out;
    a.n_ptr = n_ptr;
    a.total = total;
    a.ws = static_cast<WsHeader *>(ws);
    a.status = reinterpret_cast<uint64_t *>(static_cast<char *>(ws) + kWsHeaderBytes);
    a.n = uint32_t(n);
    a.status_cap = status_capacity(ws_bytes);
    a.vec_ok = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0 ? 1u : 0u;
    switch (shape_key(t.block, t.ipt)) {
#define KA_CASE(B, I) \
    case shape_key(B, I): return launch_scan_shape<B, I>(a, n, stream);
        KA_FOR_EACH_SHAPE(KA_CASE)
#undef KA_CASE
    default: return KA_E_ARG;
    }
}

}  // namespace ka

using namespace ka;

extern "C" ka_status ka_exclusive_scan(const uint32_t *d_in, uint64_t n, const uint32_t *d_n, uint32_t *d_out,
                                       uint32_t *d_total, void *d_ws, uint64_t ws_bytes, const ka_tile *tile,
                                       void *stream) {
    return launch_exclusive_scan(d_in, n, d_n, d_out, d_total, d_ws, ws_bytes, resolve_tile(KA_KERNEL_SCAN, n, tile),
                                 static_cast<cudaStream_t>(stream));
}
