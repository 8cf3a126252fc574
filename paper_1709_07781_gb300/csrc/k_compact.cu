// Fused single-pass stream compaction (Sec. 4.1's flag, prefix-sum and move
// phases in one kernel; the paper's own OpenCL version fuses only the last
// two, and Sec. 3.6 names "several kernels inside one actor" as the way to
// avoid inter-stage traffic). The per-tile work is compact_tile (ka_tile.cuh).
// Blocks are persistent (grid = resident blocks) and take tiles by ticket.
// Output offsets never exceed input positions, so out == in is safe: a tile
// writes only after all its predecessors have loaded their input.
#include "ka_internal.h"
#include "ka_tile.cuh"

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
    __shared__ CompactSmem<BLOCK, IPT> sm;
    __shared__ uint32_t s_ticket, s_epoch, s_n, s_spin;
    const int tid = threadIdx.x;

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
    const uint32_t spin = s_spin;
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
        compact_tile<BLOCK, IPT>(sm, a.in + base, a.out, valid, a.vec_ok != 0u, a.mul, a.pred, a.status, tile, 0u,
                                 epoch, spin, a.ws, tile == live_tiles - 1 ? a.count : nullptr);
    }
}

template <int BLOCK, int IPT>
static ka_status launch_shape(const CompactArgs &a, uint64_t cap, cudaStream_t stream) {
    constexpr int T = BLOCK * IPT;
    static PerDeviceInt occ_cache;
    const int occupancy = per_device_value(occ_cache, current_device(), [] {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_compact_fused<BLOCK, IPT>, BLOCK, 0);
        return occ > 0 ? occ : 1;
    });
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
    if (!tile_supported_for(KA_KERNEL_COMPACT, t.block, t.ipt)) return KA_E_ARG;
    const uint64_t tiles = tiles_for(L.n, t.block * t.ipt);
    const ka_status ws_ok = check_workspace(L.ws, L.ws_bytes, tiles);
    if (ws_ok != KA_OK) return ws_ok;
    if (compact_tma_eligible(L)) return launch_compact_tma(L, stream);
    if (!tile_supported(t.block, t.ipt)) return KA_E_ARG;  // a TMA-only shape beyond its size limit
    CompactArgs a;
    a.in = L.in;
    a.out = L.out;
    a.n_ptr = L.n_ptr;
    a.count = L.count;
    a.ws = static_cast<WsHeader *>(L.ws);
    a.status = reinterpret_cast<uint64_t *>(static_cast<char *>(L.ws) + kWsHeaderBytes);
    a.n = uint32_t(L.n);
    a.status_cap = status_capacity(L.ws_bytes);
    a.mul = L.mul;
    a.vec_ok = (reinterpret_cast<uintptr_t>(L.in) & 15u) == 0 ? 1u : 0u;
    a.pred = L.pred;
    switch (shape_key(t.block, t.ipt)) {
#define KA_CASE(B, I) \
    case shape_key(B, I): return launch_shape<B, I>(a, L.n, stream);
        KA_FOR_EACH_SHAPE(KA_CASE)
#undef KA_CASE
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
