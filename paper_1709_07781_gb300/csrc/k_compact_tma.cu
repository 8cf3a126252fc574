// Entry points of the warp-specialised TMA kernel (ka_tma_pass.cuh): the
// fused compaction and the exclusive scan for the TMA tile shapes, with any
// 4-byte-aligned input (tiles are shifted back to a 16-byte boundary). The
// kernels are instantiated in k_tma_<shape>.cu, one file per tile shape.
#include "ka_tma_pass.cuh"

namespace ka {

using namespace tma;

namespace {

// tile (768, 16): 26 compute warps, 13312 entries, 4 stages of 52 KiB and a 13 KiB
//                 spill ring (8 slots of 16 entries per warp), 1 block per SM;
// tile (512, 16): 16 compute warps, 8192 entries, 3 stages of 32 KiB, 2 blocks per SM;
// tile (256, 16): 8 compute warps, 4096 entries, 4 stages of 16 KiB, 3 blocks per SM.
ka_status launch_tma(const TmaArgs &a, ka_tile tile, bool scan, int32_t pk, uint64_t cap, cudaStream_t stream) {
    if (tile.block == 768) return launch_tma_768(a, scan, pk, cap, stream);
    if (tile.block == 512) return launch_tma_512(a, scan, pk, cap, stream);
    return launch_tma_256(a, scan, pk, cap, stream);
}

}  // namespace

bool tma_shape(uint32_t block, uint32_t ipt) {
    return ipt == 16 && (block == 256 || block == 512 || block == 768);
}

bool compact_tma_eligible(const CompactLaunch &L) {
    // the shifted length n + lead must fit 32 bits
    return tma_shape(L.tile.block, L.tile.ipt) && L.n <= 0xFFFFFFFCull;
}

ka_status launch_compact_tma(const CompactLaunch &L, cudaStream_t stream) {
    TmaArgs a;
    a.lead = uint32_t(reinterpret_cast<uintptr_t>(L.in) & 15u) / 4u;
    a.in = L.in - a.lead;
    a.out = L.out;
    a.n_ptr = L.n_ptr;
    a.count = L.count;
    a.ws = static_cast<WsHeader *>(L.ws);
    a.status = reinterpret_cast<uint64_t *>(static_cast<char *>(L.ws) + kWsHeaderBytes);
    a.n = uint32_t(L.n);
    a.status_cap = status_capacity(L.ws_bytes);
    a.mul = L.mul;
    a.pred = L.pred;
    a.out_vec = 0;
    return launch_tma(a, L.tile, false, L.pred.kind, L.n + a.lead, stream);
}

ka_status launch_scan_tma(const uint32_t *in, uint64_t n, const uint32_t *n_ptr, uint32_t *out, uint32_t *total,
                          void *ws, uint64_t ws_bytes, ka_tile tile, cudaStream_t stream) {
    TmaArgs a;
    a.lead = uint32_t(reinterpret_cast<uintptr_t>(in) & 15u) / 4u;
    a.in = in - a.lead;
    a.out = out;
    a.out_vec = ((reinterpret_cast<uintptr_t>(out) - 4u * a.lead) & 15u) == 0 ? 1u : 0u;
    a.n_ptr = n_ptr;
    a.count = total;
    a.ws = static_cast<WsHeader *>(ws);
    a.status = reinterpret_cast<uint64_t *>(static_cast<char *>(ws) + kWsHeaderBytes);
    a.n = uint32_t(n);
    a.status_cap = status_capacity(ws_bytes);
    a.mul = 1u;
    a.pred = PredDev{};
    return launch_tma(a, tile, true, kAll, n + a.lead, stream);
}

}  // namespace ka
