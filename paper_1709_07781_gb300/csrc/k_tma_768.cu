// Kernels of the TMA tile shape (768, 16): the compaction for every predicate
// kind and the scan (see ka_tma_pass.cuh), with 26 compute warps (tiles of
// 13312 entries): the largest tile whose four stages and an 8-slot spill ring
// of 16-entry slots fit a block's shared memory (fewer tiles, fewer look-back
// resolutions).
#include "ka_tma_pass.cuh"

namespace ka {
namespace tma {

ka_status launch_tma_768(const TmaArgs &a, bool scan, int32_t pk, uint64_t cap, cudaStream_t stream) {
    return launch_tma_config<26, 4, 3, 160, 1, 8, 3>(a, scan, pk, cap, stream);
}

}  // namespace tma
}  // namespace ka
