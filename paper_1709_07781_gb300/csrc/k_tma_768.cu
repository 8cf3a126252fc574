// Kernels of the TMA tile shape (768, 16): the compaction for every predicate
// kind and the scan (see ka_tma_pass.cuh).
#include "ka_tma_pass.cuh"

namespace ka {
namespace tma {

ka_status launch_tma_768(const TmaArgs &a, bool scan, int32_t pk, uint64_t cap, cudaStream_t stream) {
    return launch_tma_config<24, 4, 3, 160, 1, 8, 3>(a, scan, pk, cap, stream);
}

}  // namespace tma
}  // namespace ka
