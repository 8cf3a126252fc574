// Kernels of the TMA tile shape (512, 16): the compaction for every predicate
// kind and the scan (see ka_tma_pass.cuh).
#include "ka_tma_pass.cuh"

namespace ka {
namespace tma {

ka_status launch_tma_512(const TmaArgs &a, bool scan, int32_t pk, uint64_t cap, cudaStream_t stream) {
    return launch_tma_config<16, 3, 2, 320, 2, 4, 1>(a, scan, pk, cap, stream);
}

}  // namespace tma
}  // namespace ka
