// Move phase of the compaction (phase 3 of Sec. 4.1): out[o[i]] = x[i] for
// every flagged entry. Because o is the exclusive prefix sum of 0/1 flags, the
// kept entries of one tile land on one contiguous run
// [o[first], o[last] + f[last]) of the output; each block stages that run in
// shared memory at tile-local offsets and then writes it with consecutive
// threads on consecutive words, instead of scattering single words.
// Tiles are independent (no look-back): a grid-stride loop over tiles.
#include "ka_internal.h"

namespace ka {

constexpr int kScatterBlock = 256;
constexpr int kScatterIpt = 8;

struct ScatterArgs {
    const uint32_t *x;
    const uint32_t *f;
    const uint32_t *o;
    const uint32_t *n_ptr;
    uint32_t *out;
    uint32_t *count_out;  // optional: receives the result length o[n-1] + f[n-1]
    uint32_t n;
    uint32_t vec_ok;
};

__global__ void __launch_bounds__(kScatterBlock) k_scatter(const ScatterArgs a) {
    constexpr int BLOCK = kScatterBlock;
    constexpr int T = kScatterBlock * kScatterIpt;
    constexpr int ROWS = kScatterIpt / 4;
    __shared__ uint32_t s_out[T];
    const int tid = threadIdx.x;

    uint32_t n = a.n;
    if (a.n_ptr) {
        const uint32_t d = *a.n_ptr;
        n = d < n ? d : n;
    }
    const uint32_t live_tiles = uint32_t((uint64_t(n) + T - 1) / T);
    if (a.count_out && blockIdx.x == 0 && tid == 0 && live_tiles == 0) *a.count_out = 0u;
    for (uint32_t tile = blockIdx.x; tile < live_tiles; tile += gridDim.x) {
        const uint32_t base = tile * uint32_t(T);
        const uint32_t valid = (n - base) < uint32_t(T) ? (n - base) : uint32_t(T);
        const uint32_t last = base + valid - 1;
        const uint32_t o0 = a.o[base];
        const uint32_t end = a.o[last] + (a.f[last] ? 1u : 0u);
        if (a.count_out && tid == 0 && tile == live_tiles - 1) *a.count_out = end;
        uint32_t kept = end - o0;
        if (kept > valid) kept = valid;  // only if flags/offsets are inconsistent
        if (valid == uint32_t(T) && a.vec_ok) {
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const uint32_t e = base + (r * BLOCK + tid) * 4;
                const uint4 xv = ld_stream_v4(a.x + e);
                const uint4 fv = ld_stream_v4(a.f + e);
                const uint4 ov = ld_stream_v4(a.o + e);
                const uint32_t xs[4] = {xv.x, xv.y, xv.z, xv.w};
                const uint32_t fs[4] = {fv.x, fv.y, fv.z, fv.w};
                const uint32_t os[4] = {ov.x, ov.y, ov.z, ov.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t local = os[j] - o0;
                    if (fs[j] && local < uint32_t(T)) s_out[local] = xs[j];
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t idx = uint32_t(r * BLOCK + tid) * 4 + j;
                    if (idx < valid && a.f[base + idx]) {
                        const uint32_t local = a.o[base + idx] - o0;
                        if (local < uint32_t(T)) s_out[local] = a.x[base + idx];
                    }
                }
            }
        }
        __syncthreads();
        uint32_t *dst = a.out + o0;
        for (uint32_t k = tid; k < kept; k += BLOCK) dst[k] = s_out[k];
        __syncthreads();
    }
}

ka_status launch_scatter(const uint32_t *x, const uint32_t *flags, const uint32_t *offsets, uint64_t n,
                         const uint32_t *n_ptr, uint32_t *out, uint32_t *count_out, cudaStream_t stream) {
    if (n > 0xFFFFFFFFull) return KA_E_ARG;
    if (n && (!x || !flags || !offsets || !out)) return KA_E_ARG;
    if (count_out && count_out == n_ptr) return KA_E_ARG;
    if (n == 0 && !count_out) return KA_OK;
    ScatterArgs a;
    a.x = x;
    a.f = flags;
    a.o = offsets;
    a.n_ptr = n_ptr;
    a.out = out;
    a.count_out = count_out;
    a.n = uint32_t(n);
    a.vec_ok = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(flags) |
                 reinterpret_cast<uintptr_t>(offsets)) & 15u) == 0 ? 1u : 0u;
    constexpr int T = kScatterBlock * kScatterIpt;
    static PerDeviceInt occ_cache;
    const int occupancy = per_device_value(occ_cache, current_device(), [] {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_scatter, kScatterBlock, 0);
        return occ > 0 ? occ : 1;
    });
    uint64_t grid = (n + T - 1) / T;
    const uint64_t resident = uint64_t(device_info().sm_count) * occupancy;
    if (grid > resident) grid = resident;
    if (grid < 1) grid = 1;
    k_scatter<<<unsigned(grid), kScatterBlock, 0, stream>>>(a);
    return cuda_status(cudaGetLastError());
}

}  // namespace ka

using namespace ka;

extern "C" ka_status ka_scatter(const uint32_t *d_x, const uint32_t *d_flags, const uint32_t *d_offsets, uint64_t n,
                                const uint32_t *d_n, uint32_t *d_out, void *stream) {
    return launch_scatter(d_x, d_flags, d_offsets, n, d_n, d_out, nullptr, static_cast<cudaStream_t>(stream));
}
