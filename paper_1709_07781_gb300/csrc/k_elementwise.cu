// Element-wise stage kernels: seeded input, hash map, flag map (phase 1 of the
// compaction of Sec. 4.1), the interleave of fuseFillsLiterals (Sec. 4.1,
// Listing 5), and a count-forwarding empty stage (the empty kernel the paper
// uses to price one message-passing stage, Sec. 3.6).
//
// All are HBM-bound streams: grid-stride loops over 16-byte vectors with two
// vectors in flight per thread, grids of a few blocks per SM, scalar code for
// the ragged head/tail and for inputs that are not 16-byte aligned. Live
// lengths may come from a device word (the previous stage's count). Scalar
// entry indices are 64-bit: with n near 2^32, a 32-bit index plus the grid
// stride would wrap below n and the loop would not end.
#include "ka_internal.h"

namespace ka {

constexpr int kEwBlock = 256;

__device__ __forceinline__ uint64_t splitmix64_dev(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t live_n(const uint32_t *n_ptr, uint64_t n) {
    if (!n_ptr) return uint32_t(n);
    const uint32_t d = *n_ptr;
    return uint64_t(d) < n ? d : uint32_t(n);
}

__device__ __forceinline__ void st_v4(uint32_t *p, uint4 v) { *reinterpret_cast<uint4 *>(p) = v; }

static unsigned ew_grid(uint64_t work_items) {
    const uint64_t per_block = uint64_t(kEwBlock) * 2;
    uint64_t g = (work_items + per_block - 1) / per_block;
    const uint64_t cap = uint64_t(device_info().sm_count) * 8;
    if (g > cap) g = cap;
    return unsigned(g < 1 ? 1 : g);
}

static inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kEwBlock) k_generate(uint32_t *out, uint32_t n, uint64_t seed, int vec,
                                                        uint32_t *n_out) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t stride = gridDim.x * blockDim.x;
    if (tid == 0 && n_out) *n_out = n;
    if (vec) {
        const uint32_t n4 = n / 4;
        for (uint32_t i = tid; i < n4; i += stride) {
            const uint64_t e = uint64_t(i) * 4;
            uint4 v;
            v.x = uint32_t(splitmix64_dev(seed, e) >> 32);
            v.y = uint32_t(splitmix64_dev(seed, e + 1) >> 32);
            v.z = uint32_t(splitmix64_dev(seed, e + 2) >> 32);
            v.w = uint32_t(splitmix64_dev(seed, e + 3) >> 32);
            st_v4(out + e, v);
        }
        for (uint64_t e = uint64_t(n4) * 4 + tid; e < n; e += stride) out[e] = uint32_t(splitmix64_dev(seed, e) >> 32);
    } else {
        for (uint64_t e = tid; e < n; e += stride) out[e] = uint32_t(splitmix64_dev(seed, e) >> 32);
    }
}

ka_status launch_generate(uint32_t *out, uint64_t n, uint64_t seed, uint32_t *n_out, cudaStream_t stream) {
    if (n > 0xFFFFFFFFull || (n && !out)) return KA_E_ARG;
    k_generate<<<ew_grid((n + 3) / 4), kEwBlock, 0, stream>>>(out, uint32_t(n), seed, aligned16(out), n_out);
    return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Hash map (mul = 2654435761) and flag map share one kernel shape: read a
// vector, transform or test each entry, write a vector.
template <bool FLAGS>
__global__ void __launch_bounds__(kEwBlock) k_map(const uint32_t *in, uint64_t cap, const uint32_t *n_ptr,
                                                  uint32_t *out, uint32_t *n_out, PredDev pred, int vec) {
    const uint32_t n = live_n(n_ptr, cap);
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t stride = gridDim.x * blockDim.x;
    if (tid == 0 && n_out) *n_out = n;
    auto f = [&](uint32_t x) -> uint32_t { return FLAGS ? uint32_t(pred_keep(pred, x)) : x * kHashMul; };
    if (vec) {
        const uint32_t n4 = n / 4;
        uint32_t i = tid;
        for (; i + stride < n4; i += 2 * stride) {
            const uint4 a = ld_stream_v4(in + uint64_t(i) * 4);
            const uint4 b = ld_stream_v4(in + uint64_t(i + stride) * 4);
            st_v4(out + uint64_t(i) * 4, make_uint4(f(a.x), f(a.y), f(a.z), f(a.w)));
            st_v4(out + uint64_t(i + stride) * 4, make_uint4(f(b.x), f(b.y), f(b.z), f(b.w)));
        }
        for (; i < n4; i += stride) {
            const uint4 a = ld_stream_v4(in + uint64_t(i) * 4);
            st_v4(out + uint64_t(i) * 4, make_uint4(f(a.x), f(a.y), f(a.z), f(a.w)));
        }
        for (uint64_t e = uint64_t(n4) * 4 + tid; e < n; e += stride) out[e] = f(in[e]);
    } else {
        for (uint64_t e = tid; e < n; e += stride) out[e] = f(in[e]);
    }
}

ka_status launch_map_hash(const uint32_t *in, uint64_t n, const uint32_t *n_ptr, uint32_t *out,
                          uint32_t *n_out, cudaStream_t stream) {
    if (n > 0xFFFFFFFFull || (n && (!in || !out))) return KA_E_ARG;
    if (n_out && n_out == n_ptr) return KA_E_ARG;
    PredDev none{};
    const int vec = aligned16(in) && aligned16(out);
    k_map<false><<<ew_grid((n + 3) / 4), kEwBlock, 0, stream>>>(in, n, n_ptr, out, n_out, none, vec);
    return cuda_status(cudaGetLastError());
}

ka_status launch_predicate(const uint32_t *x, uint64_t n, const uint32_t *n_ptr, const PredDev &pred,
                           uint32_t *flags, uint32_t *n_out, cudaStream_t stream) {
    if (n > 0xFFFFFFFFull || (n && (!x || !flags))) return KA_E_ARG;
    if (n_out && n_out == n_ptr) return KA_E_ARG;
    const int vec = aligned16(x) && aligned16(flags);
    k_map<true><<<ew_grid((n + 3) / 4), kEwBlock, 0, stream>>>(x, n, n_ptr, flags, n_out, pred, vec);
    return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kEwBlock) k_prepare_index(const uint32_t *a, const uint32_t *b, uint64_t cap,
                                                             const uint32_t *k_ptr, uint32_t *index,
                                                             uint32_t *n_out, int vec) {
    const uint32_t k = live_n(k_ptr, cap);
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t stride = gridDim.x * blockDim.x;
    if (tid == 0 && n_out) *n_out = 2u * k;
    if (vec) {
        // eight independent 16-byte loads per array in flight per thread (a
        // single pair per iteration leaves too few bytes in flight per SM to
        // cover the memory latency), consecutive threads on consecutive
        // chunks; the index is written with streaming stores (written once,
        // read by the next stage from DRAM or whatever of it L2 still holds)
        constexpr uint32_t U = 8;
        const uint32_t k4 = k / 4;
        for (uint32_t i0 = tid; i0 < k4; i0 += U * stride) {
            uint4 p[U], q[U];
#pragma unroll
            for (uint32_t u = 0; u < U; ++u) {
                const uint64_t i = uint64_t(i0) + uint64_t(u) * stride;
                if (i < k4) {
                    p[u] = ld_stream_v4(a + i * 4);
                    q[u] = ld_stream_v4(b + i * 4);
                }
            }
#pragma unroll
            for (uint32_t u = 0; u < U; ++u) {
                const uint64_t i = uint64_t(i0) + uint64_t(u) * stride;
                if (i < k4) {
                    __stcs(reinterpret_cast<uint4 *>(index + i * 8), make_uint4(p[u].x, q[u].x, p[u].y, q[u].y));
                    __stcs(reinterpret_cast<uint4 *>(index + i * 8 + 4), make_uint4(p[u].z, q[u].z, p[u].w, q[u].w));
                }
            }
        }
        for (uint32_t e = k4 * 4 + tid; e < k; e += stride) {
            index[2ull * e] = a[e];
            index[2ull * e + 1] = b[e];
        }
    } else {
        for (uint32_t e = tid; e < k; e += stride) {
            index[2ull * e] = a[e];
            index[2ull * e + 1] = b[e];
        }
    }
}

ka_status launch_prepare_index(const uint32_t *a, const uint32_t *b, uint64_t k, const uint32_t *k_ptr,
                               uint32_t *index, uint32_t *n_out, cudaStream_t stream) {
    if (k > 0x7FFFFFFFull || (k && (!a || !b || !index))) return KA_E_ARG;
    if (n_out && n_out == k_ptr) return KA_E_ARG;
    const int vec = aligned16(a) && aligned16(b) && aligned16(index);
    k_prepare_index<<<ew_grid((k + 3) / 4), kEwBlock, 0, stream>>>(a, b, k, k_ptr, index, n_out, vec);
    return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
__global__ void k_copy_count(const uint32_t *n_ptr, uint64_t n, uint32_t *n_out) {
    if (threadIdx.x == 0 && n_out) *n_out = live_n(n_ptr, n);
}

ka_status launch_copy_count(const uint32_t *n_ptr, uint64_t n, uint32_t *n_out, cudaStream_t stream) {
    k_copy_count<<<1, 32, 0, stream>>>(n_ptr, n, n_out);
    return cuda_status(cudaGetLastError());
}

// Result publication: n words from device memory (or, with src null, the
// value `fixed` as one word) and, when err is given, the device error word,
// stored straight into host-mapped pinned memory. One small launch stands in
// for device-to-host copies, whose copy-engine round trip costs several
// microseconds even for a single word. With dst_tag, the value `tag` is
// stored there last, after a system-scope fence: a host thread that reads
// the tag knows that the words before it, and all work issued on the stream
// before this launch, are complete (one block only).
__global__ void k_publish(const uint32_t *src, uint32_t n, uint32_t fixed, const uint32_t *err, uint32_t *dst,
                          uint32_t *dst_err, uint32_t *dst_tag, uint32_t tag) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (!src) {
        if (t == 0) dst[0] = fixed;
    } else {
        for (uint32_t i = t; i < n; i += blockDim.x * gridDim.x) dst[i] = src[i];
    }
    if (err && t == 0) *dst_err = *err;
    if (dst_tag) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence_system();
            *reinterpret_cast<volatile uint32_t *>(dst_tag) = tag;
        }
    }
}

ka_status launch_publish(const uint32_t *src, uint32_t n, uint32_t fixed, const uint32_t *err, uint32_t *dst,
                         uint32_t *dst_err, cudaStream_t stream, uint32_t *dst_tag, uint32_t tag) {
    if (!dst || (err && !dst_err)) return KA_E_ARG;
    const uint32_t blocks = src && n > 256 ? std::min<uint32_t>((n + 255) / 256, 16u) : 1u;
    if (dst_tag && blocks != 1) return KA_E_ARG;
    k_publish<<<blocks, 256, 0, stream>>>(src, n, fixed, err, dst, dst_err, dst_tag, tag);
    return cuda_status(cudaGetLastError());
}

// The empty stage: one launch that does no work (prices a message-passing stage).
__global__ void k_empty() {}

ka_status launch_empty(cudaStream_t stream) {
    k_empty<<<1, 32, 0, stream>>>();
    return cuda_status(cudaGetLastError());
}

}  // namespace ka

using namespace ka;

extern "C" {

ka_status ka_generate(uint32_t *d_out, uint64_t n, uint64_t seed, void *stream) {
    return launch_generate(d_out, n, seed, nullptr, static_cast<cudaStream_t>(stream));
}

ka_status ka_map_hash(const uint32_t *d_in, uint64_t n, const uint32_t *d_n, uint32_t *d_out, uint32_t *d_n_out,
                      void *stream) {
    return launch_map_hash(d_in, n, d_n, d_out, d_n_out, static_cast<cudaStream_t>(stream));
}

ka_status ka_predicate(const uint32_t *d_x, uint64_t n, const uint32_t *d_n, int32_t pred, uint32_t param,
                       uint32_t *d_flags, void *stream) {
    PredDev p;
    const ka_status s = make_pred(pred, param, &p);
    if (s != KA_OK) return s;
    return launch_predicate(d_x, n, d_n, p, d_flags, nullptr, static_cast<cudaStream_t>(stream));
}

ka_status ka_prepare_index(const uint32_t *d_chunk_ids, const uint32_t *d_literals, uint64_t k, const uint32_t *d_k,
                           uint32_t *d_index, uint32_t *d_n_out, void *stream) {
    return launch_prepare_index(d_chunk_ids, d_literals, k, d_k, d_index, d_n_out, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
