// Device helpers shared by the warp-specialised TMA kernels: mbarrier
// operations, bounded waits, bulk copies into shared memory, and the warp's
// realigning copy of a compacted segment to global memory.
#pragma once

#include "ka_dev.cuh"

namespace ka {
namespace tma {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }

// 32-bit store to a shared-memory address (a cvta-to-shared address).
__device__ __forceinline__ void st_shared_u32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *m) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(m)) : "memory");
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

// Non-blocking test of the same (try_wait may suspend the thread for a while
// when the phase is not complete; test_wait returns at once).
__device__ __forceinline__ bool mbar_test_wait(uint64_t *m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits until the phase of parity `parity` of m has completed. Gives up after
// kWaitNs of wall time and returns false.
constexpr uint64_t kWaitNs = 2000000000ull;
__device__ __forceinline__ bool mbar_wait(uint64_t *m, uint32_t parity) {
    if (mbar_try_wait(m, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(m, parity)) return true;
        if ((i & 15u) == 0u && global_ns() - t0 > kWaitNs) return false;
    }
}

// Bulk copy global -> this block's shared memory, completing on mbarrier m.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *m) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(m))
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

constexpr int kSeg = 512;         // entries per compute warp and tile (32 lanes x 4 rows x 4)


// The 4-entry keep mask for predicate kind PK (-1: the kind in p, chosen at
// run time).
template <int PK>
__device__ __forceinline__ uint32_t mask4_of(const PredDev &p, uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3) {
    if constexpr (PK < 0) return pred_mask4(p, x0, x1, x2, x3);
    else if constexpr (PK == kAll) return 0xFu;
    else return mask4_k<PK>(p, x0, x1, x2, x3);
}

// One warp counts the kept entries of its 512-entry segment (entries
// [vlo, vhi) are input entries; the others are ignored) and compacts them in
// place at the segment's front, in order. Returns the count.
template <int PK>
__device__ __forceinline__ uint32_t compact_segment(uint32_t *seg, const PredDev &pred, uint32_t mul, uint32_t vlo,
                                                    uint32_t vhi, int lane) {
    constexpr int ROWS = 4;
    uint32_t v[ROWS][4], m[ROWS], packed = 0;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const uint32_t e0 = uint32_t(r * 128 + lane * 4);
        const uint4 q = *reinterpret_cast<const uint4 *>(seg + e0);
        v[r][0] = q.x;
        v[r][1] = q.y;
        v[r][2] = q.z;
        v[r][3] = q.w;
    }
    if (mul != 1u) {
#pragma unroll
        for (int r = 0; r < ROWS; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) v[r][c] *= mul;
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const uint32_t e0 = uint32_t(r * 128 + lane * 4);
        uint32_t mk = mask4_of<PK>(pred, v[r][0], v[r][1], v[r][2], v[r][3]);
        if (vlo != 0u || vhi != uint32_t(kSeg)) {
            const uint32_t skip = vlo > e0 ? min(vlo - e0, 4u) : 0u;
            const uint32_t left = vhi > e0 ? vhi - e0 : 0u;
            mk &= (0xFu << skip) & (left >= 4 ? 0xFu : ((1u << left) - 1u));
        }
        m[r] = mk;
        packed += uint32_t(__popc(mk)) << (8 * r);
    }
    // per-row counts, 8 bits each (a row of the warp keeps at most 128)
    const uint32_t incl = warp_incl_scan(packed, lane);
    const uint32_t excl = incl - packed;
    const uint32_t rows = __shfl_sync(kFull, incl, 31);
    __syncwarp();  // every lane holds its entries before any is overwritten
    uint32_t rowbase = 0;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        uint32_t pos = rowbase + ((excl >> (8 * r)) & 0xFFu);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if ((m[r] >> c) & 1u) seg[pos++] = v[r][c];
        }
        rowbase += (rows >> (8 * r)) & 0xFFu;
    }
    return rowbase;
}

// One warp copies cnt compacted entries from shared memory (16-byte aligned)
// to dst (4-byte aligned): single entries up to dst's next 16-byte boundary,
// then 16-byte stores, each assembled from two aligned 16-byte shared loads,
// then the remaining single entries. cnt <= kSeg.
// The 16-byte loops are kept rolled: a lane makes at most 4 trips, and in a
// kernel with registers to spare the compiler unrolled them into predicated
// stores that issue even when switched off. Those cost the held write-out
// throughput (same array, same process: 273 -> 263 us at 50 % kept and 346
// -> 324 us at 99 % in the five-stage shape, 352 -> 338 us at 99 % in the
// four-stage one; the store instructions dropped from 578 K to 508 K).
__device__ __forceinline__ void warp_copy_out(const uint32_t *src, uint32_t *dst, uint32_t cnt, int lane) {
    const uint32_t to16 = uint32_t((16u - (reinterpret_cast<uintptr_t>(dst) & 15u)) & 15u) >> 2;
    const uint32_t head = to16 < cnt ? to16 : cnt;
    if (uint32_t(lane) < head) dst[lane] = src[lane];
    const uint32_t body = (cnt - head) >> 2;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst + head);
    // Output chunk i holds src[head + 4i .. head + 4i + 3]: the tail of source
    // chunk i and the front of chunk i + 1 (index <= 127 since cnt <= 512).
    switch (head) {
    case 0:
#pragma unroll 1
        for (uint32_t i = uint32_t(lane); i < body; i += 32) d4[i] = s4[i];
        break;
    case 1:
#pragma unroll 1
        for (uint32_t i = uint32_t(lane); i < body; i += 32) {
            const uint4 x = s4[i], y = s4[i + 1];
            d4[i] = make_uint4(x.y, x.z, x.w, y.x);
        }
        break;
    case 2:
#pragma unroll 1
        for (uint32_t i = uint32_t(lane); i < body; i += 32) {
            const uint4 x = s4[i], y = s4[i + 1];
            d4[i] = make_uint4(x.z, x.w, y.x, y.y);
        }
        break;
    default:
#pragma unroll 1
        for (uint32_t i = uint32_t(lane); i < body; i += 32) {
            const uint4 x = s4[i], y = s4[i + 1];
            d4[i] = make_uint4(x.w, y.x, y.y, y.z);
        }
        break;
    }
    const uint32_t t0 = head + 4 * body;
    if (uint32_t(lane) < cnt - t0) dst[t0 + lane] = src[t0 + lane];
}

}  // namespace tma
}  // namespace ka
