// Device-side building blocks shared by the stage kernels of libka.
//
// Single-pass scans here use decoupled look-back (Merrill & Garland, "Single-
// pass Parallel Prefix Scan with Decoupled Look-back", NVIDIA TR 2016): each
// tile publishes its aggregate as soon as it is known, then walks back over
// its predecessors' published words until it meets an inclusive prefix.
//
// Status word of one tile (64 bits, written and read as one relaxed atomic
// access, so flag and value always travel together):
//     bits  0..31  value (aggregate or inclusive prefix, mod 2^32)
//     bits 32..33  flag: 0 invalid, 1 aggregate, 2 inclusive prefix, 3 error
//     bits 34..63  launch epoch (30 bits)
// A word from an earlier launch carries an older epoch and reads as invalid,
// so the status array never has to be cleared between launches.
//
// Tile tickets: one 64-bit word per workspace, high half = epoch, low half =
// tickets handed out in the current launch. Blocks take tiles in ticket
// order (never by blockIdx), which guarantees every predecessor of a tile
// belongs to a block that is already running. The block that takes the very
// last ticket of a launch (tiles + gridDim.x tickets in all, since every block
// stops after its first ticket past the end) resets the count and advances
// the epoch for the next launch on the same workspace.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ka {

constexpr uint32_t kFlagInvalid = 0;
constexpr uint32_t kFlagAggregate = 1;
constexpr uint32_t kFlagInclusive = 2;
constexpr uint32_t kFlagError = 3;
constexpr uint32_t kEpochMask = 0x3FFFFFFFu;

// Device error codes (same values as the ka_status codes of ka.h).
constexpr uint32_t kDevErrTimeout = 7;     // -KA_E_DEVICE_TIMEOUT
constexpr uint32_t kDevErrWorkspace = 13;  // -KA_E_WORKSPACE

constexpr uint32_t kDefaultSpinLimit = 1u << 22;

// Workspace header: 256 bytes at the start of every single-pass workspace.
struct WsHeader {
    unsigned long long ticket;  // (epoch << 32) | tickets taken
    uint32_t error;             // first device error (0: none)
    uint32_t error_tile;        // tile that recorded it
    uint32_t spin_limit;        // polls before a look-back gives up (0: default)
    uint32_t magic;             // kWsMagic once initialised
    uint32_t reserved[58];
};
static_assert(sizeof(WsHeader) == 256, "workspace header is 256 bytes");
constexpr uint32_t kWsMagic = 0x4B415753u;  // "KAWS"

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t pack_status(uint32_t epoch, uint32_t flag, uint32_t value) {
    return (uint64_t(epoch & kEpochMask) << 34) | (uint64_t(flag) << 32) | uint64_t(value);
}

// Streaming 128-bit load of read-once input (not kept in L1).
__device__ __forceinline__ uint4 ld_stream_v4(const uint32_t *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ uint32_t ld_stream_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void record_error(WsHeader *ws, uint32_t code, uint32_t tile) {
    if (atomicCAS(&ws->error, 0u, code) == 0u) ws->error_tile = tile;
}

// ---------------------------------------------------------------------------
// Predicates, canonicalised on the host (see make_pred in ka_internal.h):
//   kAndMaskEq0: keep (x & a) == 0
//   kLt:         keep x < a            (also (x >> 28) < p, as x < p << 28)
//   kPopcOdd:    keep popcount(x) odd
//   kModNe0:     keep x % d != 0, d = 2^c * d' (d' odd), tested without a
//                division: x is a multiple of d iff its low c bits are zero and
//                (x >> c) * inverse(d') mod 2^32 <= floor((2^32 - 1) / d')
//                (Granlund & Montgomery 1994, divisibility by an invariant
//                integer). a = inverse(d'), b = that bound, c = low-bit mask.
//   kNe:         keep x != a
//   kAll:        keep everything
// ---------------------------------------------------------------------------
enum PredKind : int32_t { kAndMaskEq0 = 0, kLt = 1, kPopcOdd = 3, kModNe0 = 4, kNe = 5, kAll = 6 };

struct PredDev {
    int32_t kind;
    uint32_t a, b, c, d;  // see the table above; d = shift c of kModNe0
};

__host__ __device__ __forceinline__ uint32_t popc32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return __popc(x);
#else
    return (uint32_t)__builtin_popcount(x);
#endif
}

// Inverse of an odd d modulo 2^32 by Newton iteration: x <- x (2 - d x)
// doubles the number of correct low bits each step, starting from x = d
// (correct to 3 bits for odd d).
__host__ __device__ __forceinline__ uint32_t inverse_odd(uint32_t d) {
    uint32_t x = d;
    for (int i = 0; i < 5; ++i) x *= 2u - d * x;
    return x;
}

// Canonical predicate for an API (kind, param): 0 on success, -1 for an
// unknown kind or a zero modulus. Kind numbers are those of ka_pred_kind.
__host__ __device__ __forceinline__ int pred_canon(int32_t kind, uint32_t param, PredDev *out) {
    PredDev p{};
    switch (kind) {
    case 0: p.kind = kAndMaskEq0; p.a = param; break;  // KA_PRED_AND_MASK_EQ0
    case 1: p.kind = kLt; p.a = param; break;          // KA_PRED_LT
    case 2:                                            // KA_PRED_TOPBITS_LT
        // (x >> 28) < p  <=>  x < p * 2^28 for p <= 15; every x passes for p >= 16.
        if (param >= 16u) {
            p.kind = kAll;
        } else {
            p.kind = kLt;
            p.a = param << 28;
        }
        break;
    case 3: p.kind = kPopcOdd; break;                  // KA_PRED_POPC_ODD
    case 4: {                                          // KA_PRED_MOD_NE0
        if (param == 0u) return -1;
        uint32_t shift = 0, odd = param;
        while ((odd & 1u) == 0u) {
            odd >>= 1;
            ++shift;
        }
        p.kind = kModNe0;
        p.a = inverse_odd(odd);
        p.b = 0xFFFFFFFFu / odd;
        p.c = shift == 0 ? 0u : (0xFFFFFFFFu >> (32 - shift));
        p.d = shift;
        break;
    }
    case 5: p.kind = kNe; p.a = param; break;          // KA_PRED_NE
    case 6: p.kind = kAll; break;                      // KA_PRED_ALL
    default: return -1;
    }
    *out = p;
    return 0;
}

template <int K>
__host__ __device__ __forceinline__ bool keep_k(const PredDev &p, uint32_t x) {
    if (K == kAndMaskEq0) return (x & p.a) == 0u;
    if (K == kLt) return x < p.a;
    if (K == kPopcOdd) return (popc32(x) & 1u) != 0u;
    if (K == kModNe0) return !(((x & p.c) == 0u) && ((x >> p.d) * p.a) <= p.b);
    if (K == kNe) return x != p.a;
    return true;
}

__host__ __device__ __forceinline__ bool pred_keep(const PredDev &p, uint32_t x) {
    switch (p.kind) {
    case kAndMaskEq0: return keep_k<kAndMaskEq0>(p, x);
    case kLt: return keep_k<kLt>(p, x);
    case kPopcOdd: return keep_k<kPopcOdd>(p, x);
    case kModNe0: return keep_k<kModNe0>(p, x);
    case kNe: return keep_k<kNe>(p, x);
    default: return true;
    }
}

template <int K>
__device__ __forceinline__ uint32_t mask4_k(const PredDev &p, uint32_t x0, uint32_t x1, uint32_t x2,
                                            uint32_t x3) {
    return uint32_t(keep_k<K>(p, x0)) | (uint32_t(keep_k<K>(p, x1)) << 1) |
           (uint32_t(keep_k<K>(p, x2)) << 2) | (uint32_t(keep_k<K>(p, x3)) << 3);
}

// Keep-mask of four consecutive entries (bit j = entry j kept). The switch is
// on a value uniform across the block, so it costs one uniform branch per
// four entries.
__device__ __forceinline__ uint32_t pred_mask4(const PredDev &p, uint32_t x0, uint32_t x1, uint32_t x2,
                                               uint32_t x3) {
    switch (p.kind) {
    case kAndMaskEq0: return mask4_k<kAndMaskEq0>(p, x0, x1, x2, x3);
    case kLt: return mask4_k<kLt>(p, x0, x1, x2, x3);
    case kPopcOdd: return mask4_k<kPopcOdd>(p, x0, x1, x2, x3);
    case kModNe0: return mask4_k<kModNe0>(p, x0, x1, x2, x3);
    case kNe: return mask4_k<kNe>(p, x0, x1, x2, x3);
    default: return 0xFu;
    }
}

// ---------------------------------------------------------------------------
// Warp helpers.
// ---------------------------------------------------------------------------
constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}

// Inclusive scan across the lanes of a warp (mod 2^32, or field-wise on
// packed counters whose fields cannot carry).
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, v, d);
        if (lane >= d) v += y;
    }
    return v;
}

__device__ __forceinline__ uint64_t warp_incl_scan64(uint64_t v, int lane, int width) {
    for (int d = 1; d < width; d <<= 1) {
        const uint64_t y = __shfl_up_sync(kFull, v, d);
        if (lane >= d) v += y;
    }
    return v;
}

// Four 8-bit fields -> four 16-bit fields.
__device__ __forceinline__ uint64_t spread8to16(uint32_t x) {
    return uint64_t(x & 0xFFu) | (uint64_t((x >> 8) & 0xFFu) << 16) | (uint64_t((x >> 16) & 0xFFu) << 32) |
           (uint64_t(x >> 24) << 48);
}

// ---------------------------------------------------------------------------
// Status entries are spread kStatusStride words apart (one 32-byte sector
// each): hundreds of blocks poll the most recent entries, and packing them
// into a few cache lines turns those lines into an L2 hot spot (measured on
// GB300: 34% of HBM bandwidth packed, 52-58% spread, same kernel).
// ---------------------------------------------------------------------------
constexpr int kStatusStride = 4;

__device__ __forceinline__ uint64_t *status_at(uint64_t *status, uint64_t idx) {
    return status + idx * kStatusStride;
}

// Brings the sector holding *p into L2 ahead of its first use.
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// ---------------------------------------------------------------------------
// Decoupled look-back, run by one full warp for tile `tile` whose first tile
// of its segment is `first_tile` (0 for a single array; the first tile of
// an instance in a batch). Publishes the tile's aggregate (or, for the first
// tile, its inclusive prefix), walks back 32 predecessors per poll until it
// meets an inclusive prefix, then publishes its own. Returns the exclusive
// prefix. Every poll loop is bounded by `spin_limit`; on time-out, or when a
// predecessor reports an error, the tile publishes the error flag (so its
// successors stop at once), the first error is recorded in the workspace
// header, and *err is set. (A wider window - several loads per lane - was
// measured slower: the extra status traffic costs more than the round trips
// it saves.)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t lookback_warp(uint64_t *status, uint32_t tile, uint32_t first_tile,
                                                  uint32_t epoch, uint32_t aggregate, uint32_t spin_limit,
                                                  WsHeader *ws, bool *err) {
    const int lane = threadIdx.x & 31;
    if (tile == first_tile) {
        if (lane == 0) st_relaxed_u64(status_at(status, tile), pack_status(epoch, kFlagInclusive, aggregate));
        *err = false;
        return 0u;
    }
    if (lane == 0) st_relaxed_u64(status_at(status, tile), pack_status(epoch, kFlagAggregate, aggregate));
    uint32_t exclusive = 0;
    bool failed = false;
    int64_t window = int64_t(tile) - 1;
    const uint32_t want_epoch = epoch & kEpochMask;
    for (;;) {
        const int64_t idx = window - lane;
        uint32_t flag = kFlagInclusive, value = 0;
        uint32_t polls = 0, sleep_ns = 0;
        for (;;) {
            if (idx >= int64_t(first_tile)) {
                const uint64_t s = ld_relaxed_u64(status_at(status, uint64_t(idx)));
                flag = uint32_t(s >> 34) == want_epoch ? uint32_t(s >> 32) & 3u : kFlagInvalid;
                value = uint32_t(s);
            }
            if (__all_sync(kFull, flag != kFlagInvalid)) break;
            if (++polls >= spin_limit) {
                failed = true;
                break;
            }
            if (polls > 4) {
                __nanosleep(sleep_ns);
                sleep_ns = sleep_ns < 128 ? sleep_ns * 2 + 32 : 128;
            }
        }
        if (failed) {
            if (lane == 0) record_error(ws, kDevErrTimeout, tile);
            break;
        }
        const uint32_t stop = __ballot_sync(kFull, flag >= kFlagInclusive);
        if (stop) {
            const int first = __ffs(stop) - 1;
            exclusive += warp_sum(lane <= first ? value : 0u);
            failed = __shfl_sync(kFull, flag, first) == kFlagError;
            break;
        }
        exclusive += warp_sum(value);
        window -= 32;
    }
    if (lane == 0)
        st_relaxed_u64(status_at(status, tile),
                       pack_status(epoch, failed ? kFlagError : kFlagInclusive, exclusive + aggregate));
    *err = failed;
    return exclusive;
}

// Ticket for the next tile. Called by one thread. Returns the ticket and sets
// *epoch; performs the end-of-launch reset when it draws the last ticket.
__device__ __forceinline__ uint32_t take_ticket(WsHeader *ws, uint32_t live_tiles, uint32_t *epoch,
                                                bool *was_last) {
    const unsigned long long t = atomicAdd(&ws->ticket, 1ull);
    const uint32_t ticket = uint32_t(t);
    *epoch = uint32_t(t >> 32);
    *was_last = false;
    if (ticket >= live_tiles && ticket == live_tiles + gridDim.x - 1) {
        *was_last = true;
        atomicExch(&ws->ticket, (unsigned long long)(*epoch + 1u) << 32);
    }
    return ticket;
}

}  // namespace ka
