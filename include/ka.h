/*
 * ka.h - C ABI of libka.so: order-preserving stream compaction run as composed
 * kernel actors on GPU-resident data (GB300, sm_103a).
 *
 * The calls follow the programming model of Hiesgen, Charousset and Schmidt,
 * "OpenCL Actors - Adding Data Parallelism to Actor-based Programming with CAF"
 * (arXiv 1709.07781):
 *   - a kernel actor wraps one data-parallel stage (Sec. 3.2, 3.4);
 *   - messages carry references to device buffers, typed and sized, so the
 *     next stage runs on the same memory (Sec. 3.5, the mem_ref type);
 *   - actors compose as C = B (.) A, C(msg) = B(A(msg)) (Sec. 3.5);
 *   - the first stage uploads, the last reads back and answers the requester
 *     (Sec. 3.5);
 *   - a configuration word carries the element count into a stage and the new
 *     length out of a compaction (Sec. 4.1);
 *   - a device reference cannot be serialised (Sec. 3.5, option (a)).
 * The compaction itself is the one of Sec. 4.1: remove every entry that fails
 * a test, keep the rest in order; the paper runs it as flag, prefix sum and
 * move phases (Listing 5). Here it also exists as one fused single-pass kernel
 * (the "several kernels inside one actor" alternative of Sec. 3.6).
 *
 * Conventions for every call:
 *   - Every call returns a ka_status; outputs are written only on KA_OK.
 *     No C++ exception crosses this boundary.
 *   - "d_" arguments are device pointers (cudaMalloc, a pool, or a torch
 *     tensor's data_ptr); "h_" arguments are host pointers. The library never
 *     takes ownership of caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Kernel calls are asynchronous on that stream; device-side
 *     failures (a look-back that timed out) are recorded in the workspace and
 *     read back by ka_workspace_status.
 *   - Element type is uint32. Lengths are uint64 in the API; a single array is
 *     limited to 2^32 - 1 elements (device counts are uint32).
 *   - Live lengths: where a call takes (n, d_n), d_n == NULL means n is the
 *     live length; otherwise n is the capacity (it sizes the launch) and the
 *     live length is min(*d_n, n), read on the device. This is how a stage
 *     consumes the previous stage's result without a host round trip.
 *   - Handles (ka_system, ka_ref, ka_actor, ka_request_h) are opaque and are
 *     released by the caller with the matching release call.
 */
#ifndef KA_H
#define KA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------ */
/* Status codes                                                             */
/* ------------------------------------------------------------------------ */
typedef int32_t ka_status;
#define KA_OK                   0
#define KA_E_ARG               -1  /* bad argument (null pointer, size, alias)          */
#define KA_E_TYPE              -2  /* message does not match the actor's signature      */
#define KA_E_OOM               -3  /* device or host allocation failed                  */
#define KA_E_BUDGET            -4  /* request larger than the memory budget             */
#define KA_E_STALE             -5  /* handle already released                           */
#define KA_E_CUDA              -6  /* a CUDA runtime call failed                        */
#define KA_E_DEVICE_TIMEOUT    -7  /* a bounded device-side wait gave up                */
#define KA_E_CLOSED            -8  /* system or mailbox closed                          */
#define KA_E_NOT_SERIALIZABLE  -9  /* device references never leave the process        */
#define KA_E_TIMEOUT          -10  /* host-side wait (ka_receive) timed out             */
#define KA_E_UNSUPPORTED      -11  /* option not supported                              */
#define KA_E_INJECTED         -12  /* failure injected on the host by a test hook       */
#define KA_E_WORKSPACE        -13  /* workspace too small or not initialised            */
#define KA_E_TOO_LARGE        -14  /* size above ka_compact_static's limit              */

/* Text for a status code (static storage). */
const char *ka_strerror(ka_status s);
/* Library version: major * 100 + minor. */
int32_t ka_version(void);
/* The cudaError_t value behind the last KA_E_CUDA that a call made on this
 * thread returned (0 if none has). */
int32_t ka_last_cuda_error(void);

/* ------------------------------------------------------------------------ */
/* Predicates: which entries a compaction keeps (Sec. 4.1 removes entries    */
/* equal to a given value; KA_PRED_NE is that case, the others generalise it */
/* to a keep-test).                                                         */
/* ------------------------------------------------------------------------ */
typedef enum ka_pred_kind {
    KA_PRED_AND_MASK_EQ0 = 0, /* keep (x & param) == 0                     */
    KA_PRED_LT = 1,           /* keep x < param                            */
    KA_PRED_TOPBITS_LT = 2,   /* keep (x >> 28) < param                    */
    KA_PRED_POPC_ODD = 3,     /* keep popcount(x) odd (param ignored)      */
    KA_PRED_MOD_NE0 = 4,      /* keep x % param != 0; param == 0: KA_E_ARG */
    KA_PRED_NE = 5,           /* keep x != param                           */
    KA_PRED_ALL = 6           /* keep every entry (a pure map stage)       */
} ka_pred_kind;

/* Value transform applied to each entry before its test; the transformed
 * value is what is tested and written. */
#define KA_XFORM_NONE 0u
#define KA_XFORM_HASH 1u      /* x -> x * 2654435761 mod 2^32 */

/* Tile shape of a tiled kernel: threads per block and items per thread.
 * Supported: block 128, 256 or 512 with ipt 4, 8 or 16, block 1024 with ipt
 * 4 or 8, and (768, 16); the batch kernel also takes (704, 16). The shapes
 * (256, 16), (512, 16), (704, 16) and (768, 16) select the warp-specialised
 * TMA kernels (compaction, scan, batch): compute warps of 512 entries each,
 * plus a look-back warp and a producer warp; block / 32 compute warps, except
 * that the compaction and the scan of (768, 16) have 26 (tiles of 13312
 * entries; its batch kernel has 24). A tile holds 512 to 13312 entries.
 * A NULL tile, or {0, 0}, picks the library default (or the autotuned shape
 * once ka_autotune has run for that kernel). */
typedef struct ka_tile {
    uint32_t block;
    uint32_t ipt;
} ka_tile;

/* ------------------------------------------------------------------------ */
/* Workspace of the single-pass kernels: a 256-byte header (tile ticket and  */
/* launch epoch, device error word, spin limit) followed by one 64-bit       */
/* status word per tile for the decoupled look-back. Caller-allocated device */
/* memory; initialise once with ka_workspace_init, then reuse for any number */
/* of launches ordered on one stream (each launch leaves it ready for the    */
/* next). Launches that may overlap on the GPU need separate workspaces.     */
/* ------------------------------------------------------------------------ */
ka_status ka_workspace_size(uint64_t capacity, const ka_tile *tile, uint64_t *bytes);
ka_status ka_workspace_init(void *d_ws, uint64_t bytes, void *stream);
/* Synchronises `stream`, then reads the device error word: *device_status is
 * KA_OK or the first device-side error (KA_E_DEVICE_TIMEOUT). */
ka_status ka_workspace_status(const void *d_ws, void *stream, ka_status *device_status);
/* Test hook: polls a look-back makes before it gives up (default 1 << 22,
 * about a second with back-off). Asynchronous on `stream`. */
ka_status ka_workspace_set_spin_limit(void *d_ws, uint32_t polls, void *stream);

/* ------------------------------------------------------------------------ */
/* Stage kernels, called directly (no actor layer).                          */
/* ------------------------------------------------------------------------ */

/* Seeded input: d_out[i] = high 32 bits of SplitMix64(seed, i), where
 * SplitMix64(seed, i) is the (i+1)-th output of the generator whose state
 * starts at `seed` (Steele, Lea & Flood 2014). Stands in for the upload the
 * paper's first stage performs (Sec. 3.5). */
ka_status ka_generate(uint32_t *d_out, uint64_t n, uint64_t seed, void *stream);

/* Hash map stage: d_out[i] = d_in[i] * 2654435761 mod 2^32 for i < live n.
 * d_n_out (optional) receives the live n, so the output carries its length. */
ka_status ka_map_hash(const uint32_t *d_in, uint64_t n, const uint32_t *d_n, uint32_t *d_out,
                      uint32_t *d_n_out, void *stream);

/* Phase 1 of Sec. 4.1 (flag map): d_flags[i] = P(x[i]) in {0, 1}, i < live n. */
ka_status ka_predicate(const uint32_t *d_x, uint64_t n, const uint32_t *d_n, int32_t pred,
                       uint32_t param, uint32_t *d_flags, void *stream);

/* Phase 2 of Sec. 4.1 (prefix sum): d_out[i] = sum_{j<i} d_in[j] mod 2^32 for
 * i < live n, and *d_total = the sum of all live entries (0 for n = 0).
 * Single pass with decoupled look-back; needs a workspace. d_out may equal d_in. */
ka_status ka_exclusive_scan(const uint32_t *d_in, uint64_t n, const uint32_t *d_n, uint32_t *d_out,
                            uint32_t *d_total, void *d_ws, uint64_t ws_bytes, const ka_tile *tile,
                            void *stream);

/* Phase 3 of Sec. 4.1 (move): d_out[d_offsets[i]] = d_x[i] for every i < live n
 * with d_flags[i] == 1. d_flags must hold 0/1 and d_offsets their exclusive
 * prefix sum (what ka_predicate and ka_exclusive_scan produce). */
ka_status ka_scatter(const uint32_t *d_x, const uint32_t *d_flags, const uint32_t *d_offsets,
                     uint64_t n, const uint32_t *d_n, uint32_t *d_out, void *stream);

/* Fused single-pass compaction (flag, scan and move in one kernel with
 * decoupled look-back): d_out[0..k) = the entries of x (after `xform`) that
 * pass the test, in input order; *d_count = k. Entries d_out[k..) are not
 * written. d_out may equal d_in (in place). d_count must not alias d_n. */
ka_status ka_compact(const uint32_t *d_in, uint64_t n, const uint32_t *d_n, int32_t pred,
                     uint32_t param, uint32_t xform, uint32_t *d_out, uint32_t *d_count,
                     void *d_ws, uint64_t ws_bytes, const ka_tile *tile, void *stream);

/* Compaction for callers that cannot allocate device memory. The paper has
 * no counterpart: it exists for code that is handed only the buffers it reads
 * and writes (plug-ins inside another framework's memory management, paths
 * that must not synchronise, which cudaMalloc and cudaFree may do), and so
 * cannot supply ka_compact's workspace.
 *
 * Same arguments and result as ka_compact without d_ws / ws_bytes: the
 * workspace is a fixed array of about 2 MiB inside the library, held by every
 * GPU on which the library's code is loaded until the process exits. The call
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 * The caller still owns d_in, d_out, d_count and d_n.
 *
 * Limit: n (the capacity when d_n is set) <= KA_STATIC_MAX_N = 2^24 entries;
 * a larger n returns KA_E_TOO_LARGE and launches nothing.
 * Set-up: the first call on a device (the current device) finds and clears
 * the array there, on `stream`, and waits for `stream`; make that first call
 * before any stream capture (during a capture it returns KA_E_UNSUPPORTED).
 * Every call on a device shares the one array, which keeps what the previous
 * call left in it; calls whose kernels overlap on the GPU (unordered streams)
 * race and give undefined results, so order them (one stream, or events).
 * A device-side failure (a look-back that gave up after its bounded wait) is
 * recorded in the shared array's header, like ka_compact's in its workspace:
 * read it with ka_workspace_status on the address ka_compact_static_workspace
 * returns; the count and output of a call after which it reports an error
 * are undefined. The error stays recorded (first error wins) until
 * ka_workspace_init is run on that address. */
#define KA_STATIC_MAX_N (1ull << 24)
ka_status ka_compact_static(const uint32_t *d_in, uint64_t n, const uint32_t *d_n, int32_t pred,
                            uint32_t param, uint32_t xform, uint32_t *d_out, uint32_t *d_count,
                            const ka_tile *tile, void *stream);
/* The shared array of the current device, as a workspace: *d_ws its device
 * address, *bytes its size. Allocates nothing; sets the array up as the first
 * ka_compact_static call does (same rule on stream capture) if no call has
 * yet. With it a caller checks a call (ka_workspace_status: synchronises
 * `stream`, copies the 256-byte header into host memory), clears a recorded
 * error (ka_workspace_init on `stream`, ordered after the calls), or sets the
 * spin limit (ka_workspace_set_spin_limit). Errors: KA_E_ARG (null output),
 * KA_E_UNSUPPORTED (first use during a capture, or device ordinal >= 64),
 * KA_E_CUDA. The paper has no counterpart. */
ka_status ka_compact_static_workspace(void *stream, void **d_ws, uint64_t *bytes);

/* Three-phase compaction (Sec. 4.1: count, prefix sum, move, after Billeter
 * et al.): per-segment kept counts (segments of 512 entries, one warp's
 * share), an exclusive scan of the counts, then each kept entry moved to its
 * segment's offset plus its rank in the segment. Same result as ka_compact;
 * reads the input twice. Workspace:
 * ka_three_phase_workspace_size bytes, 256-byte aligned, initialised once
 * with ka_workspace_init; ka_workspace_status on it reports a device-side
 * failure (a look-back of the counts' scan that gave up). d_count must not
 * alias d_n. */
ka_status ka_three_phase_workspace_size(uint64_t capacity, uint64_t *bytes);
ka_status ka_compact_three_phase(const uint32_t *d_in, uint64_t n, const uint32_t *d_n, int32_t pred,
                                 uint32_t param, uint32_t xform, uint32_t *d_out, uint32_t *d_count,
                                 void *d_ws, uint64_t ws_bytes, void *stream);

/* Compaction of a host array, streamed (the value mode of Sec. 3.5, where the
 * first actor uploads the data and the last reads the result back; the paper
 * has no streamed form). h_in[0..n) is uploaded in chunks of `chunk` entries
 * (0: 2^24), each chunk is compacted on the device once per predicate
 * p < n_pred (pred[p], param[p], xform[p] as for ka_compact), and the kept
 * entries of each chunk are copied back into h_out[p], after those of the
 * earlier chunks, as soon as the chunk's counts are known. Uploads of later
 * chunks, compactions and read-backs of earlier chunks overlap. On KA_OK,
 * count[p] is the number of kept entries and h_out[p][0..count[p]) holds them
 * in input order; h_out[p] needs room for n entries. n may exceed 2^32.
 * h_in and h_out[p] should be pinned (cudaHostAlloc or cudaHostRegister) for
 * the transfers to overlap; pageable memory gives the same result, slower.
 * d_scratch: ka_compact_host_scratch_size(chunk, n_pred) bytes of device
 * memory, 256-byte aligned, owned by the caller, needing no initialisation,
 * not used by anything else during the call. The call uses the current device
 * and streams of its own, serialises with other calls on that device, and
 * returns when the results are in host memory (every upload, kernel and copy
 * it issued has finished, also on error). Errors: KA_E_ARG (n_pred of 0 or
 * above KA_HOST_MAX_PRED, null pointers, chunk above 2^32 - 4, unaligned
 * scratch), KA_E_WORKSPACE (scratch too small), a predicate's error,
 * KA_E_CUDA, or a device status of the compaction (then h_out and count are
 * undefined). */
#define KA_HOST_MAX_PRED 4
ka_status ka_compact_host_scratch_size(uint64_t chunk, uint32_t n_pred, uint64_t *bytes);
ka_status ka_compact_host(const uint32_t *h_in, uint64_t n, uint32_t n_pred, const int32_t *pred,
                          const uint32_t *param, const uint32_t *xform, uint32_t *const *h_out, uint64_t *count,
                          uint64_t chunk, void *d_scratch, uint64_t scratch_bytes);

/* Escape-time Mandelbrot image, the paper's compute workload (Sec. 5.4):
 * d_out[y * width + x] = number of steps z <- z^2 + c taken from z = 0 while
 * |z|^2 <= 4, at most max_iter, for c = (re_min + x dre, im_min + y dim),
 * dre = (re_max - re_min) / width, dim = (im_max - im_min) / height, every
 * operation a single-precision IEEE operation in that order (no fused
 * multiply-add). The Mandelbrot actor stage uses the paper's rectangle
 * -0.5 - 0.7375i .. 0.1 - 0.1375i. width * height < 2^32. */
ka_status ka_mandelbrot(uint32_t *d_out, uint32_t width, uint32_t height, float re_min, float im_min,
                        float re_max, float im_max, uint32_t max_iter, void *stream);

/* Interleave of fuseFillsLiterals (Sec. 4.1, Listing 5): d_index[2i] =
 * d_chunk_ids[i], d_index[2i+1] = d_literals[i] for i < live k; d_n_out
 * (optional) receives 2 * live k. */
ka_status ka_prepare_index(const uint32_t *d_chunk_ids, const uint32_t *d_literals, uint64_t k,
                           const uint32_t *d_k, uint32_t *d_index, uint32_t *d_n_out, void *stream);

/* ------------------------------------------------------------------------ */
/* Batched compaction: many independent instances in one persistent launch.  */
/* ------------------------------------------------------------------------ */
typedef struct ka_batch_item {
    const uint32_t *in;     /* device input                                   */
    uint32_t *out;          /* device output, room for n entries (may = in)   */
    const uint32_t *n_ptr;  /* optional device live length (NULL: use n)      */
    uint32_t *count;        /* device word receiving the kept count           */
    uint32_t n;             /* length, or capacity when n_ptr is set          */
    int32_t pred;           /* ka_pred_kind                                   */
    uint32_t param;         /* predicate parameter                            */
    uint32_t xform;         /* KA_XFORM_*                                     */
} ka_batch_item;            /* 48 bytes */

/* Workspace for batches of up to `max_items` items whose inputs total at most
 * `total_capacity` entries. Layout: the 256-byte header, per-item plan
 * records (tile offset, canonical predicate, live length) for max_items items,
 * then one status word per tile. Initialise with ka_workspace_init. */
ka_status ka_batch_workspace_size(uint32_t max_items, uint64_t total_capacity, const ka_tile *tile,
                                  uint64_t *bytes);
/* Compacts every item of d_items (a device array of n_items descriptors, read
 * on the device, so a captured CUDA graph can be replayed over new contents):
 * item i's kept entries go to out_i[0..k_i) in order and *count_i = k_i.
 * max_items must be the value the workspace was sized for (it fixes the
 * layout); n_items <= max_items. `grid` = 0 picks one persistent block per SM
 * slot. Two launches: a plan kernel (one block per 256 items: live lengths,
 * canonical predicates, and per-item tile offsets by a scan chained across
 * its blocks through one status word per block; for the TMA shapes also the
 * item of each tile of an item of at most 8 tiles) and one persistent kernel
 * that walks the flattened (item, tile) ticket space with a decoupled
 * look-back per item. A workspace with fewer status words than
 * ceil(n_items / 256) returns KA_E_WORKSPACE (ka_batch_workspace_size always
 * leaves max_items + 1 or more). Because the plan records each live length
 * before any compaction runs, count_i may alias n_ptr_i (the paper's in_out
 * configuration word). An invalid item
 * (unknown predicate, zero modulus) gets count 0 and sets the workspace error
 * KA_E_ARG; more tiles than the workspace holds set KA_E_WORKSPACE. */
ka_status ka_compact_batch(const ka_batch_item *d_items, uint32_t n_items, uint32_t max_items, void *d_ws,
                           uint64_t ws_bytes, const ka_tile *tile, uint32_t grid, void *stream);

/* Seeded input for many buffers at once: out_i[j] = hi32(SplitMix64(seed_i, j))
 * for j < n_i (the batched form of ka_generate). d_items is a device array;
 * the workspace is one sized by ka_batch_workspace_size for max_items items. */
typedef struct ka_gen_item {
    uint32_t *out;
    uint64_t seed;
    uint32_t n;
    uint32_t pad;
} ka_gen_item;              /* 24 bytes */
ka_status ka_generate_batch(const ka_gen_item *d_items, uint32_t n_items, uint32_t max_items, void *d_ws,
                            uint64_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* Autotuner: times each tile shape of a kernel on the current device with   */
/* CUDA events and keeps the fastest per size bucket (a power of two of n),  */
/* in memory and in a small JSON cache file.                                 */
/* ------------------------------------------------------------------------ */
#define KA_KERNEL_COMPACT 0
#define KA_KERNEL_SCAN    1
#define KA_KERNEL_BATCH   2
/* COMPACT and SCAN: one array of n entries, keep x < 2^31. BATCH: a synthetic
 * batch of at most 4096 instances with sizes log-uniform in 2^8..2^20 and
 * n entries in total; its result applies to every batch (ka_compact_batch
 * looks up one entry). Allocates its inputs with cudaMalloc and synchronises
 * `stream`; do not call it during a stream capture. */
ka_status ka_autotune(int32_t kernel, uint64_t n, const char *cache_path, ka_tile *best,
                      float *best_us, void *stream);
/* Shape the library uses for (kernel, n) now (default or autotuned). */
ka_status ka_tile_for(int32_t kernel, uint64_t n, ka_tile *tile);
ka_status ka_autotune_load(const char *cache_path);

/* ------------------------------------------------------------------------ */
/* Actor layer (Sec. 3.2-3.5).                                              */
/* ------------------------------------------------------------------------ */
typedef struct ka_system ka_system;
typedef struct ka_ref ka_ref;
typedef struct ka_actor ka_actor;
typedef struct ka_request_h ka_request_h;

typedef struct ka_config {
    int32_t device;              /* CUDA device ordinal                                */
    int32_t debug;               /* 1: check the device error word after each request */
    void *stream;                /* borrowed cudaStream_t; NULL: the system makes one */
    uint64_t budget_bytes;       /* device memory budget of the pool (0: 64 GiB)      */
    const char *autotune_cache;  /* JSON cache file to load, or NULL                  */
} ka_config;

typedef enum ka_dtype { KA_U32 = 0 } ka_dtype;
typedef enum ka_access { KA_READ = 1, KA_WRITE = 2, KA_READ_WRITE = 3 } ka_access;

ka_status ka_system_create(const ka_config *cfg, ka_system **out);
/* Stops the dispatcher. Fails with KA_E_ARG while requests are in flight
 * unless force != 0 (then queued requests fail with KA_E_CLOSED and launched
 * ones finish). Afterwards every handle of the system (its requests,
 * references and actors) is invalid: calls on it return KA_E_STALE. Borrowed
 * memory stays the caller's; pool memory is returned. */
ka_status ka_system_destroy(ka_system *sys, int32_t force);
/* Bytes of pool memory held by live references. */
ka_status ka_system_pool_bytes(ka_system *sys, uint64_t *in_use, uint64_t *budget);

/* A reference to device memory (the paper's mem_ref<T>): element type, live
 * length, capacity, access rights. ka_ref_wrap borrows caller memory (the
 * caller keeps it alive until every request using it has been received);
 * ka_ref_alloc takes memory from the system's pool and returns it when the
 * last holder releases it. */
ka_status ka_ref_wrap(ka_system *sys, void *d_ptr, uint64_t n, uint64_t capacity, ka_dtype dtype,
                      ka_access access, ka_ref **out);
ka_status ka_ref_alloc(ka_system *sys, uint64_t capacity, ka_dtype dtype, ka_ref **out);
/* Live length (waits for the work that produces it). */
ka_status ka_ref_count(ka_ref *ref, uint64_t *n);
ka_status ka_ref_info(ka_ref *ref, void **d_ptr, uint64_t *capacity, int32_t *dtype, int32_t *access);
ka_status ka_ref_retain(ka_ref *ref);
ka_status ka_ref_release(ka_ref *ref);
/* Device references are process-local: always KA_E_NOT_SERIALIZABLE. */
ka_status ka_ref_serialize(const ka_ref *ref, void *buf, uint64_t cap, uint64_t *written);

typedef enum ka_stage_kind {
    KA_STAGE_GENERATE = 0,  /* () -> (x)          seed from the message          */
    KA_STAGE_MAP_HASH = 1,  /* (x) -> (h)                                        */
    KA_STAGE_PREDICATE = 2, /* (x) -> (x, f)                                     */
    KA_STAGE_EXSCAN = 3,    /* (x, f) -> (x, f, o)   o's count word = total      */
    KA_STAGE_SCATTER = 4,   /* (x, f, o) -> (y)                                  */
    KA_STAGE_COMPACT = 5,   /* (x) -> (y)            fused single pass           */
    KA_STAGE_PREPARE = 6,   /* (a, b) -> (index)     interleave, 2k entries      */
    KA_STAGE_EMPTY = 7,     /* (x) -> (x)            empty kernel, overhead probe */
    KA_STAGE_MANDELBROT = 8 /* () -> (image)         Sec. 5.4 region; pred = width,
                               xform = height, param = iterations (see ka_mandelbrot) */
} ka_stage_kind;

typedef struct ka_stage_desc {
    int32_t kind;    /* ka_stage_kind                  */
    int32_t pred;    /* ka_pred_kind (PREDICATE, COMPACT) */
    uint32_t param;
    uint32_t xform;  /* KA_XFORM_* (COMPACT)           */
    ka_tile tile;    /* {0, 0}: default / autotuned    */
} ka_stage_desc;

ka_status ka_spawn_stage(ka_system *sys, const ka_stage_desc *desc, ka_actor **out);
/* C = B (.) A: messages to C go to A, A's result goes to B (Sec. 3.5).
 * KA_E_TYPE if A's result arity differs from B's input arity. The composite
 * holds its own references to A and B. */
ka_status ka_compose(ka_actor *b, ka_actor *a, ka_actor **c_out);
/* Arity of an actor's input and result messages. */
ka_status ka_actor_arity(ka_actor *actor, int32_t *in_refs, int32_t *out_refs);
ka_status ka_actor_release(ka_actor *actor);

#define KA_MSG_MAX_REFS 4
typedef struct ka_msg {
    uint32_t n_refs;
    ka_ref *refs[KA_MSG_MAX_REFS];
    /* value mode, in: the first stage uploads h_in[0..h_n) into a pool buffer
     * that replaces refs[0] (Sec. 3.5: the first actor transfers the data). */
    const uint32_t *h_in;
    uint64_t h_n;
    /* value mode, out: the last stage reads the result back into
     * h_out[0..h_out_cap) (Sec. 3.5: the last actor reads back). */
    uint32_t *h_out;
    uint64_t h_out_cap;
    uint64_t seed;       /* for KA_STAGE_GENERATE */
    uint64_t gen_n;      /* for KA_STAGE_GENERATE */
    /* filled by ka_receive */
    uint64_t count;      /* live length of the result's first reference */
    ka_status status;
} ka_msg;

/* Sends `in` to the actor and returns at once. The caller keeps ownership of
 * the references in `in` (the request holds its own). */
ka_status ka_request(ka_actor *actor, const ka_msg *in, ka_request_h **out);
/* Waits up to timeout_ns (< 0: forever) for the response. On KA_OK, *out holds
 * the result: its references (owned by the caller, release them) and count;
 * in value mode the data is in h_out. A stage failure is returned as that
 * stage's status; the request's references are released. The handle is freed
 * by a KA_OK or error return, but not by KA_E_TIMEOUT (call again). */
ka_status ka_receive(ka_request_h *req, int64_t timeout_ns, ka_msg *out);

/* Host evaluation of the predicate exactly as the kernels evaluate it (after
 * the library's canonicalisation, e.g. the division-free modulus test); lets
 * a CPU test compare it with the plain definition. *keep = 0 or 1. */
ka_status ka_debug_pred_keep(int32_t pred, uint32_t param, uint32_t x, int32_t *keep);
/* Test hook for the per-device launch caches (no GPU needed): looks up
 * devices[i] in order in a fresh cache whose computation for lookup i
 * returns values[i], and writes what each lookup returned to out[i]. A value
 * is cached per device ordinal only when positive, and only for ordinals
 * below 64. */
ka_status ka_debug_device_cache(const int32_t *devices, const int32_t *values, uint32_t n, int32_t *out);

/* Test hooks (host-side fault injection; no GPU fault involved). */
ka_status ka_debug_fail_stage(ka_actor *stage_actor, int32_t fail_after);  /* -1: off */
ka_status ka_debug_kill_dispatcher(ka_system *sys);
typedef void (*ka_monitor_fn)(void *user, ka_status reason);
/* Called once from the system's threads when the dispatcher dies (link/monitor
 * notification, Sec. 2.1). */
ka_status ka_system_monitor(ka_system *sys, ka_monitor_fn fn, void *user);

/* ------------------------------------------------------------------------ */
/* Native timing loops for the actor-overhead measurement (Sec. 5.2-5.3: an   */
/* actor against the same kernels driven directly, task after task).         */
/* ------------------------------------------------------------------------ */
/* Sends `msg` to `actor` iters times with at most `inflight` requests
 * outstanding (1 = each request waits for the previous response), releases
 * every result, and returns the wall time in *seconds and the last result
 * length in *last_count. */
ka_status ka_bench_request_loop(ka_actor *actor, const ka_msg *msg, uint32_t iters, uint32_t inflight,
                                double *seconds, uint64_t *last_count);
/* The same stage chain launched directly (no actor layer) on `stream`,
 * iters times, each followed by a read-back of the result length (a
 * one-thread kernel storing it into host-mapped memory) and a wait. flags 0:
 * the wait is cudaStreamSynchronize, as plain CUDA code would wait.
 * KA_BENCH_WAIT_TAG: the wait is the one ka_receive uses (a completion tag
 * that the same kernel stores last, polled in host memory; an event when the
 * length is known on the host), so the two loops differ only by the actor
 * layer. Buffers are allocated once; three untimed warm-up runs. A first
 * stage KA_STAGE_PREPARE (the interleave of fuseFillsLiterals) reads its two
 * inputs from d_in: n chunk ids, then n literals. */
#define KA_BENCH_WAIT_TAG 1u
ka_status ka_bench_direct_chain(const ka_stage_desc *stages, uint32_t n_stages, const uint32_t *d_in, uint64_t n,
                                uint32_t iters, void *stream, uint32_t flags, double *seconds,
                                uint64_t *last_count);

/* ------------------------------------------------------------------------ */
/* Request loop with continuous batching (serving).                          */
/* ------------------------------------------------------------------------ */
typedef struct ka_serve_stage {
    int32_t pred;    /* ka_pred_kind; KA_PRED_ALL with KA_XFORM_HASH = hash map */
    uint32_t param;
    uint32_t xform;
} ka_serve_stage;

typedef struct ka_serve_request {
    double arrival_s;            /* offset from the start of the run               */
    uint64_t seed;               /* data: n entries of the seeded stream           */
    uint32_t n;
    uint32_t n_stages;           /* 1..4                                           */
    ka_serve_stage stages[4];
    uint32_t *h_out;             /* optional: final data copied here (value mode)  */
    uint64_t h_out_cap;
} ka_serve_request;

typedef struct ka_serve_result {
    double admit_s;              /* when the request was admitted                   */
    double done_s;               /* when its result was ready on the host           */
    uint32_t count;              /* final live length                               */
    ka_status status;
} ka_serve_result;

typedef struct ka_serve_options {
    uint32_t mode;               /* 0: continuous batching, each tick one CUDA graph launch;
                                    1: plain launches per request; 2: continuous
                                    batching with the tick's launches issued directly */
    uint32_t max_inflight;       /* admitted requests at most (0: 4096)              */
    uint64_t budget_bytes;       /* admission budget (0: the system's); the first
                                    min(budget, 4 GiB) are reserved in the run's
                                    memory pool before the loop starts           */
    double time_scale;           /* arrival_s multiplier (1.0 = real time)           */
    ka_tile tile;                /* batched kernel shape ({0,0}: autotuned/default)  */
    uint32_t flags;              /* KA_SERVE_* below (0: none)                       */
} ka_serve_options;
/* Modes 0 and 2 issue a tick that holds a single request as that request's
 * plain launch sequence (generate, one compaction per stage, count
 * publication), without the batch tables and plan kernels; this flag batches
 * such a tick like any other. */
#define KA_SERVE_BATCH_LONE 1u

typedef struct ka_serve_stats {
    double wall_s;
    uint64_t elements;           /* input elements of completed requests             */
    uint64_t launches;           /* kernel launches issued (graph nodes counted)     */
    uint64_t iterations;         /* batch iterations (mode 0)                        */
    uint64_t peak_bytes;         /* peak admitted bytes                              */
    uint32_t max_inflight_seen;
    uint32_t rejected;           /* requests larger than the whole budget            */
    uint64_t graph_launches;     /* ticks issued as one CUDA graph launch (mode 0)   */
    uint64_t lone_ticks;         /* ticks of one request issued as plain launches    */
    /* Host-side timing of the serving loop, to locate stalls: its longest step
     * (taking arrivals, polling completions, issuing work), the number of steps
     * longer than 1 ms, and the longest single admission allocation, buffer
     * release, issue (launches or graph launch) and completion poll. */
    double max_step_s;
    uint64_t slow_steps;
    double max_alloc_s, max_free_s, max_issue_s, max_poll_s;
} ka_serve_stats;

ka_status ka_serve_run(ka_system *sys, const ka_serve_request *reqs, uint32_t n_reqs,
                       const ka_serve_options *opt, ka_serve_result *results, ka_serve_stats *stats);

#ifdef __cplusplus
}
#endif
#endif /* KA_H */
