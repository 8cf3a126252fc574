// Tile-shape selection: explicit shape, else the autotuned winner for the
// kernel and size bucket, else a default chosen so that a launch has several
// tiles per SM. The autotuner times every supported (block, items-per-thread)
// shape of a kernel with CUDA events on the caller's stream and keeps the
// fastest, in memory and in a small JSON file.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ka_internal.h"

namespace ka {

namespace {
std::mutex g_mu;
std::map<std::pair<int, int>, std::pair<ka_tile, float>> g_table;
std::atomic<uint32_t> g_table_gen{1};  // advanced (under g_mu) with every change of g_table

int bucket_of(uint64_t n) {
    int b = 0;
    while ((1ull << b) < n && b < 40) ++b;
    return b;
}

const ka_tile kShapes[] = {
#define KA_SHAPE(B, I) {B, I},
    KA_FOR_EACH_SHAPE(KA_SHAPE)
#undef KA_SHAPE
};

// The TMA kernels (compaction, scan, batch) also have the shape (768, 16).
const ka_tile kTmaOnlyShapes[] = {{768, 16}};
// The batch kernel also has (704, 16), its default.
const ka_tile kBatchOnlyShapes[] = {{704, 16}};

ka_tile default_tile(int32_t kernel, uint64_t n) {
    if (kernel == KA_KERNEL_COMPACT && n >= (1ull << 22)) return ka_tile{768, 16};  // TMA kernel
    if (kernel == KA_KERNEL_BATCH) return ka_tile{704, 16};                         // TMA batch kernel
    if (kernel == KA_KERNEL_SCAN && n >= (1ull << 22)) return ka_tile{512, 16};      // TMA kernel, scan mode
    if (n >= (1ull << 24)) return ka_tile{256, 16};
    if (n >= (1ull << 21)) return ka_tile{256, 8};
    return ka_tile{256, 4};
}

bool save_table(const char *path) {
    FILE *f = std::fopen(path, "w");
    if (!f) return false;
    std::fprintf(f, "{\"entries\": [\n");
    bool first = true;
    for (const auto &kv : g_table) {
        std::fprintf(f, "%s  {\"kernel\": %d, \"bucket\": %d, \"block\": %u, \"ipt\": %u, \"us\": %.3f}",
                     first ? "" : ",\n", kv.first.first, kv.first.second, kv.second.first.block,
                     kv.second.first.ipt, kv.second.second);
        first = false;
    }
    std::fprintf(f, "\n]}\n");
    std::fclose(f);
    return true;
}

// Reads the objects written by save_table: one {...} per entry with the five
// keys above, in any order.
bool load_table(const char *path) {
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    std::fclose(f);
    auto field = [](const std::string &obj, const char *key, double *out) {
        const std::string k = std::string("\"") + key + "\"";
        const size_t p = obj.find(k);
        if (p == std::string::npos) return false;
        const size_t c = obj.find(':', p + k.size());
        if (c == std::string::npos) return false;
        *out = std::strtod(obj.c_str() + c + 1, nullptr);
        return true;
    };
    size_t pos = text.find('[');
    if (pos == std::string::npos) return false;
    for (;;) {
        const size_t o = text.find('{', pos);
        if (o == std::string::npos) break;
        const size_t e = text.find('}', o);
        if (e == std::string::npos) break;
        const std::string obj = text.substr(o, e - o + 1);
        double kernel, bucket, block, ipt, us = 0;
        if (field(obj, "kernel", &kernel) && field(obj, "bucket", &bucket) && field(obj, "block", &block) &&
            field(obj, "ipt", &ipt)) {
            field(obj, "us", &us);
            const ka_tile t{uint32_t(block), uint32_t(ipt)};
            if (tile_supported_for(int32_t(kernel), t.block, t.ipt)) {
                g_table[{int(kernel), int(bucket)}] = {t, float(us)};
                g_table_gen.fetch_add(1, std::memory_order_release);
            }
        }
        pos = e + 1;
    }
    return true;
}
}  // namespace

ka_tile resolve_tile(int32_t kernel, uint64_t n, const ka_tile *requested) {
    if (requested && requested->block && requested->ipt) return *requested;
    // The last answers of this thread, valid while the table is unchanged: a
    // pipeline stage asks the same question at every request.
    struct Memo {
        uint32_t gen;
        int32_t kernel;
        uint64_t n;
        ka_tile tile;
    };
    thread_local Memo memo[4] = {};
    thread_local uint32_t memo_next = 0;
    const uint32_t gen = g_table_gen.load(std::memory_order_acquire);
    for (const Memo &m : memo)
        if (m.gen == gen && m.kernel == kernel && m.n == n) return m.tile;
    ka_tile t = default_tile(kernel, n);
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_table.find({kernel, bucket_of(n)});
        if (it != g_table.end()) t = it->second.first;
    }
    // The TMA kernels take at most 2^32 - 4 entries (their tiles start on a
    // 16-byte boundary); above that, a shape the register kernels also have.
    if (kernel != KA_KERNEL_BATCH && !tile_supported(t.block, t.ipt) && n > 0xFFFFFFFCull) t = ka_tile{512, 16};
    memo[memo_next++ & 3u] = Memo{gen, kernel, n, t};  // (tagged with the generation read before the lookup)
    return t;
}

// Times `launch` over `reps` runs after `warm` untimed runs; returns the median
// per-launch microseconds, or a negative value on failure.
template <class F>
static float time_launches(F launch, cudaStream_t st, int warm, int reps) {
    for (int i = 0; i < warm; ++i)
        if (launch() != KA_OK) return -1.f;
    std::vector<float> t;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int i = 0; i < reps; ++i) {
        cudaEventRecord(e0, st);
        if (launch() != KA_OK) {
            t.clear();
            break;
        }
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        t.push_back(ms * 1000.f);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (t.empty()) return -1.f;
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

// Batch shape search: a synthetic batch (sizes log-uniform in 2^8..2^20 from
// a fixed SplitMix64 stream, each instance 16-byte aligned, keep x < 2^31),
// every shape timed on it; the winner is stored under the bucket that
// ka_compact_batch looks up.
ka_status autotune_batch(uint64_t total, const char *cache_path, ka_tile *best, float *best_us, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<uint32_t> sizes;
    uint64_t sum = 0, z = 0x5EEDull;
    while (sum < total && sizes.size() < 4096) {
        z += 0x9E3779B97F4A7C15ull;
        uint64_t m = z;
        m = (m ^ (m >> 30)) * 0xBF58476D1CE4E5B9ull;
        m = (m ^ (m >> 27)) * 0x94D049BB133111EBull;
        m ^= m >> 31;
        const double u = double(m >> 11) * (1.0 / 9007199254740992.0);
        uint32_t sz = uint32_t(std::pow(2.0, 8.0 + 12.0 * u));
        sz = std::min<uint64_t>(sz, total - sum);
        sizes.push_back(sz);
        sum += sz;
    }
    const uint32_t m = uint32_t(sizes.size());
    std::vector<uint64_t> off(m + 1, 0);
    for (uint32_t i = 0; i < m; ++i) off[i + 1] = off[i] + (uint64_t(sizes[i]) + 3) / 4 * 4;
    uint32_t *in = nullptr, *out = nullptr, *count = nullptr;
    ka_batch_item *d_items = nullptr;
    void *ws = nullptr;
    uint64_t ws_bytes = 0;
    ka_status s = ka_batch_workspace_size(m, off[m], nullptr, &ws_bytes);  // sized for the smallest tile
    if (s == KA_OK &&
        (cudaMalloc(&in, off[m] * 4 + 16) != cudaSuccess || cudaMalloc(&out, off[m] * 4 + 16) != cudaSuccess ||
         cudaMalloc(&count, size_t(m) * 4) != cudaSuccess ||
         cudaMalloc(&d_items, sizeof(ka_batch_item) * m) != cudaSuccess || cudaMalloc(&ws, ws_bytes) != cudaSuccess))
        s = KA_E_OOM;
    std::vector<ka_batch_item> items(m);
    for (uint32_t i = 0; i < m; ++i)
        items[i] = ka_batch_item{in + off[i], out + off[i], nullptr, count + i, sizes[i], KA_PRED_LT, 0x80000000u,
                                 KA_XFORM_NONE};
    if (s == KA_OK) s = launch_generate(in, off[m], 0xA5A5ull + total, nullptr, st);
    if (s == KA_OK)
        s = cuda_status(cudaMemcpyAsync(d_items, items.data(), sizeof(ka_batch_item) * m, cudaMemcpyHostToDevice, st));
    if (s == KA_OK) s = ka_workspace_init(ws, ws_bytes, st);
    ka_tile win{0, 0};
    float win_us = 1e30f;
    if (s == KA_OK) {
        std::vector<ka_tile> shapes(std::begin(kShapes), std::end(kShapes));
        shapes.insert(shapes.end(), std::begin(kTmaOnlyShapes), std::end(kTmaOnlyShapes));
        shapes.insert(shapes.end(), std::begin(kBatchOnlyShapes), std::end(kBatchOnlyShapes));
        for (const ka_tile &t : shapes) {
            auto launch = [&]() -> ka_status { return ka_compact_batch(d_items, m, m, ws, ws_bytes, &t, 0, st); };
            const float us = time_launches(launch, st, 2, 9);
            if (us > 0 && us < win_us) {
                win_us = us;
                win = t;
            }
        }
        if (win.block == 0) {  // no shape ran
            const cudaError_t e = cudaGetLastError();
            s = cuda_status(e != cudaSuccess ? e : cudaErrorUnknown);
        }
    }
    cudaStreamSynchronize(st);
    if (in) cudaFree(in);
    if (out) cudaFree(out);
    if (count) cudaFree(count);
    if (d_items) cudaFree(d_items);
    if (ws) cudaFree(ws);
    if (s != KA_OK) return s;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        g_table[{KA_KERNEL_BATCH, bucket_of(kBatchTileKey)}] = {win, win_us};
        g_table_gen.fetch_add(1, std::memory_order_release);
        if (cache_path) save_table(cache_path);
    }
    if (best) *best = win;
    if (best_us) *best_us = win_us;
    return KA_OK;
}

}  // namespace ka

using namespace ka;

extern "C" {

ka_status ka_tile_for(int32_t kernel, uint64_t n, ka_tile *tile) {
    if (!tile) return KA_E_ARG;
    *tile = resolve_tile(kernel, n, nullptr);
    return KA_OK;
}

ka_status ka_autotune_load(const char *cache_path) {
    if (!cache_path) return KA_E_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    return load_table(cache_path) ? KA_OK : KA_E_ARG;
}

ka_status ka_autotune(int32_t kernel, uint64_t n, const char *cache_path, ka_tile *best, float *best_us,
                      void *stream) {
    if (n == 0 || n > 0xFFFFFFFFull) return KA_E_ARG;
    if (kernel == KA_KERNEL_BATCH) return autotune_batch(n, cache_path, best, best_us, stream);
    if (kernel != KA_KERNEL_COMPACT && kernel != KA_KERNEL_SCAN) return KA_E_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t *in = nullptr, *out = nullptr, *count = nullptr;
    void *ws = nullptr;
    uint64_t ws_bytes = workspace_bytes_for_tiles(tiles_for(n, 512) + 1);
    ka_status s = KA_OK;
    if (cudaMalloc(&in, n * 4) != cudaSuccess || cudaMalloc(&out, n * 4) != cudaSuccess ||
        cudaMalloc(&count, 256) != cudaSuccess || cudaMalloc(&ws, ws_bytes) != cudaSuccess) {
        s = KA_E_OOM;
    }
    if (s == KA_OK) s = launch_generate(in, n, 0xA5A5ull + n, nullptr, st);
    if (s == KA_OK) s = ka_workspace_init(ws, ws_bytes, st);
    PredDev half;
    make_pred(KA_PRED_LT, 0x80000000u, &half);
    ka_tile win{0, 0};
    float win_us = 1e30f;
    std::vector<ka_tile> shapes(std::begin(kShapes), std::end(kShapes));
    shapes.insert(shapes.end(), std::begin(kTmaOnlyShapes), std::end(kTmaOnlyShapes));
    if (s == KA_OK) {
        for (const ka_tile &t : shapes) {
            auto launch = [&]() -> ka_status {
                if (kernel == KA_KERNEL_COMPACT) {
                    CompactLaunch L{in, out, nullptr, count, n, half, 1u, ws, ws_bytes, t};
                    return launch_compact(L, st);
                }
                return launch_exclusive_scan(in, n, nullptr, out, count, ws, ws_bytes, t, st);
            };
            const float us = time_launches(launch, st, 3, 15);
            if (us > 0 && us < win_us) {
                win_us = us;
                win = t;
            }
        }
        if (win.block == 0) {  // no shape ran
            const cudaError_t e = cudaGetLastError();
            s = cuda_status(e != cudaSuccess ? e : cudaErrorUnknown);
        }
    }
    cudaStreamSynchronize(st);
    if (in) cudaFree(in);
    if (out) cudaFree(out);
    if (count) cudaFree(count);
    if (ws) cudaFree(ws);
    if (s != KA_OK) return s;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        g_table[{kernel, bucket_of(n)}] = {win, win_us};
        g_table_gen.fetch_add(1, std::memory_order_release);
        if (cache_path) save_table(cache_path);
    }
    if (best) *best = win;
    if (best_us) *best_us = win_us;
    return KA_OK;
}

}  // extern "C"
