// Escape-time Mandelbrot image: the paper's compute-bound workload for
// kernel actors (Sec. 5.4), here a plain CUDA kernel and an actor stage.
//
// Pixel (x, y) is c = (re_min + x dre, im_min + y dim); from z = 0 the step
// z <- z^2 + c is applied while |z|^2 <= 4, at most max_iter times, and the
// pixel holds the number of steps. Every operation is one round-to-nearest
// single-precision operation in a fixed order (__fmul_rn / __fadd_rn /
// __fsub_rn cannot be contracted into fused multiply-adds), so each count is
// reproducible bit for bit on any IEEE machine that does the same operations.
//
// The work is ALU-bound (eight single-precision adds and multiplies per
// step, no memory traffic to speak of) and, at four instructions issued per
// SM per clock, bound by issue: the paired f32x2 multiply and add carry two
// of the operations each, which frees issue slots. Consecutive threads take consecutive
// pixels of a row, whose orbits are alike, so a warp's lanes stay together.
// The step loop runs four steps per trip, each with its own escape test, so
// the counter and the step limit cost one update and one test per four steps
// (64 % of the FP32 issue ceiling at 16000 x 16000 and 100 steps, against
// 52 % one step per trip; eight per trip was slower). The paired operations
// took that to 66 % (69 % at 1000 steps).
#include "ka_internal.h"

namespace ka {
namespace {

constexpr int kMbBlock = 256;

// Pairs of single-precision values in one 64-bit register, and the paired
// round-to-nearest multiply and add of sm_100-class GPUs (one instruction for
// two IEEE operations, each rounded as __fmul_rn / __fadd_rn would).
__device__ __forceinline__ uint64_t pair(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpair(uint64_t v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t mul_rn2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t add_rn2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__global__ void __launch_bounds__(kMbBlock) k_mandelbrot(uint32_t *out, uint32_t width, uint64_t pixels, float re_min,
                                                          float im_min, float dre, float dim, uint32_t max_iter) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t p = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < pixels; p += stride) {
        const uint32_t y = uint32_t(p / width), x = uint32_t(p - uint64_t(y) * width);
        const float cr = __fadd_rn(re_min, __fmul_rn(float(x), dre));
        const float ci = __fadd_rn(im_min, __fmul_rn(float(y), dim));
        const uint64_t c = pair(cr, ci);
        uint64_t z = pair(0.0f, 0.0f);  // (zr, zi)
        uint32_t k = 0;
        // One step: false if z has escaped (|z|^2 > 4), else z <- z^2 + c.
        // (zr^2, zi^2) is one paired multiply and (zr^2 - zi^2, 2 zr zi) + c
        // one paired add: six instructions for the eight operations.
        auto step = [&]() -> bool {
            float rr, ii, zr, zi;
            unpair(mul_rn2(z, z), rr, ii);
            if (__fadd_rn(rr, ii) > 4.0f) return false;
            unpair(z, zr, zi);
            z = add_rn2(pair(__fsub_rn(rr, ii), __fmul_rn(__fmul_rn(2.0f, zr), zi)), c);
            return true;
        };
        // four steps per trip (one counter update and bound test for four)
        while (max_iter - k >= 4u) {  // (k <= max_iter throughout: no wrap-around)
            if (!step()) goto done;
            if (!step()) {
                k += 1u;
                goto done;
            }
            if (!step()) {
                k += 2u;
                goto done;
            }
            if (!step()) {
                k += 3u;
                goto done;
            }
            k += 4u;
        }
        while (k < max_iter && step()) k += 1u;
    done:
        out[p] = k;
    }
}

__global__ void k_set_word(uint32_t *w, uint32_t v) { *w = v; }

}  // namespace

ka_status launch_mandelbrot(uint32_t *out, uint32_t width, uint32_t height, float re_min, float im_min, float re_max,
                            float im_max, uint32_t max_iter, uint32_t *n_out, cudaStream_t stream) {
    const uint64_t pixels = uint64_t(width) * height;
    if (pixels > 0xFFFFFFFFull || (pixels && !out)) return KA_E_ARG;
    if (pixels) {
        // the same single-precision expressions as the definition
        const float dre = (re_max - re_min) / float(width);
        const float dim = (im_max - im_min) / float(height);
        uint64_t blocks = (pixels + kMbBlock - 1) / kMbBlock;
        const uint64_t cap = uint64_t(device_info().sm_count) * 16;
        if (blocks > cap) blocks = cap;
        k_mandelbrot<<<unsigned(blocks), kMbBlock, 0, stream>>>(out, width, pixels, re_min, im_min, dre, dim,
                                                                max_iter);
        const ka_status s = cuda_status(cudaGetLastError());
        if (s != KA_OK) return s;
    }
    if (n_out) {
        k_set_word<<<1, 1, 0, stream>>>(n_out, uint32_t(pixels));
        return cuda_status(cudaGetLastError());
    }
    return KA_OK;
}

}  // namespace ka

using namespace ka;

extern "C" ka_status ka_mandelbrot(uint32_t *d_out, uint32_t width, uint32_t height, float re_min, float im_min,
                                   float re_max, float im_max, uint32_t max_iter, void *stream) {
    return launch_mandelbrot(d_out, width, height, re_min, im_min, re_max, im_max, max_iter, nullptr,
                             static_cast<cudaStream_t>(stream));
}
