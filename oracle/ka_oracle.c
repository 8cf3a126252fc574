/*
 * CPU oracle for order-preserving stream compaction and its pipeline stages.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library calls, links or
 * includes this file; only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg use it. It shares no source, header, table or
 * constant with the CUDA path.
 *
 * Every function is the plain sequential definition of what the paper's
 * kernels compute, written for a reader to check by eye:
 *
 *  - stream compaction (Sec. 4.1): remove from an array every entry that fails
 *    a test and keep the rest in their original order; the result is never
 *    longer than the input. The paper's instance removes entries equal to a
 *    given value (zero); the general form keeps entries for which a predicate
 *    holds. Order is kept (the Billeter et al. method the paper uses, and the
 *    bitmap index it feeds, both keep positions).
 *  - the three phases of that method (Sec. 4.1, Listing 5): flag each entry,
 *    exclusive prefix sum of the flags, move each kept entry to its offset.
 *    The new length travels back in a configuration word (Sec. 4.1).
 *  - the interleave step of fuseFillsLiterals (Sec. 4.1): chunk ids and
 *    literals, k each, merged into one 2k index before the zeros are removed.
 *  - a hash map stage h = x * 2654435761 mod 2^32 and the seeded input stream
 *    (SplitMix64, Steele, Lea & Flood 2014), which the paper leaves open.
 */
#include <stdint.h>
#include <stddef.h>

/* Predicate ids of the oracle (its own numbering). */
enum {
    ORA_AND_MASK_EQ0 = 0, /* keep (x & param) == 0          */
    ORA_LT = 1,           /* keep x < param                 */
    ORA_TOPBITS_LT = 2,   /* keep (x >> 28) < param         */
    ORA_POPC_ODD = 3,     /* keep popcount(x) odd           */
    ORA_MOD_NE0 = 4,      /* keep x mod param != 0          */
    ORA_NE = 5,           /* keep x != param (remove value) */
    ORA_ALL = 6           /* keep every entry (a map stage)  */
};

/* SplitMix64: the (i+1)-th output of the sequential generator whose 64-bit
 * state starts at `seed` (state advances by the golden-ratio increment, then
 * the output is passed through the two xor-shift-multiply rounds). */
uint64_t ora_splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Seeded uint32 input: x_i = high 32 bits of splitmix64(seed, i). */
void ora_generate(uint64_t seed, uint64_t n, uint32_t *out)
{
    for (uint64_t i = 0; i < n; i++)
        out[i] = (uint32_t)(ora_splitmix64(seed, i) >> 32);
}

static int ora_popcount(uint32_t x)
{
    int c = 0;
    for (int b = 0; b < 32; b++)
        c += (int)((x >> b) & 1u);
    return c;
}

/* P(x): 1 if x is kept, 0 if it is removed; -1 for an unknown predicate or a
 * zero modulus. */
int ora_keep(int kind, uint32_t param, uint32_t x)
{
    switch (kind) {
    case ORA_AND_MASK_EQ0: return (x & param) == 0u;
    case ORA_LT:           return x < param;
    case ORA_TOPBITS_LT:   return (x >> 28) < param;
    case ORA_POPC_ODD:     return ora_popcount(x) % 2 == 1;
    case ORA_MOD_NE0:      return param == 0u ? -1 : (x % param) != 0u;
    case ORA_NE:           return x != param;
    case ORA_ALL:          return 1;
    default:               return -1;
    }
}

/* Phase 1 (flag map): f[i] = P(x[i]). Returns 0, or -1 on a bad predicate. */
int ora_predicate_map(const uint32_t *x, uint64_t n, int kind, uint32_t param, uint32_t *f)
{
    for (uint64_t i = 0; i < n; i++) {
        int k = ora_keep(kind, param, x[i]);
        if (k < 0)
            return -1;
        f[i] = (uint32_t)k;
    }
    return 0;
}

/* Phase 2 (prefix sum): o[0] = 0, o[i+1] = o[i] + v[i], all mod 2^32.
 * Returns the total (o[n-1] + v[n-1], or 0 for n = 0). */
uint32_t ora_exclusive_scan(const uint32_t *v, uint64_t n, uint32_t *o)
{
    uint32_t running = 0;
    for (uint64_t i = 0; i < n; i++) {
        o[i] = running;
        running += v[i];
    }
    return running;
}

/* Phase 3 (move): y[o[i]] = x[i] for every flagged i. */
void ora_scatter(const uint32_t *x, const uint32_t *f, const uint32_t *o, uint64_t n, uint32_t *y)
{
    for (uint64_t i = 0; i < n; i++)
        if (f[i])
            y[o[i]] = x[i];
}

/* Stream compaction by definition: walk the input once, append every kept
 * entry. Returns the new length k; y[0..k) is defined, y[k..) is untouched.
 * Returns UINT64_MAX on a bad predicate. */
uint64_t ora_compact(const uint32_t *x, uint64_t n, int kind, uint32_t param, uint32_t *y)
{
    uint64_t k = 0;
    for (uint64_t i = 0; i < n; i++) {
        int keep = ora_keep(kind, param, x[i]);
        if (keep < 0)
            return UINT64_MAX;
        if (keep) {
            y[k] = x[i];
            k++;
        }
    }
    return k;
}

/* Hash map stage: h[i] = x[i] * 2654435761 mod 2^32. */
void ora_map_hash(const uint32_t *x, uint64_t n, uint32_t *h)
{
    for (uint64_t i = 0; i < n; i++)
        h[i] = (uint32_t)((uint64_t)x[i] * 2654435761ULL);
}

/* Interleave of fuseFillsLiterals: index[2i] = chunk_ids[i],
 * index[2i+1] = literals[i], for i < k. */
void ora_prepare_index(const uint32_t *chunk_ids, const uint32_t *literals, uint64_t k, uint32_t *index)
{
    for (uint64_t i = 0; i < k; i++) {
        index[2 * i] = chunk_ids[i];
        index[2 * i + 1] = literals[i];
    }
}

/*
 * Escape-time Mandelbrot image (the paper's compute workload, Sec. 5.4):
 * pixel (x, y) of a width x height image over the rectangle with lower-left
 * corner (re_min, im_min) is the point c = (re_min + x dre, im_min + y dim),
 * dre = (re_max - re_min) / width, dim = (im_max - im_min) / height. Starting
 * from z = 0, z <- z^2 + c is applied while |z|^2 <= 4, at most max_iter
 * times; the pixel's value is the number of steps taken. Every operation is
 * one IEEE single-precision operation in the order written (this file is
 * built without floating-point contraction), so the result is exact and
 * reproducible: z^2 + c is (zr zr - zi zi + cr, (2 zr) zi + ci) and |z|^2 is
 * zr zr + zi zi. Row y = 0 is the bottom row of the rectangle; out is row-major.
 */
void ora_mandelbrot(uint32_t width, uint32_t height, float re_min, float im_min, float re_max, float im_max,
                    uint32_t max_iter, uint32_t *out)
{
    const float dre = (re_max - re_min) / (float)width;
    const float dim = (im_max - im_min) / (float)height;
    for (uint32_t y = 0; y < height; y++) {
        for (uint32_t x = 0; x < width; x++) {
            const float cr = re_min + (float)x * dre;
            const float ci = im_min + (float)y * dim;
            float zr = 0.0f, zi = 0.0f;
            uint32_t k = 0;
            while (k < max_iter) {
                const float rr = zr * zr;
                const float ii = zi * zi;
                if (rr + ii > 4.0f) break;
                const float nr = rr - ii + cr;
                const float ni = (2.0f * zr) * zi + ci;
                zr = nr;
                zi = ni;
                k++;
            }
            out[(uint64_t)y * width + x] = k;
        }
    }
}
