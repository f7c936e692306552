/*
 * Oracle (test infrastructure only; never linked into the product path):
 * the CPU reference results of the three job kinds written as plain C loops
 * with OpenMP over the host cores. This is the CPU baseline's form of the
 * definitions in kernels.py, with the same inputs and the same arithmetic:
 *
 *   triad  a[i] = b[i] + s * c[i] in FP32, the product rounded before the
 *          sum (the STREAM triad, no fused multiply-add);
 *   SpMV   y[r] = sum over the row's non-zeros of val * x[col], products and
 *          sums in fp64 on the FP32 inputs, in CSR order, plus the row's
 *          sum of |val * x[col]| (the scale of the error bound);
 *   GEMM   the bf16-rounded inputs as fp64 matrices; the product itself is
 *          left to a library matrix multiply by the caller.
 *
 * Inputs are regenerated from their published definition (SplitMix64,
 * Steele, Lea and Flood 2014; the uniform, Box-Muller, multiply-shift and
 * inverse-CDF maps documented in tracegen.py). Nothing here is shared with
 * the CUDA library.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static const uint64_t GAMMA = 0x9E3779B97F4A7C15ull;

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* output i (0-based) of the stream seeded with k */
static inline uint64_t sm64_at(uint64_t k, uint64_t i) { return mix64(k + (i + 1) * GAMMA); }

uint64_t omp_stream_key(uint64_t job_key, uint64_t stream) { return sm64_at(job_key, stream); }

/* element e of a uniform stream with key k, in [-1, 1): 24 bits of the hash
 * out(k, e / 2) -- bits 40..63 for an even e, bits 8..31 for an odd one --
 * scaled by 2^-23, minus one (exact) */
static inline float uniform_at(uint64_t k, uint64_t e) {
    const uint64_t h = sm64_at(k, e >> 1);
    const uint64_t b = (e & 1) ? ((h >> 8) & 0xFFFFFFull) : (h >> 40);
    return (float)((double)b * 0x1p-23 - 1.0);
}

/* Box-Muller: cos branch for an even element of a pair, sin for an odd one */
static inline float normal_of(uint64_t h, int odd) {
    double u1 = ((double)(h >> 40) + 1.0) * 0x1p-24;
    double u2 = (double)((h >> 16) & 0xFFFFFFull) * 0x1p-24;
    double r = sqrt(-2.0 * log(u1));
    double ang = 2.0 * M_PI * u2;
    return (float)(odd ? r * sin(ang) : r * cos(ang));
}

/* multiply-shift of the high (even element) or low (odd) 32 bits into [0, n) */
static inline uint64_t column_of(uint64_t h, int odd, uint64_t n) {
    uint64_t w = odd ? (h & 0xFFFFFFFFull) : (h >> 32);
    return (uint64_t)(((unsigned __int128)w * n) >> 32);
}

int omp_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* FP32 triad of a job with key `key` (streams b = 1, c = 2), n elements. */
void omp_triad(uint64_t key, uint64_t n, float s, float* a) {
    const uint64_t kb = sm64_at(key, 1), kc = sm64_at(key, 2);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; i++) {
        float b = uniform_at(kb, (uint64_t)i);
        float c = uniform_at(kc, (uint64_t)i);
        float p = s * c;          /* first rounding */
        a[i] = b + p;             /* second rounding */
    }
}

/* CSR SpMV of a job with key `key`: `rows` rows, row lengths by the 64-entry
 * inverse-CDF table (stream 1), columns (2) and values (3) in pairs, x (4).
 * y and mag receive rows fp64 values; ptr (rows + 1 int64) the row offsets.
 * Returns the number of non-zeros. */
int64_t omp_spmv(uint64_t key, uint64_t rows, const uint64_t* table, double* y, double* mag, int64_t* ptr) {
    const uint64_t kl = sm64_at(key, 1), kc = sm64_at(key, 2), kv = sm64_at(key, 3), kx = sm64_at(key, 4);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < (int64_t)rows; r++) {
        uint64_t u = sm64_at(kl, (uint64_t)r) >> 32;
        int64_t len = 0;
        while (len < 64 && table[len] <= u) len++;
        ptr[r + 1] = len;
    }
    ptr[0] = 0;
    for (uint64_t r = 0; r < rows; r++) ptr[r + 1] += ptr[r];
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t r = 0; r < (int64_t)rows; r++) {
        double acc = 0.0, am = 0.0;
        for (int64_t e = ptr[r]; e < ptr[r + 1]; e++) {
            const int odd = (int)(e & 1);
            const uint64_t m = (uint64_t)e >> 1;
            const uint64_t col = column_of(sm64_at(kc, m), odd, rows);
            const double v = (double)normal_of(sm64_at(kv, m), odd);
            const double x = (double)uniform_at(kx, col);
            acc += v * x;
            am += fabs(v * x);
        }
        y[r] = acc;
        mag[r] = am;
    }
    return ptr[rows];
}

/* rows x k matrix of a GEMM operand (stream 1 = A, index i*k + j; stream
 * 2 = B^T) as fp64 values of the bf16-rounded (nearest, ties to even)
 * uniforms. Element e of a bf16 stream: 16 bits of the hash out(k, e / 4),
 * bits 16 (e mod 4) and up, scaled by 2^-15, minus one (exact). */
void omp_gemm_operand(uint64_t key, uint64_t stream, uint64_t rows, uint64_t k, double* out) {
    const uint64_t ks = sm64_at(key, stream);
    const int64_t count = (int64_t)(rows * k);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; i++) {
        const uint64_t h = sm64_at(ks, (uint64_t)i >> 2);
        const uint64_t b16 = (h >> (16 * ((uint64_t)i & 3))) & 0xFFFFull;
        float f = (float)((double)b16 * 0x1p-15 - 1.0);
        uint32_t b;
        memcpy(&b, &f, 4);
        b += 0x7FFFu + ((b >> 16) & 1u);
        b &= 0xFFFF0000u;
        float r;
        memcpy(&r, &b, 4);
        out[i] = (double)r;
    }
}
