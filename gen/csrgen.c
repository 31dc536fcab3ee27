/*
 * Seeded synthetic input generation for CSR SpMM workloads.
 *
 * This file fills the bulk arrays of the synthetic workloads (column indices
 * of a CSR pattern, uniform values, normal dense matrices).  It holds none of
 * the arithmetic of the method being tested: it only draws random numbers.
 * Both the CPU oracle and the GPU library receive the arrays it writes.
 *
 * Randomness is counter based: every draw is a pure function of
 * (seed, stream, counter) through the SplitMix64 finaliser (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), so
 * the output does not depend on the number of OpenMP threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* draw number `ctr` of stream `stream` under `seed` */
static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t ctr) {
    return mix64(mix64(seed ^ mix64(stream)) + ctr);
}

/* uniform integer in [0, k) from the top 32 bits (Lemire multiply-shift; k < 2^31) */
static inline int32_t draw_below(uint64_t h, int32_t k) {
    return (int32_t)(((h >> 32) * (uint64_t)(uint32_t)k) >> 32);
}

/* uniform double in [0, 1) with 53 random bits */
static inline double draw_unit(uint64_t h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void sort_i32(int32_t *v, int64_t n) {
    if (n <= 32) {
        for (int64_t i = 1; i < n; ++i) {
            int32_t x = v[i];
            int64_t j = i - 1;
            while (j >= 0 && v[j] > x) { v[j + 1] = v[j]; --j; }
            v[j + 1] = x;
        }
    } else {
        qsort(v, (size_t)n, sizeof(int32_t), cmp_i32);
    }
}

/*
 * Fill col_ind[row_ptr[r] .. row_ptr[r+1]) of every row r with distinct
 * column indices drawn uniformly from [0, k), sorted ascending.
 * Returns 0, or -1 if some row is longer than k.
 */
int gen_fill_columns(int32_t m, int32_t k, const int64_t *row_ptr, uint64_t seed, int32_t *col_ind) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : bad)
    for (int64_t r = 0; r < m; ++r) {
        int64_t lo = row_ptr[r], len = row_ptr[r + 1] - row_ptr[r];
        if (len <= 0) continue;
        if (len > k) { bad |= 1; continue; }
        int32_t *out = col_ind + lo;
        if (len * 4 >= (int64_t)k) {
            /* selection sampling over [0, k): already sorted */
            int64_t chosen = 0;
            for (int64_t t = 0; t < k && chosen < len; ++t) {
                double u = draw_unit(draw(seed, (uint64_t)r, (uint64_t)t));
                if ((double)(k - t) * u < (double)(len - chosen)) out[chosen++] = (int32_t)t;
            }
        } else {
            uint64_t ctr = 0;
            for (int64_t i = 0; i < len; ++i) out[i] = draw_below(draw(seed, (uint64_t)r, ctr++), k);
            sort_i32(out, len);
            for (;;) { /* redraw duplicates until every index is distinct */
                int64_t dups = 0;
                for (int64_t i = 1; i < len; ++i)
                    if (out[i] == out[i - 1]) { out[i] = draw_below(draw(seed, (uint64_t)r, ctr++), k); ++dups; }
                if (!dups) break;
                sort_i32(out, len);
            }
        }
    }
    return bad ? -1 : 0;
}

/* out[i] = lo + (hi - lo) * U_i, U_i uniform in [0, 1) with 24 bits (exact in float32) */
void gen_fill_uniform_f32(int64_t count, uint64_t seed, uint64_t stream, float lo, float hi, float *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i) {
        float u = (float)(draw(seed, stream, (uint64_t)i) >> 40) * (1.0f / 16777216.0f);
        out[i] = lo + (hi - lo) * u;
    }
}

/* standard normal draws by the Box-Muller transform, two per counter value */
void gen_fill_normal_f32(int64_t count, uint64_t seed, uint64_t stream, float *out) {
    const double two_pi = 6.283185307179586476925286766559;
    int64_t pairs = (count + 1) / 2;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < pairs; ++i) {
        uint64_t h1 = draw(seed, stream, (uint64_t)(2 * i)), h2 = draw(seed, stream, (uint64_t)(2 * i + 1));
        double u1 = ((double)(h1 >> 11) + 1.0) * (1.0 / 9007199254740992.0); /* (0, 1] */
        double u2 = draw_unit(h2);
        double rad = sqrt(-2.0 * log(u1));
        out[2 * i] = (float)(rad * cos(two_pi * u2));
        if (2 * i + 1 < count) out[2 * i + 1] = (float)(rad * sin(two_pi * u2));
    }
}

int gen_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
