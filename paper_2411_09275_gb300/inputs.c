/*
 * Seeded synthetic inputs for the Pkd-tree benchmarks and tests.
 *
 * This file holds no arithmetic of the kd-tree method itself: it only draws
 * points, query boxes and index samples.  Both the CPU oracle and the CUDA
 * path consume what it produces, so it is compiled on its own and imported by
 * neither of them.
 *
 * Random stream: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
 * output = the 64-bit finaliser of the state.  Integer-only, so the same seed
 * gives the same bytes on x86-64 and AArch64.
 *
 * Distributions (stand-ins for the paper's Uniform and Varden sets, Sec. 6
 * "Datasets"; the original Varden generator is not available here):
 *  - uniform: every coordinate = top 30 bits of one draw, i.e. uniform in
 *    [0, 2^30).
 *  - varden-like: one random walk.  Each step restarts at a uniform point with
 *    probability 1e-4; otherwise every coordinate moves by a uniform integer
 *    in [-L, L] where L is drawn log-uniformly in [1, 10^4] by octaves
 *    (octave k uniform in [0, 13], then L uniform in [2^k, 2^(k+1)), capped
 *    at 10^4), and is clamped to [0, 2^30 - 1].
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PKDIN_COORD_BITS 30
#define PKDIN_COORD_MAX ((int64_t)1 << PKDIN_COORD_BITS)

typedef struct { uint64_t s; } sm_stream;

static uint64_t sm_next(sm_stream* st) {
  uint64_t z = (st->s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Uniform integer in [0, bound) by the multiply-shift method (bound < 2^32). */
static uint64_t sm_below(sm_stream* st, uint64_t bound) {
  return ((sm_next(st) >> 32) * bound) >> 32;
}

/* First output of the stream for a seed: exported so a test can pin the
 * stream against SplitMix64's published vector. */
uint64_t pkdin_splitmix64_first(uint64_t seed) {
  sm_stream st = {seed};
  return sm_next(&st);
}

/* out[n][d] int32, each coordinate uniform in [0, 2^30). */
void pkdin_uniform(int32_t* out, uint64_t n, int d, uint64_t seed) {
  sm_stream st = {seed};
  for (uint64_t i = 0; i < n * (uint64_t)d; ++i)
    out[i] = (int32_t)(sm_next(&st) >> (64 - PKDIN_COORD_BITS));
}

/* out[n][d] int32, the varden-like random walk described above. */
void pkdin_varden(int32_t* out, uint64_t n, int d, uint64_t seed) {
  sm_stream st = {seed};
  const uint64_t restart_below = 1844674407370955ull; /* floor(2^64 / 10^4) */
  int64_t cur[16];
  for (int j = 0; j < d; ++j) cur[j] = (int64_t)(sm_next(&st) >> (64 - PKDIN_COORD_BITS));
  for (uint64_t i = 0; i < n; ++i) {
    if (i > 0) {
      if (sm_next(&st) < restart_below) {
        for (int j = 0; j < d; ++j) cur[j] = (int64_t)(sm_next(&st) >> (64 - PKDIN_COORD_BITS));
      } else {
        uint64_t k = sm_below(&st, 14);
        int64_t L = (int64_t)((1ull << k) + sm_below(&st, 1ull << k));
        if (L > 10000) L = 10000;
        for (int j = 0; j < d; ++j) {
          int64_t step = (int64_t)sm_below(&st, (uint64_t)(2 * L + 1)) - L;
          int64_t v = cur[j] + step;
          if (v < 0) v = 0;
          if (v > PKDIN_COORD_MAX - 1) v = PKDIN_COORD_MAX - 1;
          cur[j] = v;
        }
      }
    }
    for (int j = 0; j < d; ++j) out[i * (uint64_t)d + j] = (int32_t)cur[j];
  }
}

/* k distinct indices drawn from [0, n) by a partial Fisher-Yates shuffle
 * (k <= n < 2^32).  Returns 0, or -1 when scratch memory is unavailable. */
int pkdin_sample_indices(uint32_t* out, uint64_t k, uint64_t n, uint64_t seed) {
  if (k > n) return -1;
  uint32_t* a = (uint32_t*)malloc(n * sizeof(uint32_t));
  if (!a) return -1;
  for (uint64_t i = 0; i < n; ++i) a[i] = (uint32_t)i;
  sm_stream st = {seed};
  for (uint64_t i = 0; i < k; ++i) {
    uint64_t j = i + sm_below(&st, n - i);
    uint32_t t = a[i];
    a[i] = a[j];
    a[j] = t;
    out[i] = a[i];
  }
  free(a);
  return 0;
}

/* q closed query boxes lo[q][d] <= hi[q][d]: a uniform corner plus a uniform
 * side length in [0, max_side] per coordinate, clipped to the coordinate box. */
void pkdin_boxes(int32_t* lo, int32_t* hi, uint64_t q, int d, uint32_t max_side, uint64_t seed) {
  sm_stream st = {seed};
  for (uint64_t i = 0; i < q * (uint64_t)d; ++i) {
    int64_t a = (int64_t)(sm_next(&st) >> (64 - PKDIN_COORD_BITS));
    int64_t w = (int64_t)sm_below(&st, (uint64_t)max_side + 1);
    int64_t b = a + w;
    if (b > PKDIN_COORD_MAX - 1) b = PKDIN_COORD_MAX - 1;
    lo[i] = (int32_t)a;
    hi[i] = (int32_t)b;
  }
}
