// Shared definitions of the GB300 Pkd-tree kernels (sm_103a).
//
// Layouts in HBM:
//  - points: structure of arrays, coordinate j of point i at c[j*stride + i]
//    (int32, coalesced per dimension) and ids at id[i];
//  - nodes: 16-byte records {split, size, a, b} plus a byte of split
//    dimension per node (0xFF = leaf).  Interior: a/b = child slots.
//    Leaf: a = arena position of its first point, size = point count.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pkd.h"

#define PKD_DMAX 8
#define PKD_COORD_LIMIT (1 << 30)
#define PKD_LEAF 0xFF

namespace pkd {

struct Params {
  int d, phi, lambda, sigma_log2, sigma_os, count_mode, alpha_num, alpha_den;
  uint64_t seed;
};

struct __align__(16) Node {
  int32_t split;
  uint32_t size;
  uint32_t a;
  uint32_t b;
};

struct Pts {
  int32_t* c;
  uint32_t* id;
  uint64_t stride;
  __host__ __device__ int32_t* dim(int j) const { return c + (uint64_t)j * stride; }
};

// Where a subproblem's points currently live.
enum Where : uint32_t { IN_A = 0, IN_B = 1, IN_INPUT = 2 };

// A subproblem of a build: points [start, start+len) of the arena, rooted at
// node slot `root`, at tree depth `depth`.
struct Seg {
  uint64_t start;
  uint32_t len;
  uint32_t depth;
  uint32_t root;
  uint32_t where;
};

// Device-side status word shared by all kernels of one tree.
enum DevErr : int {
  DERR_NONE = 0,
  DERR_SLOT = 1,      // node slot allocator overran its range
  DERR_CAPACITY = 2,  // a bounded buffer overflowed
  DERR_STACK = 3,     // a task stack overflowed
  DERR_TIMEOUT = 4,   // a bounded wait ran out
  DERR_STATE = 5,     // an internal consistency check failed
};

struct DevStatus {
  int err;
  int detail;
  uint32_t max_depth;
  int idflags;  // id-table flags of the running call (IDF_* in ids.cuh)
  unsigned long long counters[8];
};

__device__ __forceinline__ void set_error(DevStatus* st, int code, int detail) {
  if (atomicCAS(&st->err, 0, code) == 0) st->detail = detail;
}

// True once any kernel of the tree has recorded an error.  Kernels that
// consume another kernel's counts or offsets (which a kernel that stopped
// early may have left unwritten) test it first and do nothing, so a
// failure never turns into reads or writes at garbage positions; the host
// then reports the recorded error.
__device__ __forceinline__ bool pkd_failed(const DevStatus* st) { return *(volatile const int*)&st->err != 0; }
// The same test with one answer for the whole block (thread 0 reads the
// status): the kernels that use it synchronise their threads, so all of
// them must leave together.  Call it first, from every thread.
__device__ __forceinline__ bool pkd_failed_block(const DevStatus* st) {
  return __syncthreads_or(threadIdx.x == 0 && pkd_failed(st)) != 0;
}

// Sampling hash (SplitMix64's 64-bit finaliser, Steele/Lea/Flood 2014, as a
// counter-based generator keyed by seed, depth and id).
constexpr uint64_t K_DEPTH = 0x9E3779B97F4A7C15ull;
constexpr uint64_t K_ID = 0xC2B2AE3D27D4EB4Full;

__host__ __device__ __forceinline__ uint64_t finalize64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Is point `id` in the sample of a subproblem at tree depth t, rate 2^-s?
__host__ __device__ __forceinline__ bool in_sample(uint64_t seed, uint32_t t, uint32_t id, int s) {
  if (s == 0) return true;
  uint64_t h = finalize64(seed ^ ((uint64_t)t * K_DEPTH) ^ ((uint64_t)id * K_ID));
  return (h >> (64 - s)) == 0;
}

// The same test with the per-subproblem part of the key precomputed:
// key = seed ^ t * K_DEPTH (identical results).
__host__ __device__ __forceinline__ uint64_t sample_key(uint64_t seed, uint32_t t) {
  return seed ^ ((uint64_t)t * K_DEPTH);
}
__host__ __device__ __forceinline__ bool in_sample_k(uint64_t key, uint32_t id, int s) {
  if (s == 0) return true;
  const uint64_t h = finalize64(key ^ ((uint64_t)id * K_ID));
  return (h >> (64 - s)) == 0;
}

// Sample-rate exponent for a subproblem of n points: fixed in rate mode; in
// count mode the largest s with 2^lambda * sigma_os * 2^s <= n (about
// 2^lambda * sigma_os samples, Alg. 1).
__host__ __device__ __forceinline__ int sample_shift(const Params& p, uint64_t n) {
  if (!p.count_mode) return p.sigma_log2;
  uint64_t target = ((uint64_t)1 << p.lambda) * (uint64_t)p.sigma_os;
  int s = 0;
  while (s < 40 && (target << (s + 1)) <= n) ++s;
  return s;
}

// Weight balance of Sec. 2: 0.5 - alpha <= L/N <= 0.5 + alpha, in integers.
__host__ __device__ __forceinline__ bool is_balanced(uint64_t L, uint64_t N, int num, int den) {
  uint64_t lhs = 2ull * (uint64_t)den * L;
  return lhs >= (uint64_t)(den - 2 * num) * N && lhs <= (uint64_t)(den + 2 * num) * N;
}

}  // namespace pkd
