// Id table of a Pkd-tree: the coordinates of every stored point, keyed by
// its id.  BatchDelete names points by id and Sec. 4.2 sieves points, so the
// table turns each id into the coordinates to sieve; BatchInsert uses it to
// reject ids that are stored already or repeated within the batch.
//
// Open addressing with linear probing over `cap` slots (a power of two >= 32):
//   key[s]  64-bit word: the id in bits 0..31, the point's first coordinate
//           in bits 32..61 (coordinates are below 2^30) and its state in
//           bits 62..63 (ID_LIVE, or ID_DEAD = deleted); all ones = empty
//           (id 0xFFFFFFFF is never a point's id).  A key only ever goes
//           from empty to an id, so probe sequences never break; a deleted id
//           stays as DEAD and a later insert of the same id revives that
//           slot.  One compare-and-swap of this word changes a state.
//   xs[s]   the point's other coordinates, cw int32 words per slot (cw = the
//           smallest power of two >= d - 1, 0 for d = 1), so a lookup reads
//           two sectors at most.
// Home slot: the id's chunk of 32 consecutive values, c = id >> 5, goes to
// chunk (c ^ (c >> k)) * 0x9E3779B1 mod 2^k (k = log2(cap / 32)) and keeps
// its low five bits inside it.  The multiplier is odd, so distinct chunks of
// ids below cap never collide: dense ids fill consecutive slots and a warp's
// 32 consecutive ids are one coalesced run, while the fold and the
// multiplication spread sparse labels over the table.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pkd {

constexpr unsigned long long ID_EMPTY = ~0ull;
constexpr uint32_t ID_LIVE = 0, ID_DEAD = 1;
constexpr uint32_t ID_RESERVED = 0xFFFFFFFFu;  // k-NN padding; never a point's id
constexpr uint64_t ID_NO_SLOT = ~0ull;

// Flag bits the table kernels raise (DevStatus::idflags).
constexpr int IDF_BAD_ID = 1;  // a repeated, stored or reserved id in a claim
constexpr int IDF_FULL = 2;    // a probe went round the whole table

struct IdTable {
  unsigned long long* key = nullptr;
  int32_t* xs = nullptr;
  uint64_t cap = 0;   // slots
  int lgc = 0;        // log2(cap / 32)
  int cw = 0;         // words of xs per slot (coordinates 1..d-1)
  uint64_t used = 0;  // host: upper bound on slots whose key is set
  uint64_t live = 0;  // host: live ids
};

__host__ __device__ __forceinline__ uint64_t id_home(uint32_t id, int lgc) {
  const uint32_t c = id >> 5;
  const uint32_t f = lgc > 0 ? (c ^ (c >> lgc)) : 0u;
  const uint64_t chunk = (uint64_t)(f * 0x9E3779B1u) & ((1ull << lgc) - 1ull);
  return (chunk << 5) | (id & 31u);
}

__host__ __device__ __forceinline__ unsigned long long id_key(uint32_t id, int32_t x0, uint32_t state) {
  return ((unsigned long long)state << 62) | ((unsigned long long)(uint32_t)x0 << 32) | id;
}
__host__ __device__ __forceinline__ uint32_t id_state(unsigned long long k) { return (uint32_t)(k >> 62); }
__host__ __device__ __forceinline__ int32_t id_x0(unsigned long long k) {
  return (int32_t)((k >> 32) & 0x3FFFFFFFull);
}
__host__ __device__ __forceinline__ unsigned long long id_with_state(unsigned long long k, uint32_t state) {
  return (k & ~(3ull << 62)) | ((unsigned long long)state << 62);
}

}  // namespace pkd
