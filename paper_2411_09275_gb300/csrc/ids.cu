// Id table kernels and their host side (layout and hashing in ids.cuh).
//
//  claim    build and insert: every point takes the slot of its id (an
//           empty slot, or its own DEAD slot), stores its coordinates and
//           becomes LIVE; an id found LIVE (stored, or taken by another point
//           of the same batch) raises IDF_BAD_ID.  A rejected batch gives its
//           claimed slots back as DEAD (unclaim), so the stored set is
//           unchanged.  A build with ids 0..n-1 stores its keys without
//           compare-and-swap: the table is empty and those ids have distinct
//           home slots.
//  take     delete: every id found LIVE becomes DEAD (one winner per id, so
//           repeats count once), and its coordinates and id are appended to
//           the batch buffer that the delete sieves; unknown and DEAD ids are
//           skipped (round 1 of Sec. 4.2 discards points that are not in the
//           tree).  When the delete fails, restore puts the taken ids back.
//  rehash   the LIVE entries move to a larger table (DEAD ones are dropped).
#include <algorithm>
#include <cstdio>

#include "sieve.cuh"
#include "tree_impl.hpp"

namespace pkd {

namespace {

constexpr int ID_THREADS = 256;

unsigned id_blocks(uint64_t n) {
  const uint64_t b = (n + ID_THREADS - 1) / ID_THREADS;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, 152ull * 16));
}

__global__ void __launch_bounds__(ID_THREADS) k_ids_claim(const int32_t* coords, const uint32_t* ids, uint64_t m,
                                                          int d, IdTable T, uint64_t* slots, DevStatus* st) {
  const uint64_t mask = T.cap - 1;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    const int32_t* c = coords + i * (uint64_t)d;
    const int32_t x0 = c[0];
    uint64_t got = ID_NO_SLOT;
    int bad = 0;
    if (!ids) {  // ids 0..m-1 into an empty table: distinct home slots
      got = id_home((uint32_t)i, T.lgc);
      T.key[got] = id_key((uint32_t)i, x0, ID_LIVE);
    } else {
      const uint32_t id = ids[i];
      const unsigned long long want = id_key(id, x0, ID_LIVE);
      if (id == ID_RESERVED) {
        bad = IDF_BAD_ID;
      } else {
        uint64_t s = id_home(id, T.lgc), n = 0;
        for (; n < T.cap; ++n, s = (s + 1) & mask) {
          unsigned long long k = __ldcg(&T.key[s]);
          if (k == ID_EMPTY) {
            k = atomicCAS(&T.key[s], ID_EMPTY, want);
            if (k == ID_EMPTY) {
              got = s;
              break;
            }
          }
          if ((uint32_t)k == id) {  // this id's slot: revive it if deleted
            if (id_state(k) == ID_DEAD && atomicCAS(&T.key[s], k, want) == k)
              got = s;
            else
              bad = IDF_BAD_ID;
            break;
          }
        }
        if (n == T.cap) bad = IDF_FULL;
      }
    }
    if (got != ID_NO_SLOT) {
      int32_t* x = T.xs + got * (uint64_t)T.cw;
      for (int j = 1; j < d; ++j) x[j - 1] = c[j];
    }
    if (slots) slots[i] = got;
    if (bad) atomicOr(&st->idflags, bad);
  }
}

__global__ void __launch_bounds__(ID_THREADS) k_ids_restate(const uint64_t* slots, uint64_t m, IdTable T,
                                                            uint32_t state) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t s = slots[i];
    if (s != ID_NO_SLOT) T.key[s] = id_with_state(T.key[s], state);
  }
}

// One thread per id; the winners of a block reserve their batch positions
// with one atomic (block_reserve), so the append does not serialise.
__global__ void __launch_bounds__(ID_THREADS) k_ids_take(const uint32_t* ids, uint64_t m, IdTable T, Pts W,
                                                         uint64_t* wslots, uint32_t* count, int d, DevStatus* st) {
  const uint64_t mask = T.cap - 1;
  for (uint64_t b0 = (uint64_t)blockIdx.x * blockDim.x; b0 < m; b0 += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = b0 + threadIdx.x;
    uint64_t got = ID_NO_SLOT;
    uint32_t id = ID_RESERVED;
    int32_t x0 = 0;
    if (i < m) {
      id = ids[i];
      if (id != ID_RESERVED) {
        uint64_t s = id_home(id, T.lgc), n = 0;
        for (; n < T.cap; ++n, s = (s + 1) & mask) {
          const unsigned long long k = __ldcg(&T.key[s]);
          if (k == ID_EMPTY) break;  // never stored
          if ((uint32_t)k == id) {
            if (id_state(k) == ID_LIVE && atomicCAS(&T.key[s], k, id_with_state(k, ID_DEAD)) == k) {
              got = s;
              x0 = id_x0(k);
            }
            break;
          }
        }
        if (n == T.cap) atomicOr(&st->idflags, IDF_FULL);
      }
    }
    const uint32_t c[1] = {got != ID_NO_SLOT ? 1u : 0u};
    uint32_t* const ctr[1] = {count};
    uint32_t first[1];
    block_reserve<1>(c, ctr, first);
    if (got != ID_NO_SLOT) {
      const uint64_t p = first[0];
      const int32_t* x = T.xs + got * (uint64_t)T.cw;
      W.c[p] = x0;
      for (int j = 1; j < d; ++j) W.c[(uint64_t)j * W.stride + p] = x[j - 1];
      W.id[p] = id;
      wslots[p] = got;
    }
  }
}

__global__ void __launch_bounds__(ID_THREADS) k_ids_rehash(IdTable A, IdTable B, int d, DevStatus* st) {
  const uint64_t mask = B.cap - 1;
  for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A.cap; a += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = A.key[a];
    if (k == ID_EMPTY || id_state(k) != ID_LIVE) continue;
    const uint32_t id = (uint32_t)k;
    uint64_t s = id_home(id, B.lgc), n = 0;
    for (; n < B.cap; ++n, s = (s + 1) & mask)
      if (atomicCAS(&B.key[s], ID_EMPTY, k) == ID_EMPTY) break;
    if (n == B.cap) {
      atomicOr(&st->idflags, IDF_FULL);
      continue;
    }
    for (int j = 1; j < d; ++j) B.xs[s * (uint64_t)B.cw + j - 1] = A.xs[a * (uint64_t)A.cw + j - 1];
  }
}

// Slots for n ids at a load of at most 3/4 after a quarter more arrive.
uint64_t ids_cap_for(uint64_t n) {
  const uint64_t want = std::max<uint64_t>(64, (n + n / 4) / 3 * 4 + 4);
  uint64_t c = 32;
  while (c < want) c <<= 1;
  return c;
}

int ids_alloc(IdTable& T, int d, uint64_t cap, cudaStream_t s) {
  T = IdTable{};
  if (cap > (1ull << 32)) return PKD_ENOMEM;
  T.cap = cap;
  T.lgc = 0;
  while ((32ull << T.lgc) < cap) ++T.lgc;
  T.cw = 0;
  if (d > 1) {
    T.cw = 1;
    while (T.cw < d - 1) T.cw <<= 1;
  }
  cudaError_t e = big_alloc((void**)&T.key, (size_t)cap * 8, s);
  if (e == cudaSuccess && T.cw) e = big_alloc((void**)&T.xs, (size_t)cap * T.cw * 4, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ids_release(T, s);
    return e == cudaErrorMemoryAllocation ? PKD_ENOMEM : PKD_ECUDA;
  }
  PKD_CUDA(cudaMemsetAsync(T.key, 0xFF, (size_t)cap * 8, s));
  return PKD_OK;
}

}  // namespace

void ids_release(IdTable& T, cudaStream_t s) {
  big_free(T.key, s);
  big_free(T.xs, s);
  T = IdTable{};
}

int ids_create(TreeMem& t, uint64_t n, cudaStream_t s) { return ids_alloc(t.ids, t.p.d, ids_cap_for(n), s); }

int ids_reserve(TreeMem& t, uint64_t extra, cudaStream_t s) {
  IdTable& T = t.ids;
  if (T.used + extra <= T.cap / 4 * 3) return PKD_OK;
  IdTable B;
  PKD_TRY(ids_alloc(B, t.p.d, ids_cap_for(T.live + extra), s));
  PKD_LAUNCH(k_ids_rehash<<<id_blocks(T.cap), ID_THREADS, 0, s>>>(T, B, t.p.d, t.st));
  int fl = 0;
  int e = read_idflags(t, s, &fl);
  if (e == PKD_OK && fl) e = PKD_EINTERNAL;
  if (e != PKD_OK) {
    ids_release(B, s);
    return e;
  }
  B.live = T.live;
  B.used = T.live;
  ids_release(T, s);
  T = B;
  return PKD_OK;
}

int read_idflags(TreeMem& t, cudaStream_t s, int* flags) {
  PKD_CUDA(cudaMemcpyAsync(t.st_host, t.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  PKD_CUDA(cudaStreamSynchronize(s));
  *flags = t.st_host->idflags;
  if (*flags) PKD_CUDA(cudaMemsetAsync(&t.st->idflags, 0, sizeof(int), s));
  return PKD_OK;
}

void ids_claim(TreeMem& t, const int32_t* coords, const uint32_t* ids, uint64_t m, uint64_t* slots,
               cudaStream_t s) {
  if (m == 0) return;
  PKD_LAUNCH(k_ids_claim<<<id_blocks(m), ID_THREADS, 0, s>>>(coords, ids, m, t.p.d, t.ids, slots, t.st));
}

void ids_unclaim(TreeMem& t, const uint64_t* slots, uint64_t m, cudaStream_t s) {
  if (m == 0) return;
  PKD_LAUNCH(k_ids_restate<<<id_blocks(m), ID_THREADS, 0, s>>>(slots, m, t.ids, ID_DEAD));
}

void ids_take(TreeMem& t, const uint32_t* ids, uint64_t m, Pts W, uint64_t* wslots, uint32_t* count,
              cudaStream_t s) {
  if (m == 0) return;
  PKD_LAUNCH(k_ids_take<<<id_blocks(m), ID_THREADS, 0, s>>>(ids, m, t.ids, W, wslots, count, t.p.d, t.st));
}

void ids_restore(TreeMem& t, const uint64_t* wslots, uint64_t n, cudaStream_t s) {
  if (n == 0) return;
  PKD_LAUNCH(k_ids_restate<<<id_blocks(n), ID_THREADS, 0, s>>>(wslots, n, t.ids, ID_LIVE));
}

}  // namespace pkd
