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

// CLAIM_PER ids per thread: their first probe loads, then their
// compare-and-swaps, are all issued before any is waited for (random
// accesses into a table far larger than L2).  The dense build path (ids
// 0..m-1 into an empty table) stores its keys directly.
constexpr int CLAIM_PER = 4;

__device__ __forceinline__ void claim_store(const int32_t* coords, uint64_t i, int d, const IdTable& T, uint64_t got,
                                            uint64_t* slots) {
  if (got != ID_NO_SLOT) {
    const int32_t* c = coords + i * (uint64_t)d;
    int32_t* x = T.xs + got * (uint64_t)T.cw;
    for (int j = 1; j < d; ++j) x[j - 1] = c[j];
  }
  if (slots) slots[i] = got;
}

__global__ void __launch_bounds__(ID_THREADS) k_ids_claim(const int32_t* coords, const uint32_t* ids, uint64_t m,
                                                          int d, IdTable T, uint64_t* slots, DevStatus* st) {
  const uint64_t mask = T.cap - 1;
  if (!ids) {  // ids 0..m-1 into an empty table: distinct home slots
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
      const uint64_t got = id_home((uint32_t)i, T.lgc);
      T.key[got] = id_key((uint32_t)i, coords[i * (uint64_t)d], ID_LIVE);
      claim_store(coords, i, d, T, got, slots);
    }
    return;
  }
  const uint64_t span = (uint64_t)ID_THREADS * CLAIM_PER;
  for (uint64_t b0 = (uint64_t)blockIdx.x * span; b0 < m; b0 += (uint64_t)gridDim.x * span) {
    uint32_t id[CLAIM_PER];
    int32_t x0[CLAIM_PER];
    uint64_t s[CLAIM_PER];
    unsigned long long k[CLAIM_PER];
#pragma unroll
    for (int u = 0; u < CLAIM_PER; ++u) {
      const uint64_t i = b0 + (uint64_t)u * ID_THREADS + threadIdx.x;
      id[u] = i < m ? ids[i] : ID_RESERVED;
      x0[u] = i < m ? coords[i * (uint64_t)d] : 0;
    }
    int bad = 0;
#pragma unroll
    for (int u = 0; u < CLAIM_PER; ++u) {
      const uint64_t i = b0 + (uint64_t)u * ID_THREADS + threadIdx.x;
      if (i < m && id[u] == ID_RESERVED) bad |= IDF_BAD_ID;
      s[u] = id[u] != ID_RESERVED ? id_home(id[u], T.lgc) : 0;
      k[u] = id[u] != ID_RESERVED ? __ldcg(&T.key[s[u]]) : 0ull;
    }
    uint64_t got[CLAIM_PER];
#pragma unroll
    for (int u = 0; u < CLAIM_PER; ++u) {
      got[u] = ID_NO_SLOT;
      if (id[u] == ID_RESERVED) continue;
      const unsigned long long want = id_key(id[u], x0[u], ID_LIVE);
      uint64_t n = 0;
      for (; n < T.cap; ++n) {
        if (k[u] == ID_EMPTY) {
          k[u] = atomicCAS(&T.key[s[u]], ID_EMPTY, want);
          if (k[u] == ID_EMPTY) {
            got[u] = s[u];
            break;
          }
        }
        if ((uint32_t)k[u] == id[u]) {  // this id's slot: revive it if deleted
          if (id_state(k[u]) == ID_DEAD && atomicCAS(&T.key[s[u]], k[u], want) == k[u])
            got[u] = s[u];
          else
            bad |= IDF_BAD_ID;
          break;
        }
        s[u] = (s[u] + 1) & mask;
        k[u] = __ldcg(&T.key[s[u]]);
      }
      if (n == T.cap) bad |= IDF_FULL;
    }
#pragma unroll
    for (int u = 0; u < CLAIM_PER; ++u) {
      const uint64_t i = b0 + (uint64_t)u * ID_THREADS + threadIdx.x;
      if (i < m) claim_store(coords, i, d, T, got[u], slots);
    }
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

// TAKE_PER ids per thread: every probe's first load, then every
// compare-and-swap, then every coordinate load of the thread is issued before
// any of them is waited for (the lookups are random accesses into a table far
// larger than L2, so the time is the chains' latency); the winners of a block
// then reserve their batch positions with one atomic (block_reserve), so the
// append does not serialise.  The batch order is immaterial (the delete
// treats it as a set).
constexpr int TAKE_PER = 4;

__global__ void __launch_bounds__(ID_THREADS) k_ids_take(const uint32_t* ids, uint64_t m, IdTable T, Pts W,
                                                         uint64_t* wslots, uint32_t* count, int d, DevStatus* st) {
  const uint64_t mask = T.cap - 1;
  const uint64_t span = (uint64_t)ID_THREADS * TAKE_PER;
  for (uint64_t b0 = (uint64_t)blockIdx.x * span; b0 < m; b0 += (uint64_t)gridDim.x * span) {
    uint32_t id[TAKE_PER];
    uint64_t s[TAKE_PER];
    unsigned long long k[TAKE_PER];
#pragma unroll
    for (int u = 0; u < TAKE_PER; ++u) {
      const uint64_t i = b0 + (uint64_t)u * ID_THREADS + threadIdx.x;
      id[u] = i < m ? ids[i] : ID_RESERVED;
    }
#pragma unroll
    for (int u = 0; u < TAKE_PER; ++u) {
      s[u] = id[u] != ID_RESERVED ? id_home(id[u], T.lgc) : 0;
      k[u] = id[u] != ID_RESERVED ? __ldcg(&T.key[s[u]]) : ID_EMPTY;
    }
    // the rest of each probe (rarely more than the first slot)
    uint64_t got[TAKE_PER];
    int32_t x0[TAKE_PER];
#pragma unroll
    for (int u = 0; u < TAKE_PER; ++u) {
      got[u] = ID_NO_SLOT;
      x0[u] = 0;
      if (id[u] == ID_RESERVED) continue;
      uint64_t n = 0;
      while (k[u] != ID_EMPTY && (uint32_t)k[u] != id[u] && n + 1 < T.cap) {
        s[u] = (s[u] + 1) & mask;
        ++n;
        k[u] = __ldcg(&T.key[s[u]]);
      }
      if (k[u] != ID_EMPTY && (uint32_t)k[u] != id[u]) atomicOr(&st->idflags, IDF_FULL);
      if ((uint32_t)k[u] != id[u] || k[u] == ID_EMPTY || id_state(k[u]) != ID_LIVE) k[u] = ID_EMPTY;  // not taken
    }
#pragma unroll
    for (int u = 0; u < TAKE_PER; ++u)
      if (k[u] != ID_EMPTY && atomicCAS(&T.key[s[u]], k[u], id_with_state(k[u], ID_DEAD)) == k[u]) {
        got[u] = s[u];
        x0[u] = id_x0(k[u]);
      }
    int32_t xr[TAKE_PER][3];
#pragma unroll
    for (int u = 0; u < TAKE_PER; ++u)
      if (got[u] != ID_NO_SLOT) {
        const int32_t* x = T.xs + got[u] * (uint64_t)T.cw;
#pragma unroll
        for (int j = 1; j < 4; ++j)
          if (j < d) xr[u][j - 1] = x[j - 1];
      }
    uint32_t nwin = 0;
#pragma unroll
    for (int u = 0; u < TAKE_PER; ++u) nwin += got[u] != ID_NO_SLOT;
    const uint32_t c[1] = {nwin};
    uint32_t* const ctr[1] = {count};
    uint32_t first[1];
    block_reserve<1>(c, ctr, first);
    uint64_t p = first[0];
#pragma unroll
    for (int u = 0; u < TAKE_PER; ++u) {
      if (got[u] == ID_NO_SLOT) continue;
      W.c[p] = x0[u];
      if (d <= 4) {
#pragma unroll
        for (int j = 1; j < 4; ++j)
          if (j < d) W.c[(uint64_t)j * W.stride + p] = xr[u][j - 1];
      } else {
        const int32_t* x = T.xs + got[u] * (uint64_t)T.cw;
        for (int j = 1; j < d; ++j) W.c[(uint64_t)j * W.stride + p] = x[j - 1];
      }
      W.id[p] = id[u];
      wslots[p] = got[u];
      ++p;
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
  PKD_TRY(dev_fill(T.key, 0xFF, (size_t)cap * 8, s));
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
  if (*flags) PKD_TRY(dev_fill(&t.st->idflags, 0, sizeof(int), s));
  return PKD_OK;
}

void ids_claim(TreeMem& t, const int32_t* coords, const uint32_t* ids, uint64_t m, uint64_t* slots,
               cudaStream_t s) {
  if (m == 0) return;
  const uint64_t per = ids ? CLAIM_PER : 1;
  // timed for inserts only: a build's fill runs beside its base cases on a
  // second stream, so its span is not the kernel's own time
  KTimer kt;
  if (slots) ktimer_begin(kt, "id_claim", m, s);
  PKD_LAUNCH(k_ids_claim<<<id_blocks((m + per - 1) / per), ID_THREADS, 0, s>>>(coords, ids, m, t.p.d, t.ids, slots,
                                                                              t.st));
  ktimer_end(kt);
}

void ids_unclaim(TreeMem& t, const uint64_t* slots, uint64_t m, cudaStream_t s) {
  if (m == 0) return;
  PKD_LAUNCH(k_ids_restate<<<id_blocks(m), ID_THREADS, 0, s>>>(slots, m, t.ids, ID_DEAD));
}

void ids_take(TreeMem& t, const uint32_t* ids, uint64_t m, Pts W, uint64_t* wslots, uint32_t* count,
              cudaStream_t s) {
  if (m == 0) return;
  KTimer kt;
  ktimer_begin(kt, "id_take", m, s);
  PKD_LAUNCH(k_ids_take<<<id_blocks((m + TAKE_PER - 1) / TAKE_PER), ID_THREADS, 0, s>>>(ids, m, t.ids, W, wslots,
                                                                                       count, t.p.d, t.st));
  ktimer_end(kt);
}

void ids_restore(TreeMem& t, const uint64_t* wslots, uint64_t n, cudaStream_t s) {
  if (n == 0) return;
  PKD_LAUNCH(k_ids_restate<<<id_blocks(n), ID_THREADS, 0, s>>>(wslots, n, t.ids, ID_LIVE));
}

}  // namespace pkd
