// Queries on a Pkd-tree (Sec. 5 "Queries" of the paper): k nearest neighbours
// by depth-first search (near child first, a subtree pruned when its subspace
// is strictly farther than the current k-th candidate) and range counting
// (a subtree whose subspace lies inside the box adds its stored size).
// Subspaces are not stored: each stack entry carries the box implied by the
// splitters above it, as the paper does instead of keeping bounding boxes.
// One thread per query; the stack holds at most height + 1 entries: in local
// memory (QSTACK entries) for trees of height below QSTACK - 2, which the
// sampling build and the alpha test keep every tree below for alpha <= 3/10;
// in a global scratch buffer, sized by the tree's height and processed a
// chunk of queries at a time, for deeper trees (long runs of one-sided
// updates with alpha near 1/2, where no interior node is ever rebuilt).
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "engine.hpp"
#include "tree_impl.hpp"

namespace pkd {

constexpr int QSTACK = 128;
constexpr int QTHREADS = 128;

template <int D>
struct Box {
  int32_t lo[D], hi[D];
};

template <int D>
__device__ __forceinline__ long long box_dist2(const int32_t* q, const Box<D>& b) {
  long long s = 0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    long long t = 0;
    if (q[j] < b.lo[j]) t = (long long)b.lo[j] - q[j];
    else if (q[j] > b.hi[j]) t = (long long)q[j] - b.hi[j];
    s += t * t;
  }
  return s;
}

struct QueryArgs {
  const Node* nodes;
  const uint8_t* ndim;
  Pts A;
  uint32_t root;
  const int32_t* q;
  const int32_t* hi;
  uint64_t nq;
  int k;
  uint32_t* out_ids;
  int64_t* out_d2;
  uint64_t* out_cnt;
  DevStatus* st;
  const int32_t* box;  // stored bounding boxes (node slot * 2d), or null
  // deep trees: stack entry i of query qi at [i * nq + qi] of these
  uint32_t* dv;
  void* db;      // Box<D> entries
  uint8_t* df;
  int dcap;      // entries per query (0: local stacks)
};

// The depth-first stack of one query: local arrays, or (DEEP) the query's
// column of the global scratch.
template <int D, bool DEEP>
struct QStack {
  uint32_t lv[DEEP ? 1 : QSTACK];
  Box<D> lb[DEEP ? 1 : QSTACK];
  uint8_t lf[DEEP ? 1 : QSTACK];
  uint32_t* gv;
  Box<D>* gb;
  uint8_t* gf;
  uint64_t stride, col;
  int cap;
  __device__ QStack(const QueryArgs& a, uint64_t qi) {
    if constexpr (DEEP) {
      gv = a.dv;
      gb = (Box<D>*)a.db;
      gf = a.df;
      stride = a.nq;
      col = qi;
      cap = a.dcap;
    } else {
      cap = QSTACK;
    }
  }
  __device__ __forceinline__ uint32_t& v(int i) {
    if constexpr (DEEP) return gv[(uint64_t)i * stride + col];
    else return lv[i];
  }
  __device__ __forceinline__ Box<D>& b(int i) {
    if constexpr (DEEP) return gb[(uint64_t)i * stride + col];
    else return lb[i];
  }
  __device__ __forceinline__ uint8_t& f(int i) {
    if constexpr (DEEP) return gf[(uint64_t)i * stride + col];
    else return lf[i];
  }
};

template <int D, int KMAX, bool DEEP>
__global__ void __launch_bounds__(QTHREADS) k_knn(QueryArgs a) {
  const uint64_t qi = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= a.nq) return;
  int32_t q[D];
#pragma unroll
  for (int j = 0; j < D; ++j) q[j] = a.q[qi * D + j];
  long long bd[KMAX];
  uint32_t bi[KMAX];
  const int k = a.k;
  for (int i = 0; i < KMAX; ++i) {
    bd[i] = LLONG_MAX;
    bi[i] = 0xFFFFFFFFu;
  }
  QStack<D, DEEP> S(a, qi);
  int sp = 0;
  S.v(0) = a.root;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    S.b(0).lo[j] = 0;
    S.b(0).hi[j] = PKD_COORD_LIMIT - 1;
  }
  sp = 1;
  while (sp > 0) {
    --sp;
    const uint32_t v = S.v(sp);
    const Box<D> b = S.b(sp);
    if (box_dist2<D>(q, b) > bd[k - 1]) continue;
    const uint8_t dm = a.ndim[v];
    const Node nd = a.nodes[v];
    if (dm == PKD_LEAF) {
      for (uint32_t i = 0; i < nd.size; ++i) {
        const uint64_t g = (uint64_t)nd.a + i;
        long long d2 = 0;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          long long t = (long long)a.A.c[(uint64_t)j * a.A.stride + g] - q[j];
          d2 += t * t;
        }
        const uint32_t id = a.A.id[g];
        if (d2 > bd[k - 1] || (d2 == bd[k - 1] && id >= bi[k - 1])) continue;
        int p = k - 1;
        while (p > 0 && (bd[p - 1] > d2 || (bd[p - 1] == d2 && bi[p - 1] > id))) {
          bd[p] = bd[p - 1];
          bi[p] = bi[p - 1];
          --p;
        }
        bd[p] = d2;
        bi[p] = id;
      }
      continue;
    }
    if (sp + 2 > S.cap) {
      set_error(a.st, DERR_STACK, 900);
      break;
    }
    const int j = dm;
    const int32_t x = nd.split;
    Box<D> L = b, R = b;
    L.hi[j] = min(L.hi[j], x - 1);
    R.lo[j] = max(R.lo[j], x);
    const bool near_left = q[j] < x;
    // far child first, so the near child is searched next
    S.v(sp) = near_left ? nd.b : nd.a;
    S.b(sp) = near_left ? R : L;
    ++sp;
    S.v(sp) = near_left ? nd.a : nd.b;
    S.b(sp) = near_left ? L : R;
    ++sp;
  }
  for (int i = 0; i < k; ++i) {
    a.out_d2[qi * k + i] = bd[i];
    a.out_ids[qi * k + i] = bi[i];
  }
}

template <int D, bool DEEP>
__global__ void __launch_bounds__(QTHREADS) k_range_count(QueryArgs a) {
  const uint64_t qi = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= a.nq) return;
  int32_t lo[D], hi[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    lo[j] = a.q[qi * D + j];
    hi[j] = a.hi[qi * D + j];
  }
  QStack<D, DEEP> S(a, qi);
  S.v(0) = a.root;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    S.b(0).lo[j] = 0;
    S.b(0).hi[j] = PKD_COORD_LIMIT - 1;
  }
  int sp = 1;
  unsigned long long cnt = 0;
  while (sp > 0) {
    --sp;
    const uint32_t v = S.v(sp);
    const Box<D> b = S.b(sp);
    bool disjoint = false, inside = true;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      disjoint |= (b.hi[j] < lo[j]) | (b.lo[j] > hi[j]) | (b.hi[j] < b.lo[j]);
      inside &= (b.lo[j] >= lo[j]) & (b.hi[j] <= hi[j]);
    }
    if (disjoint) continue;
    const Node nd = a.nodes[v];
    if (inside) {
      cnt += nd.size;
      continue;
    }
    const uint8_t dm = a.ndim[v];
    if (dm == PKD_LEAF) {
      for (uint32_t i = 0; i < nd.size; ++i) {
        const uint64_t g = (uint64_t)nd.a + i;
        bool in = true;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const int32_t x = a.A.c[(uint64_t)j * a.A.stride + g];
          in &= (x >= lo[j]) & (x <= hi[j]);
        }
        cnt += in;
      }
      continue;
    }
    if (sp + 2 > S.cap) {
      set_error(a.st, DERR_STACK, 901);
      break;
    }
    const int j = dm;
    Box<D> L = b, R = b;
    L.hi[j] = min(L.hi[j], nd.split - 1);
    R.lo[j] = max(R.lo[j], nd.split);
    S.v(sp) = nd.b;
    S.b(sp) = R;
    ++sp;
    S.v(sp) = nd.a;
    S.b(sp) = L;
    ++sp;
  }
  a.out_cnt[qi] = cnt;
}

// Range report: the same depth-first search as the range count; a subtree
// whose subspace lies inside the box is walked to its leaves without
// coordinate tests (its points need not be contiguous in the arena after
// updates).  Query qi writes its ids from out_ids[offsets[qi]].
template <int D, bool DEEP>
__global__ void __launch_bounds__(QTHREADS) k_range_report(QueryArgs a, const uint64_t* offsets, uint32_t* out_ids) {
  const uint64_t qi = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= a.nq) return;
  int32_t lo[D], hi[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    lo[j] = a.q[qi * D + j];
    hi[j] = a.hi[qi * D + j];
  }
  QStack<D, DEEP> S(a, qi);  // flag f: 1 when the subspace lies inside the box
  S.v(0) = a.root;
  S.f(0) = 0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    S.b(0).lo[j] = 0;
    S.b(0).hi[j] = PKD_COORD_LIMIT - 1;
  }
  int sp = 1;
  uint64_t pos = offsets[qi];
  const uint64_t end = offsets[qi + 1];
  while (sp > 0) {
    --sp;
    const uint32_t v = S.v(sp);
    bool inside = S.f(sp) != 0;
    const Box<D> b = S.b(sp);
    if (!inside) {
      bool disjoint = false;
      inside = true;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        disjoint |= (b.hi[j] < lo[j]) | (b.lo[j] > hi[j]) | (b.hi[j] < b.lo[j]);
        inside &= (b.lo[j] >= lo[j]) & (b.hi[j] <= hi[j]);
      }
      if (disjoint) continue;
    }
    const Node nd = a.nodes[v];
    const uint8_t dm = a.ndim[v];
    if (dm == PKD_LEAF) {
      for (uint32_t i = 0; i < nd.size; ++i) {
        const uint64_t g = (uint64_t)nd.a + i;
        bool in = true;
        if (!inside) {
#pragma unroll
          for (int j = 0; j < D; ++j) {
            const int32_t x = a.A.c[(uint64_t)j * a.A.stride + g];
            in &= (x >= lo[j]) & (x <= hi[j]);
          }
        }
        if (in) {
          if (pos >= end) {  // more points than counted: the tree changed
            set_error(a.st, DERR_STATE, 902);
            return;
          }
          out_ids[pos++] = a.A.id[g];
        }
      }
      continue;
    }
    if (sp + 2 > S.cap) {
      set_error(a.st, DERR_STACK, 903);
      return;
    }
    const int j = dm;
    Box<D> L = b, R = b;
    L.hi[j] = min(L.hi[j], nd.split - 1);
    R.lo[j] = max(R.lo[j], nd.split);
    S.v(sp) = nd.b;
    S.b(sp) = R;
    S.f(sp) = inside;
    ++sp;
    S.v(sp) = nd.a;
    S.b(sp) = L;
    S.f(sp) = inside;
    ++sp;
  }
}


// ---------------------------------------------------------------------------
// The same searches with stored bounding boxes (the Pkd-bb variant of Sec. 6):
// a node is pruned, counted whole or reported whole by the tight box of its
// points (a.box) instead of the subspace its ancestors' splitters imply, so
// a stack entry is a node slot only.  Answers are identical.
// ---------------------------------------------------------------------------

template <int D>
__device__ __forceinline__ Box<D> stored_box(const int32_t* box, uint32_t v) {
  Box<D> b;
  const int32_t* p = box + (uint64_t)v * 2 * D;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    b.lo[j] = p[j];
    b.hi[j] = p[D + j];
  }
  return b;
}

template <int D, int KMAX, bool DEEP>
__global__ void __launch_bounds__(QTHREADS) k_knn_bb(QueryArgs a) {
  const uint64_t qi = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= a.nq) return;
  int32_t q[D];
#pragma unroll
  for (int j = 0; j < D; ++j) q[j] = a.q[qi * D + j];
  long long bd[KMAX];
  uint32_t bi[KMAX];
  const int k = a.k;
  for (int i = 0; i < KMAX; ++i) {
    bd[i] = LLONG_MAX;
    bi[i] = 0xFFFFFFFFu;
  }
  QStack<D, DEEP> S(a, qi);
  S.v(0) = a.root;
  int sp = 1;
  while (sp > 0) {
    const uint32_t v = S.v(--sp);
    const Box<D> b = stored_box<D>(a.box, v);
    if (b.lo[0] > b.hi[0]) continue;  // an empty subtree
    if (box_dist2<D>(q, b) > bd[k - 1]) continue;
    const uint8_t dm = a.ndim[v];
    const Node nd = a.nodes[v];
    if (dm == PKD_LEAF) {
      for (uint32_t i = 0; i < nd.size; ++i) {
        const uint64_t g = (uint64_t)nd.a + i;
        long long d2 = 0;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          long long t = (long long)a.A.c[(uint64_t)j * a.A.stride + g] - q[j];
          d2 += t * t;
        }
        const uint32_t id = a.A.id[g];
        if (d2 > bd[k - 1] || (d2 == bd[k - 1] && id >= bi[k - 1])) continue;
        int p = k - 1;
        while (p > 0 && (bd[p - 1] > d2 || (bd[p - 1] == d2 && bi[p - 1] > id))) {
          bd[p] = bd[p - 1];
          bi[p] = bi[p - 1];
          --p;
        }
        bd[p] = d2;
        bi[p] = id;
      }
      continue;
    }
    if (sp + 2 > S.cap) {
      set_error(a.st, DERR_STACK, 904);
      break;
    }
    const bool near_left = q[dm] < nd.split;
    S.v(sp++) = near_left ? nd.b : nd.a;  // far child first, near child next
    S.v(sp++) = near_left ? nd.a : nd.b;
  }
  for (int i = 0; i < k; ++i) {
    a.out_d2[qi * k + i] = bd[i];
    a.out_ids[qi * k + i] = bi[i];
  }
}

// Range count (report = false) or report (true) with stored boxes.
template <int D, bool REPORT, bool DEEP>
__global__ void __launch_bounds__(QTHREADS) k_range_bb(QueryArgs a, const uint64_t* offsets, uint32_t* out_ids) {
  const uint64_t qi = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= a.nq) return;
  int32_t lo[D], hi[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    lo[j] = a.q[qi * D + j];
    hi[j] = a.hi[qi * D + j];
  }
  QStack<D, DEEP> S(a, qi);  // flag f: 1 inside the query box (report: walk without tests)
  S.v(0) = a.root;
  S.f(0) = 0;
  int sp = 1;
  unsigned long long cnt = 0;
  uint64_t pos = REPORT ? offsets[qi] : 0;
  const uint64_t end = REPORT ? offsets[qi + 1] : 0;
  while (sp > 0) {
    --sp;
    const uint32_t v = S.v(sp);
    bool inside = S.f(sp) != 0;
    if (!inside) {
      const Box<D> b = stored_box<D>(a.box, v);
      bool disjoint = false;
      inside = true;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        disjoint |= (b.hi[j] < lo[j]) | (b.lo[j] > hi[j]) | (b.hi[j] < b.lo[j]);
        inside &= (b.lo[j] >= lo[j]) & (b.hi[j] <= hi[j]);
      }
      if (disjoint) continue;
    }
    const Node nd = a.nodes[v];
    if (!REPORT && inside) {
      cnt += nd.size;
      continue;
    }
    const uint8_t dm = a.ndim[v];
    if (dm == PKD_LEAF) {
      for (uint32_t i = 0; i < nd.size; ++i) {
        const uint64_t g = (uint64_t)nd.a + i;
        bool in = true;
        if (!inside) {
#pragma unroll
          for (int j = 0; j < D; ++j) {
            const int32_t x = a.A.c[(uint64_t)j * a.A.stride + g];
            in &= (x >= lo[j]) & (x <= hi[j]);
          }
        }
        if (!in) continue;
        if constexpr (REPORT) {
          if (pos >= end) {  // more points than counted: the tree changed
            set_error(a.st, DERR_STATE, 905);
            return;
          }
          out_ids[pos++] = a.A.id[g];
        } else {
          ++cnt;
        }
      }
      continue;
    }
    if (sp + 2 > S.cap) {
      set_error(a.st, DERR_STACK, 906);
      return;
    }
    S.v(sp) = nd.b;
    S.f(sp) = inside;
    ++sp;
    S.v(sp) = nd.a;
    S.f(sp) = inside;
    ++sp;
  }
  if (!REPORT) a.out_cnt[qi] = cnt;
}

// Exclusive scan of q 64-bit counts into offsets[0..q] (offsets[q] = total):
// per-block sums, one block over the sums, then the blocks again.
constexpr int SCAN64_THREADS = 256, SCAN64_PER = 8, SCAN64_TILE = SCAN64_THREADS * SCAN64_PER;

__device__ __forceinline__ uint64_t block_scan64(uint64_t v, uint64_t* sh, uint64_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sh[w] = inc;
  __syncthreads();
  uint64_t before = 0, tot = 0;
  for (int k = 0; k < SCAN64_THREADS / 32; ++k) {
    if (k < w) before += sh[k];
    tot += sh[k];
  }
  __syncthreads();
  *total = tot;
  return before + inc - v;
}

__global__ void k_scan64_reduce(const uint64_t* in, uint64_t n, uint64_t* partial) {
  __shared__ uint64_t sh[SCAN64_THREADS / 32];
  const uint64_t base = (uint64_t)blockIdx.x * SCAN64_TILE + (uint64_t)threadIdx.x * SCAN64_PER;
  uint64_t s = 0;
  for (int k = 0; k < SCAN64_PER; ++k)
    if (base + k < n) s += in[base + k];
  uint64_t tot;
  block_scan64(s, sh, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void k_scan64_partials(uint64_t* partial, uint64_t nb) {
  __shared__ uint64_t sh[SCAN64_THREADS / 32];
  uint64_t carry = 0;
  for (uint64_t b0 = 0; b0 < nb; b0 += SCAN64_THREADS) {
    const uint64_t i = b0 + threadIdx.x;
    const uint64_t v = i < nb ? partial[i] : 0;
    uint64_t tot;
    const uint64_t ex = block_scan64(v, sh, &tot);
    if (i < nb) partial[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) partial[nb] = carry;
}

__global__ void k_scan64_apply(const uint64_t* in, uint64_t n, const uint64_t* partial, uint64_t* out) {
  __shared__ uint64_t sh[SCAN64_THREADS / 32];
  const uint64_t base = (uint64_t)blockIdx.x * SCAN64_TILE + (uint64_t)threadIdx.x * SCAN64_PER;
  uint64_t v[SCAN64_PER], s = 0;
  for (int k = 0; k < SCAN64_PER; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    s += v[k];
  }
  uint64_t tot;
  uint64_t run = partial[blockIdx.x] + block_scan64(s, sh, &tot);
  for (int k = 0; k < SCAN64_PER; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = partial[gridDim.x];
}

template <int D, bool DEEP>
static void launch_report_(const QueryArgs& a, const uint64_t* offsets, uint32_t* ids, cudaStream_t s) {
  const unsigned g = (unsigned)((a.nq + QTHREADS - 1) / QTHREADS);
  KTimer kt;
  ktimer_begin(kt, "range_report", a.nq, s);
  if (a.box) PKD_LAUNCH((k_range_bb<D, true, DEEP><<<g, QTHREADS, 0, s>>>(a, offsets, ids)));
  else PKD_LAUNCH((k_range_report<D, DEEP><<<g, QTHREADS, 0, s>>>(a, offsets, ids)));
  ktimer_end(kt);
}
template <int D>
static void launch_report(const QueryArgs& a, const uint64_t* offsets, uint32_t* ids, cudaStream_t s) {
  if (a.dcap) launch_report_<D, true>(a, offsets, ids, s);
  else launch_report_<D, false>(a, offsets, ids, s);
}

template <int D, bool DEEP>
static void launch_knn_(const QueryArgs& a, cudaStream_t s) {
  const unsigned g = (unsigned)((a.nq + QTHREADS - 1) / QTHREADS);
  KTimer kt;
  ktimer_begin(kt, "knn", a.nq, s);
  if (a.box) {
    if (a.k <= 16) PKD_LAUNCH((k_knn_bb<D, 16, DEEP><<<g, QTHREADS, 0, s>>>(a)));
    else PKD_LAUNCH((k_knn_bb<D, 128, DEEP><<<g, QTHREADS, 0, s>>>(a)));
  } else {
    if (a.k <= 16) PKD_LAUNCH((k_knn<D, 16, DEEP><<<g, QTHREADS, 0, s>>>(a)));
    else PKD_LAUNCH((k_knn<D, 128, DEEP><<<g, QTHREADS, 0, s>>>(a)));
  }
  ktimer_end(kt);
}
template <int D>
static void launch_knn(const QueryArgs& a, cudaStream_t s) {
  if (a.dcap) launch_knn_<D, true>(a, s);
  else launch_knn_<D, false>(a, s);
}

template <int D, bool DEEP>
static void launch_rc_(const QueryArgs& a, cudaStream_t s) {
  const unsigned g = (unsigned)((a.nq + QTHREADS - 1) / QTHREADS);
  KTimer kt;
  ktimer_begin(kt, "range_count", a.nq, s);
  if (a.box) PKD_LAUNCH((k_range_bb<D, false, DEEP><<<g, QTHREADS, 0, s>>>(a, nullptr, nullptr)));
  else PKD_LAUNCH((k_range_count<D, DEEP><<<g, QTHREADS, 0, s>>>(a)));
  ktimer_end(kt);
}
template <int D>
static void launch_rc(const QueryArgs& a, cudaStream_t s) {
  if (a.dcap) launch_rc_<D, true>(a, s);
  else launch_rc_<D, false>(a, s);
}

#define PKD_QDISPATCH(d, F, ...)      \
  switch (d) {                        \
    case 1: F<1>(__VA_ARGS__); break; \
    case 2: F<2>(__VA_ARGS__); break; \
    case 3: F<3>(__VA_ARGS__); break; \
    case 4: F<4>(__VA_ARGS__); break; \
    case 5: F<5>(__VA_ARGS__); break; \
    case 6: F<6>(__VA_ARGS__); break; \
    case 7: F<7>(__VA_ARGS__); break; \
    default: F<8>(__VA_ARGS__); break; \
  }

static int query_height_ok(const TreeMem& t) {
  // the depth-first stack holds at most height + 1 entries
  return t.st_host && t.st_host->max_depth + 2 < (uint32_t)QSTACK;
}

// Runs fn(args, first query) over the queries of `a`: one call with local
// stacks, or, for a tree too deep for them, chunks of queries whose stacks
// (height + 3 entries each) live in a global scratch buffer of at most
// DEEP_SCRATCH bytes.  The status must have been read (check_status).
constexpr uint64_t DEEP_SCRATCH = 1ull << 30;

template <class F>
static int for_query_chunks(const TreeMem& t, const QueryArgs& a, cudaStream_t s, F&& fn) {
  if (query_height_ok(t)) {
    fn(a, 0);
    return PKD_OK;
  }
  if (!t.st_host) return PKD_EINTERNAL;
  const int d = t.p.d;
  const uint64_t cap = (uint64_t)t.st_host->max_depth + 3;
  const uint64_t per = cap * (4 + 8 * (uint64_t)d + 1);
  const uint64_t chunk = std::max<uint64_t>(1, std::min<uint64_t>(a.nq, DEEP_SCRATCH / per));
  if (cap > (1u << 30)) return PKD_EINTERNAL;
  uint32_t* dv = nullptr;
  int32_t* db = nullptr;
  uint8_t* df = nullptr;
  int e = dalloc(&dv, chunk * cap, s);
  if (e == PKD_OK) e = dalloc(&db, chunk * cap * 2 * (uint64_t)d, s);
  if (e == PKD_OK) e = dalloc(&df, chunk * cap, s);
  if (e == PKD_OK) {
    for (uint64_t c0 = 0; c0 < a.nq; c0 += chunk) {
      QueryArgs ac = a;
      ac.nq = std::min<uint64_t>(chunk, a.nq - c0);
      ac.q = a.q + c0 * (uint64_t)d;
      if (a.hi) ac.hi = a.hi + c0 * (uint64_t)d;
      ac.dv = dv;
      ac.db = db;
      ac.df = df;
      ac.dcap = (int)cap;
      fn(ac, c0);
    }
  }
  dfree(dv, s);
  dfree(db, s);
  dfree(df, s);
  return e;
}

}  // namespace pkd

using namespace pkd;

extern "C" {

int pkd_knn(const pkd_tree* tc, const int32_t* queries, uint64_t q, int k, uint32_t* out_ids,
            int64_t* out_d2, void* stream) {
  if (!tc) return PKD_EINVAL;
  TreeMem& t = const_cast<TreeMem&>(tc->m);
  return knn_on(t, t.root, queries, q, k, out_ids, out_d2, (cudaStream_t)stream);
}

}  // extern "C"

int pkd::knn_on(TreeMem& t, uint32_t root, const int32_t* queries, uint64_t q, int k, uint32_t* out_ids,
                int64_t* out_d2, cudaStream_t s) {
  if (k < 1 || k > 128) return PKD_EINVAL;
  if (q == 0) return PKD_OK;
  if (!queries || !out_ids || !out_d2) return PKD_EINVAL;
  TreeTouch touch{&t, s};
  bool ok;
  PKD_TRY_(validate_coords(queries, q * (uint64_t)t.p.d, s, &ok));
  if (!ok) return PKD_EINVAL;
  PKD_TRY_(check_status(t, s));
  QueryArgs a{};
  a.nodes = t.nodes;
  a.ndim = t.ndim;
  a.A = t.A;
  a.root = root;
  a.q = queries;
  a.nq = q;
  a.k = k;
  a.out_ids = out_ids;
  a.out_d2 = out_d2;
  a.st = t.st;
  a.box = (t.bbox_on && root == t.root) ? t.bbox : nullptr;
  PKD_TRY_(for_query_chunks(t, a, s, [&](QueryArgs ac, uint64_t c0) {
    ac.out_ids = out_ids + c0 * (uint64_t)k;
    ac.out_d2 = out_d2 + c0 * (uint64_t)k;
    PKD_QDISPATCH(t.p.d, launch_knn, ac, s);
  }));
  PKD_CUDA(cudaGetLastError());
  return PKD_OK;
}

extern "C" {

int pkd_range_count(const pkd_tree* tc, const int32_t* lo, const int32_t* hi, uint64_t q,
                    uint64_t* out_counts, void* stream) {
  if (!tc) return PKD_EINVAL;
  if (q == 0) return PKD_OK;
  if (!lo || !hi || !out_counts) return PKD_EINVAL;
  TreeMem& t = const_cast<TreeMem&>(tc->m);
  cudaStream_t s = (cudaStream_t)stream;
  TreeTouch touch{&t, s};
  bool ok1, ok2;
  PKD_TRY_(validate_coords(lo, q * (uint64_t)t.p.d, s, &ok1));
  PKD_TRY_(validate_coords(hi, q * (uint64_t)t.p.d, s, &ok2));
  if (!ok1 || !ok2) return PKD_EINVAL;
  PKD_TRY_(check_status(t, s));
  QueryArgs a{};
  a.nodes = t.nodes;
  a.ndim = t.ndim;
  a.A = t.A;
  a.root = t.root;
  a.q = lo;
  a.hi = hi;
  a.nq = q;
  a.out_cnt = out_counts;
  a.st = t.st;
  a.box = t.bbox_on ? t.bbox : nullptr;
  PKD_TRY_(for_query_chunks(t, a, s, [&](QueryArgs ac, uint64_t c0) {
    ac.out_cnt = out_counts + c0;
    PKD_QDISPATCH(t.p.d, launch_rc, ac, s);
  }));
  PKD_CUDA(cudaGetLastError());
  return PKD_OK;
}

int pkd_range_report(const pkd_tree* tc, const int32_t* lo, const int32_t* hi, uint64_t q, uint64_t* offsets,
                     uint32_t* ids, uint64_t ids_cap, uint64_t* total, void* stream) {
  if (!tc || !total) return PKD_EINVAL;
  *total = 0;
  if (q == 0) return PKD_OK;
  if (!lo || !hi || !offsets) return PKD_EINVAL;
  TreeMem& t = const_cast<TreeMem&>(tc->m);
  cudaStream_t s = (cudaStream_t)stream;
  TreeTouch touch{&t, s};
  bool ok1, ok2;
  PKD_TRY_(validate_coords(lo, q * (uint64_t)t.p.d, s, &ok1));
  PKD_TRY_(validate_coords(hi, q * (uint64_t)t.p.d, s, &ok2));
  if (!ok1 || !ok2) return PKD_EINVAL;
  PKD_TRY_(check_status(t, s));
  // pass 1: counts (into offsets[0..q)), scanned in place into offsets[0..q]
  uint64_t* counts = nullptr;
  uint64_t* partial = nullptr;
  const uint64_t nb = (q + SCAN64_TILE - 1) / SCAN64_TILE;
  PKD_TRY_(dalloc(&counts, q, s));
  int e = dalloc(&partial, nb + 1, s);
  if (e) {
    dfree(counts, s);
    return e;
  }
  QueryArgs a{};
  a.nodes = t.nodes;
  a.ndim = t.ndim;
  a.A = t.A;
  a.root = t.root;
  a.q = lo;
  a.hi = hi;
  a.nq = q;
  a.out_cnt = counts;
  a.st = t.st;
  a.box = t.bbox_on ? t.bbox : nullptr;
  e = for_query_chunks(t, a, s, [&](QueryArgs ac, uint64_t c0) {
    ac.out_cnt = counts + c0;
    PKD_QDISPATCH(t.p.d, launch_rc, ac, s);
  });
  if (e) {
    dfree(counts, s);
    dfree(partial, s);
    return e;
  }
  PKD_LAUNCH(k_scan64_reduce<<<(unsigned)nb, SCAN64_THREADS, 0, s>>>(counts, q, partial));
  PKD_LAUNCH(k_scan64_partials<<<1, SCAN64_THREADS, 0, s>>>(partial, nb));
  PKD_LAUNCH(k_scan64_apply<<<(unsigned)nb, SCAN64_THREADS, 0, s>>>(counts, q, partial, offsets));
  dfree(counts, s);
  dfree(partial, s);
  uint64_t tot = 0;
  PKD_CUDA(cudaMemcpyAsync(&tot, offsets + q, 8, cudaMemcpyDeviceToHost, s));
  PKD_CUDA(cudaStreamSynchronize(s));
  *total = tot;
  if (tot > ids_cap || (tot > 0 && !ids)) return PKD_EINVAL;
  // pass 2: the ids
  PKD_TRY_(for_query_chunks(t, a, s, [&](QueryArgs ac, uint64_t c0) {
    PKD_QDISPATCH(t.p.d, launch_report, ac, offsets + c0, ids, s);
  }));
  PKD_CUDA(cudaGetLastError());
  return PKD_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// k-NN ids without any allocation (the paper has no counterpart)
// ----------------------------------------------------------------------------
// pkd_knn takes a status word from the library's memory pool for its
// coordinate check and needs a caller buffer for the distances.  Some callers
// can do neither: a server that has handed all spare device memory to its
// trees and may not let a pool grow while a request is in flight, or one that
// needs the latency of a query call free of allocator and mapping work.  This
// variant keeps both in a fixed scratch array compiled into the library:
//
//   bytes [0, 4)                          coordinate-check flag; must be zero
//                                         when the check kernel starts (each
//                                         call clears it on its stream first)
//   bytes [256, 256 + 8 * q * k)          the k distances of every query; no
//                                         initial value needed (written by
//                                         the search before anything reads it)
//
// The scratch is one array per device, shared by every call: two calls whose
// work overlaps on the device (different streams, or different host threads)
// race on it.  Calls issued one after the other on one stream are ordered.
// The first call on a device is the set-up: it resolves the array's address
// and launches every kernel the call uses once on an empty query set, which
// loads them and lets the driver size its local-memory reservation for the
// largest; make that call before any region in which the caller may not
// allocate.

namespace pkd {

static __device__ __align__(256) unsigned char g_knn_noalloc_scratch[256 + 8 * (uint64_t)PKD_NOALLOC_MAX_PAIRS];

__global__ void k_noalloc_check(const int32_t* c, uint64_t cnt, unsigned* bad) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  int b = 0;
  for (; i < cnt; i += stride) {
    const int32_t v = c[i];
    b |= (v < 0) | (v >= PKD_COORD_LIMIT);
  }
  if (__any_sync(0xffffffffu, b) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_noalloc_mu;
static unsigned char* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Every kernel this entry point can launch, run once on an empty query set:
// under lazy module loading a kernel's first launch loads it, and a kernel
// with more local memory per thread than any launched before makes the driver
// enlarge the device's local-memory reservation.  Both must happen in the
// set-up, not in a later call.
template <int D>
static void noalloc_warm(cudaStream_t s) {
  QueryArgs a{};
  a.nq = 0;
  a.k = 1;
  PKD_LAUNCH((k_knn<D, 16, false><<<1, QTHREADS, 0, s>>>(a)));
  PKD_LAUNCH((k_knn<D, 128, false><<<1, QTHREADS, 0, s>>>(a)));
}

// Set-up, once per device, with that device current: the scratch address,
// and every kernel of the call loaded with its local memory reserved.
static int noalloc_scratch(int dev, cudaStream_t s, unsigned char** out) {
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_knn_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      fprintf(stderr, "pkd_knn_ids_noalloc: scratch address on device %d: %s\n", dev,
              cudaGetErrorString(e));
      return e != cudaSuccess ? cuda_err(e) : PKD_ECUDA;
    }
    PKD_LAUNCH(k_noalloc_check<<<1, 256, 0, s>>>(nullptr, 0, nullptr));
    noalloc_warm<1>(s);
    noalloc_warm<2>(s);
    noalloc_warm<3>(s);
    noalloc_warm<4>(s);
    noalloc_warm<5>(s);
    noalloc_warm<6>(s);
    noalloc_warm<7>(s);
    noalloc_warm<8>(s);
    PKD_CUDA(cudaGetLastError());
    PKD_CUDA(cudaStreamSynchronize(s));
    g_noalloc_ptr[dev] = (unsigned char*)p;
  }
  *out = g_noalloc_ptr[dev];
  return PKD_OK;
}

template <int D>
static void launch_knn_noalloc(const QueryArgs& a, cudaStream_t s) {
  const unsigned g = (unsigned)((a.nq + QTHREADS - 1) / QTHREADS);
  if (a.k <= 16) PKD_LAUNCH((k_knn<D, 16, false><<<g, QTHREADS, 0, s>>>(a)));
  else PKD_LAUNCH((k_knn<D, 128, false><<<g, QTHREADS, 0, s>>>(a)));
}

}  // namespace pkd

extern "C" int pkd_knn_ids_noalloc(const pkd_tree* tc, const int32_t* queries, uint64_t q, int k,
                                   uint32_t* out_ids, void* stream) {
  if (!tc || k < 1 || k > 128) return PKD_EINVAL;
  if (q == 0) return PKD_OK;
  if (!queries || !out_ids) return PKD_EINVAL;
  if (q > (uint64_t)PKD_NOALLOC_MAX_PAIRS / (uint64_t)k) {
    fprintf(stderr,
            "pkd_knn_ids_noalloc: q*k = %llu exceeds the fixed scratch of %llu (query, neighbour) "
            "pairs; split the batch or use pkd_knn\n",
            (unsigned long long)q * (unsigned long long)k, (unsigned long long)PKD_NOALLOC_MAX_PAIRS);
    return PKD_EINVAL;
  }
  TreeMem& t = const_cast<TreeMem&>(tc->m);
  int dev = -1;
  PKD_CUDA(cudaGetDevice(&dev));
  if (dev != t.device || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return PKD_EINVAL;
  unsigned char* scratch = nullptr;
  PKD_TRY_(noalloc_scratch(dev, (cudaStream_t)stream, &scratch));
  cudaStream_t s = (cudaStream_t)stream;
  TreeTouch touch{&t, s, true};  // may not create an event
  unsigned* bad = (unsigned*)scratch;
  PKD_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned), s));
  PKD_LAUNCH(k_noalloc_check<<<152 * 8, 256, 0, s>>>(queries, q * (uint64_t)t.p.d, bad));
  unsigned h = 0;
  PKD_CUDA(cudaMemcpyAsync(&h, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  PKD_CUDA(cudaStreamSynchronize(s));
  if (h != 0) return PKD_EINVAL;
  PKD_TRY_(check_status(t, s));
  if (!query_height_ok(t)) return PKD_EINTERNAL;
  QueryArgs a{};
  a.nodes = t.nodes;
  a.ndim = t.ndim;
  a.A = t.A;
  a.root = t.root;
  a.q = queries;
  a.nq = q;
  a.k = k;
  a.out_ids = out_ids;
  a.out_d2 = (int64_t*)(scratch + 256);
  a.st = t.st;
  PKD_QDISPATCH(t.p.d, launch_knn_noalloc, a, s);
  PKD_CUDA(cudaGetLastError());
  return PKD_OK;
}
