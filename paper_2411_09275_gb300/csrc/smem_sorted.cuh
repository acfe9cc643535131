// Base case of Alg. 1 on presorted lists: one CTA finishes a subproblem of
// up to `cap` points in shared memory.
//
// The CTA first sorts the points once along every dimension (a stable LSD
// radix sort of 16-bit point indices, 8-bit digits over the bits in which
// that dimension's coordinates differ).  A node is then a position range
// [lo, hi) that holds, in each of the d lists, exactly its own points sorted
// along that list's dimension, so
//   - the bounding box is the first and last entry of each list,
//   - the element of rank floor(n/2) along the widest dimension is one
//     lookup and the number of elements below it a short search,
//   - the split dimension's list is already partitioned (its left child is
//     a prefix), and every other list is split by one stable pass that
//     keeps it sorted.
// The splitter rules, the sample, the leaves and the node records are those
// of the radix-select frame (same tree, different work): the widest
// dimension (ties lowest), rank floor(count/2), the next larger distinct
// value when nothing lies below it, equal keys to the right; a Build root
// with at least 2*sigma_os sampled points splits on the sample, otherwise
// on its points.
//
// Lists live in d + 1 physical buffers; a node's `map` names the buffer of
// each dimension (4 bits each) and the one left over is its spare, into
// which the next list is partitioned.  Nodes own disjoint position ranges,
// so their buffers never collide.
//
// Scheduling is the team scheme of the radix-select frame: the root is
// processed by all 16 warps, teams halve at every split (tiny children are
// deferred to the first warp's stack), single warps finish their subtrees
// depth first, always continuing with the smaller child.
#pragma once

#include "smem_build.cuh"

namespace pkd {

constexpr int SS_NW = 16;
constexpr int SS_THREADS = SS_NW * 32;
constexpr int SS_RED = 2 * PKD_DMAX + 8;  // reduction ints per warp
constexpr int SS_STK = 32;                // deferred tasks per warp

struct STask {
  uint16_t lo, hi, ns;
  uint8_t j, pad;
  uint32_t t;     // tree depth
  uint32_t slot;  // node slot
  uint32_t map;   // physical list buffer of dimension k in bits [4k, 4k+4)
  uint32_t pad2;
};
static_assert(sizeof(STask) == 24, "STask layout");

struct SortedLayout {
  size_t X, ID, lists, flag, red, stack, ctl, total;
};

// Shared memory of one CTA holding up to `cap` points of d dimensions.  The
// radix counters of the presort (16 warps x 256 u32) share the task stacks.
__host__ __device__ inline SortedLayout sorted_layout(int cap, int d) {
  SortedLayout L;
  size_t o = 0;
  L.X = o;
  o = align_up(o + (size_t)4 * d * cap, 16);
  L.ID = o;
  o = align_up(o + (size_t)4 * cap, 16);
  L.lists = o;
  o = align_up(o + (size_t)2 * (d + 1) * cap, 16);
  L.flag = o;
  o = align_up(o + (size_t)cap, 16);
  L.red = o;
  o = align_up(o + (size_t)SS_NW * SS_RED * 4, 16);
  L.stack = o;
  const size_t stk = (size_t)SS_NW * SS_STK * sizeof(STask), hist = (size_t)SS_NW * 256 * 4;
  o = align_up(o + (stk > hist ? stk : hist), 16);
  L.ctl = o;
  o = align_up(o + sizeof(SmemCtl), 16);
  L.total = o;
  return L;
}

__device__ __forceinline__ int mget(uint32_t m, int k) { return (int)((m >> (4 * k)) & 15u); }
__device__ __forceinline__ uint32_t mset(uint32_t m, int k, int b) {
  return (m & ~(15u << (4 * k))) | ((uint32_t)b << (4 * k));
}
template <int D>
__device__ __forceinline__ int spare_of(uint32_t m) {
  int s = D * (D + 1) / 2;
#pragma unroll
  for (int k = 0; k < D; ++k) s -= mget(m, k);
  return s;
}

template <int D>
struct SCtx {
  Params p;
  const int32_t* X;  // [D][cap]
  const uint32_t* ID;
  uint8_t* flag;
  uint16_t* lists;  // [D + 1][cap]
  int cap;
  SmemCtl* ctl;
  Pts out;
  uint64_t start;
  uint32_t slot_base;
  int slot_limit;
  Node* nodes;
  uint8_t* ndim;
  DevStatus* st;
  __device__ uint16_t* list(int b) const { return lists + b * cap; }
  __device__ int32_t key(int dim, int p) const { return X[dim * cap + p]; }
};

// ---------------------------------------------------------------------------
// Presort: one stable counting pass per 8-bit digit, all warps of the CTA.
// Warp w owns a contiguous run of positions and its own 256 counters; within
// a group of 32 positions, lanes that share a digit are ranked by their
// peer mask, so equal digits keep their order.  Loads are issued SS_BATCH groups at a
// time before any store (the compiler cannot move them past the stores).
// ---------------------------------------------------------------------------
constexpr int SS_BATCH = 4;

__device__ __forceinline__ void radix_pass(const int32_t* Xj, unsigned vmin, int shift, const uint16_t* src,
                                           uint16_t* dst, int n, unsigned* hist, int* tmp) {
  const int w = warp_id(), lane = lane_id(), tid = threadIdx.x;
  const int per = ((n + SS_THREADS - 1) / SS_THREADS) * 32;
  const int wlo = min(n, w * per), whi = min(n, wlo + per);
  const int ng = (whi - wlo + 31) >> 5;
  unsigned* H = hist + w * 256;
#pragma unroll
  for (int i = lane; i < 256; i += 32) H[i] = 0;
  __syncwarp();
  for (int g0 = 0; g0 < ng; g0 += SS_BATCH) {
    int dg[SS_BATCH];
#pragma unroll
    for (int u = 0; u < SS_BATCH; ++u) {
      const int i = wlo + (g0 + u) * 32 + lane;
      dg[u] = -1;
      if (i < whi) dg[u] = (int)((((unsigned)Xj[src ? src[i] : i] - vmin) >> shift) & 255u);
    }
#pragma unroll
    for (int u = 0; u < SS_BATCH; ++u) {
      if (g0 + u < ng) {
        if (dg[u] >= 0) atomicAdd(&H[dg[u]], 1u);
      }
    }
  }
  __syncthreads();
  // exclusive offsets per (digit, warp), digit-major: lanes 2i and 2i+1 of
  // warp w own digit 16w + i, each summing the counters of 8 warps
  {
    const int dgt = tid >> 1, h = tid & 1;
    unsigned part = 0;
#pragma unroll
    for (int v = 0; v < SS_NW / 2; ++v) part += hist[(h * (SS_NW / 2) + v) * 256 + dgt];
    const unsigned other = __shfl_xor_sync(FULL_MASK, part, 1);
    const unsigned tot = part + other;
    const unsigned inc = (unsigned)warp_incl_scan(h == 0 ? (int)tot : 0);
    if (lane == 31) tmp[w] = (int)inc;
    __syncthreads();
    unsigned run = inc - tot + (h ? other : 0u);
    for (int v = 0; v < w; ++v) run += (unsigned)tmp[v];
#pragma unroll
    for (int v = 0; v < SS_NW / 2; ++v) {
      unsigned* c = &hist[(h * (SS_NW / 2) + v) * 256 + dgt];
      const unsigned cnt = *c;
      *c = run;
      run += cnt;
    }
  }
  __syncthreads();
  for (int g0 = 0; g0 < ng; g0 += SS_BATCH) {
    int dg[SS_BATCH], pp[SS_BATCH];
#pragma unroll
    for (int u = 0; u < SS_BATCH; ++u) {
      const int i = wlo + (g0 + u) * 32 + lane;
      dg[u] = -1;
      pp[u] = 0;
      if (i < whi) {
        pp[u] = src ? src[i] : i;
        dg[u] = (int)((((unsigned)Xj[pp[u]] - vmin) >> shift) & 255u);
      }
    }
#pragma unroll
    for (int u = 0; u < SS_BATCH; ++u) {
      if (g0 + u < ng) {
        const unsigned m = peer_mask_c<8>(dg[u]);
        const int leader = __ffs(m) - 1;
        const unsigned cur = dg[u] >= 0 ? H[dg[u]] : 0u;
        if (dg[u] >= 0) dst[cur + __popc(m & lanemask_lt())] = (uint16_t)pp[u];
        __syncwarp();
        if (dg[u] >= 0 && lane == leader) H[dg[u]] = cur + (unsigned)__popc(m);
        __syncwarp();
      }
    }
  }
  __syncthreads();
}

// Sort dimension k of the n loaded points into buffer k (buffer D is the
// ping-pong partner).  vmin/vmax bound the coordinates.
template <int D>
__device__ void presort_dim(const SCtx<D>& cx, int k, int vmin, int vmax, int n, unsigned* hist, int* tmp) {
  const int32_t* Xk = cx.X + k * cx.cap;
  uint16_t* target = cx.list(k);
  uint16_t* partner = cx.list(D);
  const unsigned range = (unsigned)vmax - (unsigned)vmin;
  const int bits = range ? 32 - __clz(range) : 0;
  const int passes = (bits + 7) / 8;
  if (passes == 0) {
    for (int i = threadIdx.x; i < n; i += SS_THREADS) target[i] = (uint16_t)i;
    __syncthreads();
    return;
  }
  // the last pass must land in `target`
  uint16_t* out = (passes & 1) ? target : partner;
  const uint16_t* in = nullptr;
  for (int ps = 0; ps < passes; ++ps) {
    radix_pass(Xk, (unsigned)vmin, 8 * ps, in, out, n, hist, tmp);
    in = out;
    out = (out == target) ? partner : target;
  }
}

// Faster presort for the common case: one most-significant-digit counting
// pass over MSD_BINS bins of the top varying bits (plain shared-memory
// atomics, no ranking), then every bin, now a contiguous run of the list, is
// sorted by (coordinate, point index) by one thread.  The order is the same
// as the stable LSD sort's.  Returns false, before writing the list, when a
// bin holds more than MSD_MAX_BUCKET points (clustered coordinates); the
// caller then sorts that dimension with presort_dim.
constexpr int MSD_BITS = 12;
constexpr int MSD_BINS = 1 << MSD_BITS;  // 4096 counters fill the 16 KB radix region
constexpr int MSD_MAX_BUCKET = 64;
constexpr int MSD_PER = MSD_BINS / SS_THREADS;  // bins per thread

template <int D>
__device__ bool presort_dim_msd(const SCtx<D>& cx, int k, int vmin, int vmax, int n, unsigned* hist, int* tmp) {
  static_assert(MSD_PER * SS_THREADS == MSD_BINS && MSD_BINS <= SS_NW * 256, "bins per thread, radix region");
  const int32_t* Xk = cx.X + k * cx.cap;
  uint16_t* target = cx.list(k);
  const unsigned range = (unsigned)vmax - (unsigned)vmin;
  const int bits = range ? 32 - __clz(range) : 0;
  const int shift = max(0, bits - MSD_BITS);
  const int tid = threadIdx.x, lane = lane_id(), w = warp_id();
#pragma unroll
  for (int q = 0; q < MSD_PER; ++q) hist[q * SS_THREADS + tid] = 0;
  __syncthreads();
  for (int i = tid; i < n; i += SS_THREADS) atomicAdd(&hist[((unsigned)Xk[i] - (unsigned)vmin) >> shift], 1u);
  __syncthreads();
  // bin starts: thread t owns bins [MSD_PER t, MSD_PER (t + 1))
  unsigned c[MSD_PER], sum = 0, mx = 0;
#pragma unroll
  for (int q = 0; q < MSD_PER; ++q) {
    c[q] = hist[MSD_PER * tid + q];
    sum += c[q];
    mx = max(mx, c[q]);
  }
  const unsigned inc = (unsigned)warp_incl_scan((int)sum);
  const unsigned wmx = (unsigned)warp_max((int)mx);
  if (lane == 31) tmp[w] = (int)inc;
  if (lane == 0) tmp[SS_NW + w] = (int)wmx;
  __syncthreads();
  unsigned run = inc - sum, big = 0;
  for (int v = 0; v < SS_NW; ++v) {
    if (v < w) run += (unsigned)tmp[v];
    big = max(big, (unsigned)tmp[SS_NW + v]);
  }
  if (big > (unsigned)MSD_MAX_BUCKET) {
    __syncthreads();  // every thread has read tmp before the caller reuses it
    return false;
  }
#pragma unroll
  for (int q = 0; q < MSD_PER; ++q) {
    hist[MSD_PER * tid + q] = run;
    run += c[q];
  }
  __syncthreads();
  for (int i = tid; i < n; i += SS_THREADS)
    target[atomicAdd(&hist[((unsigned)Xk[i] - (unsigned)vmin) >> shift], 1u)] = (uint16_t)i;
  __syncthreads();
  // hist[b] is now the end of bin b; sort each bin by (coordinate, index)
  for (int b = tid; b < MSD_BINS; b += SS_THREADS) {
    const int e = (int)hist[b], st = b ? (int)hist[b - 1] : 0;
    for (int i = st + 1; i < e; ++i) {
      const int v = target[i];
      const int32_t kv = Xk[v];
      int j = i - 1;
      while (j >= st) {
        const int u = target[j];
        const int32_t ku = Xk[u];
        if (ku < kv || (ku == kv && u < v)) break;
        target[j + 1] = (uint16_t)u;
        --j;
      }
      target[j + 1] = (uint16_t)v;
    }
  }
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------
// Node steps (uniform within the team that calls them)
// ---------------------------------------------------------------------------

// First position in [a, b) whose key along `dim` is >= x (b if none).
template <int D>
__device__ __forceinline__ int lower_pos(const SCtx<D>& cx, const uint16_t* Lst, int dim, int a, int b, int x) {
  while (a < b) {
    const int mid = (a + b) >> 1;
    if (cx.key(dim, Lst[mid]) < x) a = mid + 1;
    else b = mid;
  }
  return a;
}
// First position in [a, b) whose key along `dim` is > x (b if none).
template <int D>
__device__ __forceinline__ int upper_pos(const SCtx<D>& cx, const uint16_t* Lst, int dim, int a, int b, int x) {
  while (a < b) {
    const int mid = (a + b) >> 1;
    if (cx.key(dim, Lst[mid]) <= x) a = mid + 1;
    else b = mid;
  }
  return a;
}

// A finished leaf: its node record, and its points' indices moved into
// list buffer 0 at its positions (no other node uses positions [lo, hi) of
// any buffer), from which the CTA writes every point out in one coalesced
// pass at the end.
template <int D>
__device__ __forceinline__ void semit_leaf(const Team& tm, const SCtx<D>& cx, const STask& tk) {
  const int b0 = mget(tk.map, 0);
  if (b0 != 0) {
    const uint16_t* P = cx.list(b0);
    uint16_t* Q = cx.list(0);
    for (int i = tk.lo + tm.rank(); i < tk.hi; i += tm.size()) Q[i] = P[i];
  }
  if (tm.leader()) {
    cx.nodes[tk.slot] = Node{0, (uint32_t)(tk.hi - tk.lo), (uint32_t)(cx.start + tk.lo), 0};
    cx.ndim[tk.slot] = PKD_LEAF;
    atomicMax(&cx.ctl->maxd, tk.t);
  }
}

// The number of points of [lo, hi) sampled at depth t; with WRITE also
// flag[p] = sampled.  A node first counts; only a node whose sample reaches
// the split threshold (rare below the sieve rounds) writes the flags, which
// only its splits on the sample read.
template <int D, bool WRITE>
__device__ __forceinline__ int sdraw_sample(const Team& tm, const SCtx<D>& cx, uint32_t map, int lo, int hi,
                                            uint32_t t, int shift) {
  const uint16_t* P = cx.list(mget(map, 0));
  const uint64_t key = sample_key(cx.p.seed, t);
  int c = 0;
  constexpr int U = 4;
  for (int i0 = lo + tm.rank(); i0 < hi; i0 += U * tm.size()) {
    int pp[U];
    uint32_t id[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * tm.size();
      pp[u] = i < hi ? (int)P[i] : -1;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) id[u] = pp[u] >= 0 ? cx.ID[pp[u]] : 0u;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (pp[u] >= 0) {
        const bool f = in_sample_k(key, id[u], shift);
        if (WRITE) cx.flag[pp[u]] = f;
        c += f;
      }
    }
  }
  if (WRITE) tm.sync();
  return tm.sum(c);
}

// Number of flagged entries of Lst[a, b).
template <int D>
__device__ __forceinline__ int scount_flagged(const Team& tm, const SCtx<D>& cx, const uint16_t* Lst, int a, int b) {
  int c = 0;
  for (int i = a + tm.rank(); i < b; i += tm.size()) c += cx.flag[Lst[i]];
  return tm.sum(c);
}

// First position in [a, b) whose entry is flagged (b if none).
template <int D>
__device__ __forceinline__ int sfirst_flagged(const Team& tm, const SCtx<D>& cx, const uint16_t* Lst, int a, int b) {
  int m = INT32_MAX;
  for (int i = a + tm.rank(); i < b; i += tm.size())
    if (cx.flag[Lst[i]]) {
      m = i;
      break;
    }
  m = tm.vmin(m);
  return m == INT32_MAX ? b : m;
}

// Position of the flagged entry of rank k (0-based) in Lst[lo, hi).
template <int D>
__device__ int snth_flagged(const Team& tm, const SCtx<D>& cx, const uint16_t* Lst, int lo, int hi, int k) {
  const int n = hi - lo, nw = tm.nwarps(), w = tm.my_warp(), lane = lane_id();
  const int per = ((n + nw * 32 - 1) / (nw * 32)) * 32;
  const int wlo = min(hi, lo + w * per), whi = min(hi, wlo + per);
  int c = 0;
  for (int base = wlo; base < whi; base += 32) {
    const int i = base + lane;
    c += __popc(__ballot_sync(FULL_MASK, i < whi && cx.flag[Lst[i]]));
  }
  int before = 0;
  if (nw > 1) {
    if (lane == 0) tm.red[w * SS_RED] = c;
    if (tm.leader()) tm.red[SS_RED - 1] = -1;
    tm.sync();
    before = warp_sum(lane < w ? tm.red[lane * SS_RED] : 0);
    tm.sync();
  }
  int found = -1;
  if (k >= before && k < before + c) {
    int r = k - before;
    for (int base = wlo; base < whi; base += 32) {
      const int i = base + lane;
      const unsigned b = __ballot_sync(FULL_MASK, i < whi && cx.flag[Lst[i]]);
      if (r < __popc(b)) {
        unsigned bb = b;
        for (int q = 0; q < r; ++q) bb &= bb - 1;
        found = base + __ffs(bb) - 1;
        break;
      }
      r -= __popc(b);
    }
  }
  if (nw == 1) return found;
  if (found >= 0 && lane == 0) tm.red[SS_RED - 1] = found;
  tm.sync();
  const int res = tm.red[SS_RED - 1];
  tm.sync();
  return res;
}

// Splitter on the sample of node tk (flagged points): widest dimension of the
// sample's box (ties lowest), sampled element of rank floor(ns/2), the next
// larger sampled value when no sampled point lies below it.  On success dim,
// x, L = points below x and SL = sampled points below x.  False when every
// sampled point is identical.
template <int D>
__device__ bool ssample_split(const Team& tm, const SCtx<D>& cx, const STask& tk, int& dim, int& x, int& L,
                              int& SL) {
  const int lo = tk.lo, hi = tk.hi;
  int mn[D], mx[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    mn[j] = INT32_MAX;
    mx[j] = INT32_MIN;
  }
  const uint16_t* P0 = cx.list(mget(tk.map, 0));
  for (int i = lo + tm.rank(); i < hi; i += tm.size()) {
    const int p = P0[i];
    if (!cx.flag[p]) continue;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const int v = cx.key(j, p);
      mn[j] = min(mn[j], v);
      mx[j] = max(mx[j], v);
    }
  }
#pragma unroll
  for (int j = 0; j < D; ++j) {
    mn[j] = warp_min(mn[j]);
    mx[j] = warp_max(mx[j]);
  }
  if (tm.nwarps() > 1) {
    if (lane_id() == 0) {
#pragma unroll
      for (int j = 0; j < D; ++j) {
        tm.red[tm.my_warp() * SS_RED + j] = mn[j];
        tm.red[tm.my_warp() * SS_RED + D + j] = mx[j];
      }
    }
    tm.sync();
    const int ln = lane_id();
#pragma unroll
    for (int j = 0; j < D; ++j) {
      mn[j] = warp_min(ln < tm.nwarps() ? tm.red[ln * SS_RED + j] : INT32_MAX);
      mx[j] = warp_max(ln < tm.nwarps() ? tm.red[ln * SS_RED + D + j] : INT32_MIN);
    }
    tm.sync();
  }
  int vmin, vmax;
  dim = widest_dim<D>(mn, mx, vmin, vmax);
  if (dim < 0) return false;
  const uint16_t* Ld = cx.list(mget(tk.map, dim));
  const int pos = snth_flagged<D>(tm, cx, Ld, lo, hi, tk.ns / 2);
  if (pos < lo || pos >= hi) {  // the sample count disagrees with the flags
    if (tm.leader()) set_error(cx.st, DERR_STATE, 350);
    return false;
  }
  x = cx.key(dim, Ld[pos]);
  int lb = lower_pos<D>(cx, Ld, dim, lo, pos, x);
  if (scount_flagged<D>(tm, cx, Ld, lo, lb) == 0) {
    // no sampled point below x: the next larger sampled value
    const int ub = upper_pos<D>(cx, Ld, dim, pos, hi, x);
    const int p2 = sfirst_flagged<D>(tm, cx, Ld, ub, hi);
    if (p2 >= hi) {
      if (tm.leader()) set_error(cx.st, DERR_STATE, 351);
      return false;
    }
    x = cx.key(dim, Ld[p2]);
    lb = lower_pos<D>(cx, Ld, dim, ub, p2, x);
  }
  L = lb - lo;
  SL = scount_flagged<D>(tm, cx, Ld, lo, lb);
  return true;
}

// One batch of B groups of 32 entries of src starting at base0 (entries at
// b or beyond are absent): loads first, then the stable split by
// Xd[p] < x into dst at lb (left) and rb (right), both advanced.
template <int B>
__device__ __forceinline__ void warp_split_batch(const int32_t* Xd, int x, const uint16_t* src, uint16_t* dst,
                                                 int base0, int b, int& lb, int& rb) {
  const int lane = lane_id();
  int pp[B];
  bool lf[B];
#pragma unroll
  for (int u = 0; u < B; ++u) {
    const int i = base0 + u * 32 + lane;
    pp[u] = i < b ? (int)src[i] : -1;
  }
#pragma unroll
  for (int u = 0; u < B; ++u) lf[u] = pp[u] >= 0 && Xd[pp[u]] < x;
#pragma unroll
  for (int u = 0; u < B; ++u) {
    const int rem = b - (base0 + u * 32);
    if (rem > 0) {
      const unsigned vm = rem >= 32 ? FULL_MASK : ((1u << rem) - 1u);  // lanes holding an entry
      const unsigned bl = __ballot_sync(FULL_MASK, lf[u]), br = vm & ~bl;
      if (lf[u]) dst[lb + __popc(bl & lanemask_lt())] = (uint16_t)pp[u];
      else if (pp[u] >= 0) dst[rb + __popc(br & lanemask_lt())] = (uint16_t)pp[u];
      lb += __popc(bl);
      rb += __popc(br);
    }
  }
}

// Stable split of src[a, b) by Xd[p] < x into dst: left entries from lb,
// right entries from rb (both advanced).  One warp; the batch size follows
// the run's length, so a short run issues no empty groups.
__device__ __forceinline__ void warp_split_run(const int32_t* Xd, int x, const uint16_t* src, uint16_t* dst, int a,
                                               int b, int& lb, int& rb) {
  int base0 = a;
  for (; b - base0 > 128; base0 += 256) warp_split_batch<8>(Xd, x, src, dst, base0, b, lb, rb);
  if (b - base0 > 64) warp_split_batch<4>(Xd, x, src, dst, base0, b, lb, rb);
  else if (b - base0 > 32) warp_split_batch<2>(Xd, x, src, dst, base0, b, lb, rb);
  else if (b - base0 > 0) warp_split_batch<1>(Xd, x, src, dst, base0, b, lb, rb);
}

// Number of entries of src[a, b) with Xd[p] < x, counted by one warp.
__device__ __forceinline__ int warp_count_left(const int32_t* Xd, int x, const uint16_t* src, int a, int b) {
  const int lane = lane_id();
  int c = 0;
  for (int base0 = a; base0 < b; base0 += 32 * SS_BATCH) {
    int pp[SS_BATCH];
#pragma unroll
    for (int u = 0; u < SS_BATCH; ++u) {
      const int i = base0 + u * 32 + lane;
      pp[u] = i < b ? (int)src[i] : -1;
    }
#pragma unroll
    for (int u = 0; u < SS_BATCH; ++u) c += (pp[u] >= 0 && Xd[pp[u]] < x);
  }
  return warp_sum(c);
}

// Split every list except `dim`'s around x (stable), given L points below
// x; returns the children's map.
template <int D>
__device__ uint32_t spartition(const Team& tm, const SCtx<D>& cx, uint32_t map, int lo, int hi, int dim, int x,
                               int L) {
  const int32_t* Xd = cx.X + dim * cx.cap;
  int spare = spare_of<D>(map);
  const int lane = lane_id();
  const int nw = tm.nwarps(), w = tm.my_warp(), n = hi - lo;
  if (nw == 1) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (k == dim) continue;
      int lb = lo, rb = lo + L;
      warp_split_run(Xd, x, cx.list(mget(map, k)), cx.list(spare), lo, hi, lb, rb);
      __syncwarp();
      const int freed = mget(map, k);
      map = mset(map, k, spare);
      spare = freed;
    }
    return map;
  }
  const int per = ((n + nw * 32 - 1) / (nw * 32)) * 32;
  const int wlo = min(hi, lo + w * per), whi = min(hi, wlo + per);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if (k == dim) continue;
    const int cl = warp_count_left(Xd, x, cx.list(mget(map, k)), wlo, whi);
    if (lane == 0) tm.red[w * SS_RED + k] = cl;
  }
  tm.sync();
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if (k == dim) continue;
    // left entries in the chunks of the warps before this one
    const int before = warp_sum(lane < w ? tm.red[lane * SS_RED + k] : 0);
    int lb = lo + before, rb = lo + L + (wlo - lo - before);
    warp_split_run(Xd, x, cx.list(mget(map, k)), cx.list(spare), wlo, whi, lb, rb);
    // the next list is written where this one was read
    tm.sync();
    const int freed = mget(map, k);
    map = mset(map, k, spare);
    spare = freed;
  }
  return map;
}

// Process one node; returns the number of children written to ch (0 or 2).
template <int D>
__device__ int snode(const Team& tm, const SCtx<D>& cx, STask tk, STask* ch) {
  for (;;) {
    const int lo = tk.lo, hi = tk.hi, n = hi - lo;
    int dim = 0, x = 0, L = 0, SL = 0;
    bool on_sample = false;
    if (tk.j == 0) {
      // Build(P, t): leaf wrap, heavy leaf, then sample and skeleton root.
      if (n <= cx.p.phi) {
        semit_leaf<D>(tm, cx, tk);
        return 0;
      }
      int wd = -1;
      long long ext = 0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const uint16_t* Lk = cx.list(mget(tk.map, k));
        const long long e = (long long)cx.key(k, Lk[hi - 1]) - (long long)cx.key(k, Lk[lo]);
        if (e > ext) {
          ext = e;
          wd = k;
        }
      }
      if (wd < 0) {
        semit_leaf<D>(tm, cx, tk);
        return 0;
      }
      // fewer than 2*sigma_os points cannot reach the split threshold
      int ns = 0;
      if (n >= 2 * cx.p.sigma_os) {
        const int sh = sample_shift(cx.p, (uint64_t)n);
        ns = sdraw_sample<D, false>(tm, cx, tk.map, lo, hi, tk.t, sh);
        if (ns >= 2 * cx.p.sigma_os) sdraw_sample<D, true>(tm, cx, tk.map, lo, hi, tk.t, sh);
      }
      tk.ns = (uint16_t)ns;
      if (ns >= 2 * cx.p.sigma_os && ssample_split<D>(tm, cx, tk, dim, x, L, SL)) {
        on_sample = true;
      } else {
        // one exact level on the points: rank floor(n/2) along wd
        dim = wd;
        const uint16_t* Ld = cx.list(mget(tk.map, dim));
        const int k = n / 2;
        x = cx.key(dim, Ld[lo + k]);
        L = (k > 0 && cx.key(dim, Ld[lo + k - 1]) < x) ? k : lower_pos<D>(cx, Ld, dim, lo, lo + k, x) - lo;
        if (L == 0) {
          const int ub = upper_pos<D>(cx, Ld, dim, lo + k, hi, x);
          x = ub < hi ? cx.key(dim, Ld[ub]) : x;
          L = ub - lo;  // hi - lo (caught below) only if the list were unsorted
        }
      }
    } else {
      // skeleton node: a bucket when deep enough, too few samples or identical
      if (tk.j >= cx.p.lambda || tk.ns < 2 * cx.p.sigma_os) {
        tk.j = 0;
        continue;
      }
      if (!ssample_split<D>(tm, cx, tk, dim, x, L, SL)) {
        tk.j = 0;
        continue;
      }
      on_sample = true;
    }
    if (L <= 0 || L >= n) {
      if (tm.leader()) set_error(cx.st, DERR_STATE, 300 + L);
      return 0;
    }
    // both children wrap into leaves (at most phi points each, and neither
    // is a skeleton node that its sample would split further): their points
    // are the two runs of the list sorted along dim, so no other list needs
    // splitting and no child task is made
    const bool sk_child = on_sample && tk.j + 1 < cx.p.lambda;
    const bool leaves = L <= cx.p.phi && n - L <= cx.p.phi &&
                        (!sk_child || (SL < 2 * cx.p.sigma_os && tk.ns - SL < 2 * cx.p.sigma_os));
    const uint32_t cmap = leaves ? tk.map : spartition<D>(tm, cx, tk.map, lo, hi, dim, x, L);
    int b = 0;
    if (tm.leader()) b = atomicAdd(&cx.ctl->next_slot, 2);
    b = tm.bcast(b);
    if (b + 2 > cx.slot_limit) {
      if (tm.leader()) set_error(cx.st, DERR_SLOT, b);
      return 0;
    }
    const uint32_t sl = cx.slot_base + (uint32_t)b, sr = sl + 1;
    if (tm.leader()) {
      cx.nodes[tk.slot] = Node{x, (uint32_t)n, sl, sr};
      cx.ndim[tk.slot] = (uint8_t)dim;
    }
    if (leaves) {
      const int bd = mget(tk.map, dim);
      if (bd != 0) {  // leaves are written out from list buffer 0
        const uint16_t* P = cx.list(bd);
        uint16_t* Q = cx.list(0);
        for (int i = lo + tm.rank(); i < hi; i += tm.size()) Q[i] = P[i];
      }
      if (tm.leader()) {
        cx.nodes[sl] = Node{0, (uint32_t)L, (uint32_t)(cx.start + lo), 0};
        cx.ndim[sl] = PKD_LEAF;
        cx.nodes[sr] = Node{0, (uint32_t)(n - L), (uint32_t)(cx.start + lo + L), 0};
        cx.ndim[sr] = PKD_LEAF;
        atomicMax(&cx.ctl->maxd, tk.t + 1);
      }
      return 0;
    }
    const uint8_t nj = on_sample ? (uint8_t)(tk.j + 1) : (uint8_t)0;
    const int SR = on_sample ? tk.ns - SL : 0;
    ch[0] = STask{(uint16_t)lo, (uint16_t)(lo + L), (uint16_t)(on_sample ? SL : 0), nj, 0, tk.t + 1, sl, cmap, 0};
    ch[1] = STask{(uint16_t)(lo + L), (uint16_t)hi, (uint16_t)SR, nj, 0, tk.t + 1, sr, cmap, 0};
    return 2;
  }
}

// One warp finishes its subtree depth first; `stk` holds sp0 deferred tasks.
template <int D>
__device__ void swarp_run(const Team& wt, const SCtx<D>& cx, STask tk, STask* stk, int sp0) {
  int sp = sp0;
  for (int iter = 1;; ++iter) {
    STask ch[2];
    const int nch = snode<D>(wt, cx, tk, ch);
    if ((iter & 63) == 0) {  // another CTA's failure ends this one early
      const int err = *(volatile int*)&cx.st->err;
      if (__shfl_sync(FULL_MASK, err, 0)) return;  // warp-uniform exit
    }
    if (nch == 2) {
      const int s0 = ch[0].hi - ch[0].lo, s1 = ch[1].hi - ch[1].lo;
      const STask big = s0 >= s1 ? ch[0] : ch[1];
      const STask small = s0 >= s1 ? ch[1] : ch[0];
      if (sp >= SS_STK) {
        if (lane_id() == 0) set_error(cx.st, DERR_STACK, sp);
        return;
      }
      if (lane_id() == 0) stk[sp] = big;
      __syncwarp();
      ++sp;
      tk = small;
    } else {
      if (sp == 0) return;
      --sp;
      __syncwarp();
      tk = stk[sp];
      __syncwarp();
    }
  }
}

// Drive the warps of the CTA over the root task.
template <int D>
__device__ void srun_tasks(const SCtx<D>& cx, STask root, int* sred, STask* wstack) {
  const int w = warp_id();
  int f = 0, nw = SS_NW;
  STask tk = root;
  bool have_task = true;
  while (nw > 1) {
    const Team tm{f, nw, team_barrier(f, nw, SS_NW), nullptr, sred + f * SS_RED};
    STask ch[2];
    const int nch = snode<D>(tm, cx, tk, ch);
    if (nch == 0) {
      have_task = false;
      break;
    }
    const int s0 = ch[0].hi - ch[0].lo, s1 = ch[1].hi - ch[1].lo;
    const int big = s0 >= s1 ? 0 : 1;
    const int small_n = min(s0, s1);
    tm.sync();
    const bool defer = small_n <= DEFER_MAX && small_n * 8 <= max(s0, s1) && cx.ctl->wsp[f] < SS_STK;
    tm.sync();
    if (defer) {
      if (tm.leader()) {
        wstack[f * SS_STK + cx.ctl->wsp[f]] = ch[big ^ 1];
        cx.ctl->wsp[f] += 1;
      }
      tm.sync();
      tk = ch[big];
      continue;
    }
    const int half = nw / 2;
    const bool second = w >= f + half;
    tk = second ? ch[1] : ch[0];
    if (second) f += half;
    nw = half;
  }
  __syncwarp();
  int sp0 = cx.ctl->wsp[w];
  if (!have_task) {
    if (sp0 == 0) return;
    tk = wstack[w * SS_STK + --sp0];
  }
  __syncwarp();
  const Team wt{w, 1, 0, nullptr, sred + w * SS_RED};
  swarp_run<D>(wt, cx, tk, wstack + w * SS_STK, sp0);
}

}  // namespace pkd
