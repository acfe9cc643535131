// Cooperative primitives for one warp or one thread block working on a set
// of points held in shared memory: min/max per dimension, exact selection of
// the element of a given rank (radix select, 8-bit digits), and stable
// partition of an index list around a splitter.  The same templates serve the
// whole-block phase and the per-warp phase of the shared-memory kernels.
#pragma once

#include "common.cuh"

namespace pkd {

constexpr unsigned FULL_MASK = 0xffffffffu;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }
__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
  return v;
}
__device__ __forceinline__ int warp_min(int v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(FULL_MASK, v, o));
  return v;
}
__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(FULL_MASK, v, o));
  return v;
}
__device__ __forceinline__ int warp_incl_scan(int v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(FULL_MASK, v, o);
    if (lane_id() >= o) v += t;
  }
  return v;
}

// Red scratch: RED_INTS ints per team.
constexpr int RED_INTS = 32 * (2 * PKD_DMAX + 2) + 8;

struct WarpTeam {
  unsigned* hist;  // 256 counters
  int* red;
  __device__ int rank() const { return lane_id(); }
  __device__ int size() const { return 32; }
  __device__ bool leader() const { return lane_id() == 0; }
  __device__ void sync() const { __syncwarp(); }
  __device__ int nwarps() const { return 1; }
  __device__ int my_warp() const { return 0; }
  __device__ int bcast(int v) const { return __shfl_sync(FULL_MASK, v, 0); }
  __device__ int sum(int v) const { return warp_sum(v); }
};

template <int NW>
struct BlockTeam {
  unsigned* hist;
  int* red;
  __device__ int rank() const { return threadIdx.x; }
  __device__ int size() const { return NW * 32; }
  __device__ bool leader() const { return threadIdx.x == 0; }
  __device__ void sync() const { __syncthreads(); }
  __device__ int nwarps() const { return NW; }
  __device__ int my_warp() const { return warp_id(); }
  __device__ int bcast(int v) const {
    if (threadIdx.x == 0) red[0] = v;
    __syncthreads();
    int r = red[0];
    __syncthreads();
    return r;
  }
  __device__ int sum(int v) const {
    v = warp_sum(v);
    if (lane_id() == 0) red[warp_id()] = v;
    __syncthreads();
    int r = 0;
    for (int i = 0; i < NW; ++i) r += red[i];
    __syncthreads();
    return r;
  }
};

// Shared-memory view of the points of one subproblem.
struct SmemPts {
  const int32_t* X;   // [d][cap]
  const uint32_t* ID; // [cap]
  const uint8_t* flag;
  int cap;
  int d;
  __device__ int32_t x(int j, int p) const { return X[j * cap + p]; }
};

// Min and max of every dimension over idx[lo, hi) (only flagged points when
// `sampled_only`).  Results are valid in every thread of the team.
template <class T>
__device__ void team_minmax(const T& tm, const SmemPts& s, const uint16_t* idx, int lo, int hi,
                            bool sampled_only, int* mn, int* mx) {
  int lmn[PKD_DMAX], lmx[PKD_DMAX];
#pragma unroll
  for (int j = 0; j < PKD_DMAX; ++j) {
    lmn[j] = INT32_MAX;
    lmx[j] = INT32_MIN;
  }
  for (int i = lo + tm.rank(); i < hi; i += tm.size()) {
    int p = idx[i];
    if (sampled_only && !s.flag[p]) continue;
#pragma unroll
    for (int j = 0; j < PKD_DMAX; ++j) {
      if (j < s.d) {
        int v = s.x(j, p);
        lmn[j] = min(lmn[j], v);
        lmx[j] = max(lmx[j], v);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < PKD_DMAX; ++j) {
    if (j < s.d) {
      lmn[j] = warp_min(lmn[j]);
      lmx[j] = warp_max(lmx[j]);
    }
  }
  if (tm.nwarps() == 1) {
#pragma unroll
    for (int j = 0; j < PKD_DMAX; ++j) {
      mn[j] = lmn[j];
      mx[j] = lmx[j];
    }
    return;
  }
  const int stride = 2 * PKD_DMAX;
  if (lane_id() == 0) {
#pragma unroll
    for (int j = 0; j < PKD_DMAX; ++j) {
      tm.red[tm.my_warp() * stride + j] = lmn[j];
      tm.red[tm.my_warp() * stride + PKD_DMAX + j] = lmx[j];
    }
  }
  tm.sync();
#pragma unroll
  for (int j = 0; j < PKD_DMAX; ++j) {
    int a = INT32_MAX, b = INT32_MIN;
    if (j < s.d) {
      for (int w = 0; w < tm.nwarps(); ++w) {
        a = min(a, tm.red[w * stride + j]);
        b = max(b, tm.red[w * stride + PKD_DMAX + j]);
      }
    }
    mn[j] = a;
    mx[j] = b;
  }
  tm.sync();
}

// Widest dimension (ties: lowest); -1 when every extent is zero.
__device__ __forceinline__ int widest_dim(const int* mn, const int* mx, int d) {
  int best = -1;
  long long ext = 0;
#pragma unroll
  for (int j = 0; j < PKD_DMAX; ++j) {
    long long e = (long long)mx[j] - (long long)mn[j];
    if (j < d && e > ext) {
      ext = e;
      best = j;
    }
  }
  return best;
}

// One warp scans hist[0..256): finds digit with below <= k < below+hist[digit].
__device__ __forceinline__ void warp_find_digit(const unsigned* hist, int k, int& digit, int& below,
                                                int& eq) {
  int lane = lane_id();
  int c[8];
  int s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    c[i] = (int)hist[lane * 8 + i];
    s += c[i];
  }
  int incl = warp_incl_scan(s);
  int excl = incl - s;
  unsigned hit = __ballot_sync(FULL_MASK, excl <= k && k < incl);
  int src = __ffs(hit) - 1;
  int dg = 0, bl = 0, e = 0;
  if (lane == src) {
    int acc = excl;
    bool found = false;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (!found && k < acc + c[i]) {  // acc <= k here, so c[i] > 0
        found = true;
        dg = lane * 8 + i;
        bl = acc;
        e = c[i];
      }
      acc += c[i];
    }
  }
  digit = __shfl_sync(FULL_MASK, dg, src < 0 ? 0 : src);
  below = __shfl_sync(FULL_MASK, bl, src < 0 ? 0 : src);
  eq = __shfl_sync(FULL_MASK, e, src < 0 ? 0 : src);
}

// The element of rank k (0-based) of dimension `dim` over idx[lo, hi)
// (flagged points only when `sampled_only`).  count_less / count_eq: how many
// of those elements are below / equal to it.  Coordinates are < 2^30, so the
// four 8-bit digits from bit 24 down cover them exactly.
//
// vmin/vmax bound the values: bits above their highest differing bit are
// common to every element, so the digits start just below them (a deep node
// with a narrow range needs fewer passes, and its first digit spreads over
// the bins instead of piling every element onto one counter).  Counter
// updates are aggregated per warp over lanes that hit the same bin.
template <class T>
__device__ int team_select(const T& tm, const SmemPts& s, const uint16_t* idx, int lo, int hi,
                           bool sampled_only, int dim, int k, int vmin, int vmax, int& count_less,
                           int& count_eq) {
  const int32_t* X = s.X + dim * s.cap;
  if (vmin == vmax) {
    count_less = 0;
    count_eq = k + 1;  // not used by callers in this case
    return vmin;
  }
  const int hb = 31 - __clz((unsigned)(vmin ^ vmax));  // highest differing bit
  unsigned mask = hb >= 31 ? 0u : ~((2u << hb) - 1u);
  unsigned prefix = (unsigned)vmin & mask;
  int less = 0, eq = 0;
  const int stride = tm.size();
  const int wbase = tm.my_warp() * 32;
  for (int top = hb; top >= 0; top -= 8) {
    const int shift = max(top - 7, 0);
    const unsigned dmask = (2u << (top - shift)) - 1u;
    for (int i = tm.rank(); i < 256; i += tm.size()) tm.hist[i] = 0;
    tm.sync();
    for (int base = lo + wbase; base < hi; base += stride) {
      const int i = base + lane_id();
      int key = -1;
      if (i < hi) {
        const int p = idx[i];
        const unsigned v = (unsigned)X[p];
        if ((!sampled_only || s.flag[p]) && (v & mask) == prefix) key = (int)((v >> shift) & dmask);
      }
      const unsigned m = __match_any_sync(FULL_MASK, key);
      if (key >= 0 && lane_id() == __ffs(m) - 1) atomicAdd(&tm.hist[key], (unsigned)__popc(m));
    }
    tm.sync();
    int digit, below, e;
    if (tm.nwarps() == 1) {
      warp_find_digit(tm.hist, k, digit, below, e);
    } else {
      if (warp_id() == 0) {
        warp_find_digit(tm.hist, k, digit, below, e);
        if (lane_id() == 0) {
          tm.red[0] = digit;
          tm.red[1] = below;
          tm.red[2] = e;
        }
      }
      tm.sync();
      digit = tm.red[0];
      below = tm.red[1];
      e = tm.red[2];
    }
    tm.sync();
    prefix |= (unsigned)digit << shift;
    mask |= dmask << shift;
    k -= below;
    less += below;
    eq = e;
  }
  count_less = less;
  count_eq = eq;
  return (int)prefix;
}

// Smallest value of dimension `dim` strictly above `x` over idx[lo, hi).
template <class T>
__device__ int team_min_above(const T& tm, const SmemPts& s, const uint16_t* idx, int lo, int hi,
                              bool sampled_only, int dim, int x) {
  int m = INT32_MAX;
  for (int i = lo + tm.rank(); i < hi; i += tm.size()) {
    int p = idx[i];
    if (sampled_only && !s.flag[p]) continue;
    int v = s.x(dim, p);
    if (v > x) m = min(m, v);
  }
  m = warp_min(m);
  if (tm.nwarps() == 1) return m;
  if (lane_id() == 0) tm.red[warp_id()] = m;
  tm.sync();
  int r = INT32_MAX;
  for (int w = 0; w < tm.nwarps(); ++w) r = min(r, tm.red[w]);
  tm.sync();
  return r;
}

// Splitter rule on the (flagged) points of idx[lo, hi): widest dimension,
// element of rank floor(count/2), or the next larger distinct value when
// nothing lies below it.  Returns false when the points are all identical.
template <class T>
__device__ bool team_split_rule(const T& tm, const SmemPts& s, const uint16_t* idx, int lo, int hi,
                                bool sampled_only, int count, int& dim, int& x) {
  int mn[PKD_DMAX], mx[PKD_DMAX];
  team_minmax(tm, s, idx, lo, hi, sampled_only, mn, mx);
  dim = widest_dim(mn, mx, s.d);
  if (dim < 0) return false;
  int less, eq;
  int vmn = mn[0], vmx = mx[0];
#pragma unroll
  for (int j = 1; j < PKD_DMAX; ++j)
    if (j == dim) {
      vmn = mn[j];
      vmx = mx[j];
    }
  x = team_select(tm, s, idx, lo, hi, sampled_only, dim, count / 2, vmn, vmx, less, eq);
  if (less == 0) x = team_min_above(tm, s, idx, lo, hi, sampled_only, dim, x);
  return true;
}

// Stable partition of src[lo, hi) into dst[lo, hi): points with coordinate
// `dim` below x first.  Returns the left count and the flagged counts on
// each side.
template <class T>
__device__ void team_partition(const T& tm, const SmemPts& s, const uint16_t* src, uint16_t* dst,
                               int lo, int hi, int dim, int x, int& L, int& SL, int& SR) {
  const int32_t* X = s.X + dim * s.cap;
  const int n = hi - lo;
  const int nw = tm.nwarps();
  const int per = ((n + nw * 32 - 1) / (nw * 32)) * 32;
  const int w = tm.my_warp();
  const int wlo = min(hi, lo + w * per), whi = min(hi, wlo + per);
  int cl = 0, csl = 0, csr = 0;
  for (int base = wlo; base < whi; base += 32) {
    int i = base + lane_id();
    bool valid = i < whi;
    int p = valid ? src[i] : 0;
    bool left = valid && X[p] < x;
    bool smp = valid && s.flag[p];
    cl += __popc(__ballot_sync(FULL_MASK, left));
    csl += __popc(__ballot_sync(FULL_MASK, left && smp));
    csr += __popc(__ballot_sync(FULL_MASK, !left && valid && smp));
  }
  int lbase, rbase;
  if (nw == 1) {
    L = cl;
    SL = csl;
    SR = csr;
    lbase = lo;
    rbase = lo + cl;
  } else {
    if (lane_id() == 0) {
      tm.red[3 * w + 0] = cl;
      tm.red[3 * w + 1] = csl;
      tm.red[3 * w + 2] = csr;
    }
    tm.sync();
    int tl = 0, tsl = 0, tsr = 0, before_l = 0, before_n = 0;
    for (int v = 0; v < nw; ++v) {
      int c = tm.red[3 * v];
      if (v < w) {
        before_l += c;
        before_n += min(hi, lo + v * per + per) - min(hi, lo + v * per);
      }
      tl += c;
      tsl += tm.red[3 * v + 1];
      tsr += tm.red[3 * v + 2];
    }
    L = tl;
    SL = tsl;
    SR = tsr;
    lbase = lo + before_l;
    rbase = lo + tl + (before_n - before_l);
    tm.sync();
  }
  for (int base = wlo; base < whi; base += 32) {
    int i = base + lane_id();
    bool valid = i < whi;
    int p = valid ? src[i] : 0;
    bool left = valid && X[p] < x;
    unsigned bl = __ballot_sync(FULL_MASK, left);
    unsigned br = __ballot_sync(FULL_MASK, valid && !left);
    if (left) dst[lbase + __popc(bl & lanemask_lt())] = (uint16_t)p;
    else if (valid) dst[rbase + __popc(br & lanemask_lt())] = (uint16_t)p;
    lbase += __popc(bl);
    rbase += __popc(br);
  }
  tm.sync();
}

// Set flag[p] = sampled(seed, depth, id, s) for idx[lo, hi); returns the count.
template <class T>
__device__ int team_draw_sample(const T& tm, const SmemPts& s, uint8_t* flag, const uint16_t* idx,
                                int lo, int hi, uint64_t seed, uint32_t depth, int shift) {
  int c = 0;
  for (int i = lo + tm.rank(); i < hi; i += tm.size()) {
    int p = idx[i];
    bool f = in_sample(seed, depth, s.ID[p], shift);
    flag[p] = f;
    c += f;
  }
  tm.sync();
  return tm.sum(c);
}

}  // namespace pkd
