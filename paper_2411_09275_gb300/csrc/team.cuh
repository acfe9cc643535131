// Cooperative primitives for a team of warps working on a set of points
// held in shared memory: min/max per dimension, exact selection of the
// element of a given rank (radix select), and stable partition of an index
// list around a splitter.
//
// A team is a contiguous, power-of-two range of the CTA's warps.  A team of
// one warp synchronises with __syncwarp and reduces with shuffles; a larger
// team uses its own named barrier (bar.sync id, threads), so teams that work
// on different subproblems of the same CTA never wait for each other.
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

// Lanes of the warp whose key equals this lane's, for keys in [0, 2^bits)
// (a negative key means "no key"; such lanes get an unspecified mask).
// One ballot per key bit instead of match.any, which on sm_103a issues at
// one warp-instruction per 64 cycles per SM against about one per cycle for
// a ballot.
__device__ __forceinline__ unsigned peer_mask(int key, int bits) {
  const bool valid = key >= 0;
  unsigned m = __ballot_sync(FULL_MASK, valid);
  m = valid ? m : ~m;
  for (int b = 0; b < bits; ++b) {
    const bool bit = (key >> b) & 1;
    const unsigned vb = __ballot_sync(FULL_MASK, bit);
    m &= bit ? vb : ~vb;
  }
  return m;
}
template <int BITS>
__device__ __forceinline__ unsigned peer_mask_c(int key) {
  const bool valid = key >= 0;
  unsigned m = __ballot_sync(FULL_MASK, valid);
  m = valid ? m : ~m;
#pragma unroll
  for (int b = 0; b < BITS; ++b) {
    const bool bit = (key >> b) & 1;
    const unsigned vb = __ballot_sync(FULL_MASK, bit);
    m &= bit ? vb : ~vb;
  }
  return m;
}

// Scratch ints per team (reductions over up to 16 warps and 8 dimensions).
constexpr int RED_INTS = 16 * (2 * PKD_DMAX) + 16;

struct Team {
  int first;    // first warp of the team
  int nw;       // warps in the team (power of two)
  int bar;      // named barrier id (teams of >= 2 warps)
  unsigned* hist;  // 256 counters owned by the team
  int* red;        // RED_INTS ints owned by the team
  __device__ int rank() const { return (int)threadIdx.x - first * 32; }
  __device__ int size() const { return nw * 32; }
  __device__ bool leader() const { return rank() == 0; }
  __device__ int nwarps() const { return nw; }
  __device__ int my_warp() const { return warp_id() - first; }
  __device__ void sync() const {
    if (nw == 1) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nw * 32) : "memory");
  }
  __device__ int bcast(int v) const {
    if (nw == 1) return __shfl_sync(FULL_MASK, v, 0);
    if (leader()) red[0] = v;
    sync();
    int r = red[0];
    sync();
    return r;
  }
  // Team-wide sum / minimum: each warp reduces, then every warp reduces the
  // nw partial values with one load per lane (nw <= 32).
  __device__ int sum(int v) const {
    v = warp_sum(v);
    if (nw == 1) return v;
    if (lane_id() == 0) red[my_warp()] = v;
    sync();
    const int r = warp_sum(lane_id() < nw ? red[lane_id()] : 0);
    sync();
    return r;
  }
  __device__ int vmin(int v) const {
    v = warp_min(v);
    if (nw == 1) return v;
    if (lane_id() == 0) red[my_warp()] = v;
    sync();
    const int r = warp_min(lane_id() < nw ? red[lane_id()] : INT32_MAX);
    sync();
    return r;
  }
};

// Named barrier of the team of nw warps that starts at warp f inside a CTA
// of 16 warps: the teams form a binary tree (16 | 8,8 | 4x4 | 2x8), numbered
// 1..15 like a heap, so teams alive at the same time never share an id.
__host__ __device__ __forceinline__ int team_barrier(int f, int nw, int cta_warps) {
  return cta_warps / nw + f / nw;
}

// Shared-memory view of the points of one subproblem.
template <int D>
struct SmemPts {
  const int32_t* X;    // [D][cap]
  const uint32_t* ID;  // [cap]
  const uint8_t* flag;
  int cap;
  __device__ int32_t x(int j, int p) const { return X[j * cap + p]; }
};

// Min and max of every dimension over idx[lo, hi) (only flagged points when
// `sampled_only`).  Results are valid in every thread of the team.
template <int D>
__device__ __forceinline__ void team_minmax(const Team& tm, const SmemPts<D>& s, const uint16_t* idx, int lo, int hi,
                            bool sampled_only, int* mn, int* mx) {
  int lmn[D], lmx[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    lmn[j] = INT32_MAX;
    lmx[j] = INT32_MIN;
  }
  for (int i = lo + tm.rank(); i < hi; i += tm.size()) {
    const int p = idx[i];
    if (sampled_only && !s.flag[p]) continue;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const int v = s.x(j, p);
      lmn[j] = min(lmn[j], v);
      lmx[j] = max(lmx[j], v);
    }
  }
#pragma unroll
  for (int j = 0; j < D; ++j) {
    lmn[j] = warp_min(lmn[j]);
    lmx[j] = warp_max(lmx[j]);
  }
  if (tm.nwarps() == 1) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      mn[j] = lmn[j];
      mx[j] = lmx[j];
    }
    return;
  }
  if (lane_id() == 0) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      tm.red[tm.my_warp() * 2 * D + j] = lmn[j];
      tm.red[tm.my_warp() * 2 * D + D + j] = lmx[j];
    }
  }
  tm.sync();
#pragma unroll
  for (int j = 0; j < D; ++j) {
    int a = INT32_MAX, b = INT32_MIN;
    for (int w = 0; w < tm.nwarps(); ++w) {
      a = min(a, tm.red[w * 2 * D + j]);
      b = max(b, tm.red[w * 2 * D + D + j]);
    }
    mn[j] = a;
    mx[j] = b;
  }
  tm.sync();
}

// Widest dimension (ties: lowest); -1 when every extent is zero.  Also the
// bounds of that dimension.
template <int D>
__device__ __forceinline__ int widest_dim(const int* mn, const int* mx, int& vmin, int& vmax) {
  int best = -1;
  long long ext = 0;
  vmin = vmax = 0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const long long e = (long long)mx[j] - (long long)mn[j];
    if (e > ext) {
      ext = e;
      best = j;
      vmin = mn[j];
      vmax = mx[j];
    }
  }
  return best;
}

// Runtime-d variant for the device-wide kernels.
__device__ __forceinline__ int widest_dim_rt(const int* mn, const int* mx, int d) {
  int best = -1;
  long long ext = 0;
  for (int j = 0; j < d; ++j) {
    const long long e = (long long)mx[j] - (long long)mn[j];
    if (e > ext) {
      ext = e;
      best = j;
    }
  }
  return best;
}

// One warp scans hist[0..256): finds digit with below <= k < below+hist[digit].
__device__ __forceinline__ void warp_find_digit(const unsigned* hist, int k, int& digit, int& below,
                                                int& eq) {
  const int lane = lane_id();
  int c[8];
  int s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    c[i] = (int)hist[lane * 8 + i];
    s += c[i];
  }
  const int incl = warp_incl_scan(s);
  const int excl = incl - s;
  const unsigned hit = __ballot_sync(FULL_MASK, excl <= k && k < incl);
  const int src = hit ? __ffs(hit) - 1 : 0;
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
  digit = __shfl_sync(FULL_MASK, dg, src);
  below = __shfl_sync(FULL_MASK, bl, src);
  eq = __shfl_sync(FULL_MASK, e, src);
}

// Single-warp variant of team_select with 5-bit digits: the 32 counters are
// one per lane, so clearing them is one store and finding the digit is one
// warp scan (small subproblems are dominated by these fixed costs).
template <int D>
__device__ __forceinline__ int warp_select32(const Team& tm, const SmemPts<D>& s, const uint16_t* idx, int lo,
                                             int hi, bool sampled_only, int dim, int k, int vmin, int vmax,
                                             int& count_less, int& count_eq) {
  const int32_t* X = s.X + dim * s.cap;
  const int lane = lane_id();
  const int hb = 31 - __clz((unsigned)(vmin ^ vmax));
  unsigned mask = hb >= 31 ? 0u : ~((2u << hb) - 1u);
  unsigned prefix = (unsigned)vmin & mask;
  int less = 0, eq = 0;
  for (int top = hb; top >= 0; top -= 5) {
    const int shift = max(top - 4, 0);
    const unsigned dmask = (2u << (top - shift)) - 1u;
    tm.hist[lane] = 0;
    __syncwarp();
    for (int base = lo; base < hi; base += 32) {
      const int i = base + lane;
      int key = -1;
      if (i < hi) {
        const int p = idx[i];
        const unsigned v = (unsigned)X[p];
        if ((!sampled_only || s.flag[p]) && (v & mask) == prefix) key = (int)((v >> shift) & dmask);
      }
      if (key >= 0) atomicAdd(&tm.hist[key], 1u);
    }
    __syncwarp();
    const int c = (int)tm.hist[lane];
    const int incl = warp_incl_scan(c);
    const int excl = incl - c;
    const unsigned hit = __ballot_sync(FULL_MASK, excl <= k && k < incl);
    const int digit = hit ? __ffs(hit) - 1 : 0;
    const int below = __shfl_sync(FULL_MASK, excl, digit);
    eq = __shfl_sync(FULL_MASK, c, digit);
    __syncwarp();
    prefix |= (unsigned)digit << shift;
    mask |= dmask << shift;
    k -= below;
    less += below;
  }
  count_less = less;
  count_eq = eq;
  return (int)prefix;
}

// The element of rank k (0-based) of dimension `dim` over idx[lo, hi)
// (flagged points only when `sampled_only`), with count_less / count_eq =
// how many of those elements are below / equal to it.
//
// vmin < vmax bound the values: the bits above their highest differing bit
// are common to every element, so the 8-bit digits start just below them (a
// deep node with a narrow range needs fewer passes, and its first digit
// spreads over the bins instead of piling every element onto one counter).
// Counters are plain shared-memory atomics (lanes that hit the same bin
// serialise in hardware, which is cheaper than finding the peers first).
template <int D>
__device__ __forceinline__ int team_select(const Team& tm, const SmemPts<D>& s, const uint16_t* idx, int lo, int hi,
                           bool sampled_only, int dim, int k, int vmin, int vmax, int& count_less,
                           int& count_eq) {
  if (tm.nwarps() == 1)
    return warp_select32<D>(tm, s, idx, lo, hi, sampled_only, dim, k, vmin, vmax, count_less, count_eq);
  const int32_t* X = s.X + dim * s.cap;
  const int hb = 31 - __clz((unsigned)(vmin ^ vmax));  // highest differing bit
  unsigned mask = hb >= 31 ? 0u : ~((2u << hb) - 1u);
  unsigned prefix = (unsigned)vmin & mask;
  int less = 0, eq = 0;
  const int stride = tm.size();
  const int wbase = tm.my_warp() * 32;
  for (int top = hb; top >= 0; top -= 8) {
    const int shift = max(top - 7, 0);
    const unsigned dmask = (2u << (top - shift)) - 1u;
    for (int i = tm.rank(); i < 256; i += stride) tm.hist[i] = 0;
    tm.sync();
    for (int base = lo + wbase; base < hi; base += stride) {
      const int i = base + lane_id();
      int key = -1;
      if (i < hi) {
        const int p = idx[i];
        const unsigned v = (unsigned)X[p];
        if ((!sampled_only || s.flag[p]) && (v & mask) == prefix) key = (int)((v >> shift) & dmask);
      }
      if (key >= 0) atomicAdd(&tm.hist[key], 1u);
    }
    tm.sync();
    int digit, below, e;
    if (tm.nwarps() == 1) {
      warp_find_digit(tm.hist, k, digit, below, e);
    } else {
      if (tm.my_warp() == 0) {
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
template <int D>
__device__ __forceinline__ int team_min_above(const Team& tm, const SmemPts<D>& s, const uint16_t* idx, int lo, int hi,
                              bool sampled_only, int dim, int x) {
  int m = INT32_MAX;
  for (int i = lo + tm.rank(); i < hi; i += tm.size()) {
    const int p = idx[i];
    if (sampled_only && !s.flag[p]) continue;
    const int v = s.x(dim, p);
    if (v > x) m = min(m, v);
  }
  return tm.vmin(m);
}

// Splitter rule on the (flagged) points of idx[lo, hi): widest dimension,
// element of rank floor(count/2), or the next larger distinct value when
// nothing lies below it.  With the min/max already known (mn/mx valid), the
// min/max pass is skipped.  Returns false when the points are all identical.
template <int D>
__device__ __forceinline__ bool team_split_rule(const Team& tm, const SmemPts<D>& s, const uint16_t* idx, int lo, int hi,
                                bool sampled_only, int count, const int* mn_in, const int* mx_in, int& dim,
                                int& x) {
  int mn[D], mx[D];
  if (mn_in) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      mn[j] = mn_in[j];
      mx[j] = mx_in[j];
    }
  } else {
    team_minmax<D>(tm, s, idx, lo, hi, sampled_only, mn, mx);
  }
  int vmin, vmax;
  dim = widest_dim<D>(mn, mx, vmin, vmax);
  if (dim < 0) return false;
  int less, eq;
  x = team_select<D>(tm, s, idx, lo, hi, sampled_only, dim, count / 2, vmin, vmax, less, eq);
  if (less == 0) x = team_min_above<D>(tm, s, idx, lo, hi, sampled_only, dim, x);
  return true;
}

// Stable partition of src[lo, hi) into dst[lo, hi): points with coordinate
// `dim` below x first.  Returns the left count and the flagged counts on
// each side.
template <int D>
__device__ __forceinline__ void team_partition(const Team& tm, const SmemPts<D>& s, const uint16_t* src, uint16_t* dst,
                               int lo, int hi, int dim, int x, int& L, int& SL, int& SR) {
  const int32_t* X = s.X + dim * s.cap;
  const int n = hi - lo;
  const int nw = tm.nwarps();
  const int per = ((n + nw * 32 - 1) / (nw * 32)) * 32;
  const int w = tm.my_warp();
  const int wlo = min(hi, lo + w * per), whi = min(hi, wlo + per);
  int cl = 0, csl = 0, csr = 0;
  for (int base = wlo; base < whi; base += 32) {
    const int i = base + lane_id();
    const bool valid = i < whi;
    const int p = valid ? src[i] : 0;
    const bool left = valid && X[p] < x;
    const bool smp = valid && s.flag[p];
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
      const int c = tm.red[3 * v];
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
    const int i = base + lane_id();
    const bool valid = i < whi;
    const int p = valid ? src[i] : 0;
    const bool left = valid && X[p] < x;
    const unsigned bl = __ballot_sync(FULL_MASK, left);
    const unsigned br = __ballot_sync(FULL_MASK, valid && !left);
    if (left) dst[lbase + __popc(bl & lanemask_lt())] = (uint16_t)p;
    else if (valid) dst[rbase + __popc(br & lanemask_lt())] = (uint16_t)p;
    lbase += __popc(bl);
    rbase += __popc(br);
  }
  tm.sync();
}

// Set flag[p] = sampled(seed, depth, id, s) for idx[lo, hi); returns the count.
template <int D>
__device__ __forceinline__ int team_draw_sample(const Team& tm, const SmemPts<D>& s, uint8_t* flag, const uint16_t* idx,
                                int lo, int hi, uint64_t seed, uint32_t depth, int shift) {
  int c = 0;
  for (int i = lo + tm.rank(); i < hi; i += tm.size()) {
    const int p = idx[i];
    const bool f = in_sample(seed, depth, s.ID[p], shift);
    flag[p] = f;
    c += f;
  }
  tm.sync();
  return tm.sum(c);
}

// Clear the flags of idx[lo, hi) (a Build root too small to reach the
// sampling threshold draws no sample).
__device__ __forceinline__ void team_clear_flags(const Team& tm, uint8_t* flag, const uint16_t* idx, int lo,
                                                 int hi) {
  for (int i = lo + tm.rank(); i < hi; i += tm.size()) flag[idx[i]] = 0;
  tm.sync();
}

}  // namespace pkd
