// Sieve machinery shared by the build and the batch updates: point sources,
// device-wide scans, per-round arguments, and the count / scatter kernels
// that move every point of a subproblem to its bucket of a heap skeleton.
#pragma once

#include <algorithm>
#include <vector>

#include "engine.hpp"
#include "smem_build.cuh"

namespace pkd {

constexpr uint32_t SEG_SKIP = 0xFFFFFFFFu;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_TILE = SCAN_ITEMS * SCAN_THREADS;
constexpr int JOB_TILE = 2048;
constexpr int JOB_THREADS = 256;
constexpr int SIEVE_THREADS = 1024;
constexpr int SIEVE_PER = 4;  // points per thread: TILE <= SIEVE_PER * SIEVE_THREADS

struct Src {
  Pts soa;
  const int32_t* aos;
  const uint32_t* aos_ids;
  int is_aos;
  __device__ __forceinline__ int32_t x(int d, int j, uint64_t g) const {
    return is_aos ? aos[g * (uint64_t)d + j] : soa.c[(uint64_t)j * soa.stride + g];
  }
  __device__ __forceinline__ uint32_t id(uint64_t g) const {
    return is_aos ? (aos_ids ? aos_ids[g] : (uint32_t)g) : soa.id[g];
  }
};

// Exclusive block scan of one value per thread; returns the prefix, *total.
template <class V>
__device__ V block_excl_scan(V v, V* sh, V* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  V incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    V t = __shfl_up_sync(FULL_MASK, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) sh[w] = incl;
  __syncthreads();
  if (w == 0) {
    V s = lane < nw ? sh[lane] : V(0);
    V si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      V t = __shfl_up_sync(FULL_MASK, si, o);
      if (lane >= o) si += t;
    }
    if (lane < nw) sh[lane] = si - s;
    if (lane == 31) sh[32] = si;
  }
  __syncthreads();
  V r = sh[w] + incl - v;
  *total = sh[32];
  __syncthreads();
  return r;
}

// Block-wide reservation in K lists, one atomic per list and block: thread
// t asks c[k] entries of list k (length counter ctr[k]) and receives the
// index of its first one in first[k].  Appending to a list through one
// counter serialises at that counter's address, so the fewer updates the
// better.  Every thread of the block calls it (c = 0 when it adds nothing).
template <int K>
__device__ __forceinline__ void block_reserve(const uint32_t (&c)[K], uint32_t* const (&ctr)[K],
                                              uint32_t (&first)[K]) {
  __shared__ uint32_t part[K][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t incl[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    incl[k] = c[k];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(FULL_MASK, incl[k], o);
      if (lane >= o) incl[k] += t;
    }
    if (lane == 31) part[k][w] = incl[k];
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint32_t v = lane < nw ? part[k][lane] : 0u;
      uint32_t s = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL_MASK, s, o);
        if (lane >= o) s += t;
      }
      if (lane < nw) part[k][lane] = s - v;
      const uint32_t tot = __shfl_sync(FULL_MASK, s, 31);
      if (lane == 0) part[k][32] = tot ? atomicAdd(ctr[k], tot) : 0u;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) first[k] = part[k][32] + part[k][w] + incl[k] - c[k];
  __syncthreads();  // part is rewritten by the next call
}

// Block-wide 64-bit sums added to K counters, one atomic per counter and
// block.  Every thread of the block calls it.
template <int K>
__device__ __forceinline__ void block_add64(const unsigned long long (&v)[K], unsigned long long* const (&ctr)[K]) {
  __shared__ unsigned long long part64[K][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    unsigned long long s = v[k];
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o);
    if (lane == 0) part64[k][w] = s;
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      unsigned long long s = lane < nw ? part64[k][lane] : 0ull;
#pragma unroll
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o);
      if (lane == 0 && s) atomicAdd(ctr[k], s);
    }
  }
  __syncthreads();
}

// Per-block sums of in[0, n).
static __global__ void k_scan_reduce(const uint32_t* in, uint64_t n, uint32_t* partial) {
  __shared__ uint32_t sh[33];
  uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
  uint32_t s = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    uint64_t i = base + (uint64_t)threadIdx.x * SCAN_ITEMS + k;
    if (i < n) s += in[i];
  }
  uint32_t tot;
  block_excl_scan<uint32_t>(s, sh, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// Single-block exclusive scan in place over x[0, n).
static __global__ void k_scan_single(uint32_t* x, uint64_t n) {
  __shared__ uint32_t sh[33];
  uint32_t carry = 0;
  for (uint64_t base = 0; base < n; base += blockDim.x) {
    uint64_t i = base + threadIdx.x;
    uint32_t v = i < n ? x[i] : 0;
    uint32_t tot;
    uint32_t e = block_excl_scan<uint32_t>(v, sh, &tot);
    if (i < n) x[i] = carry + e;
    carry += tot;
  }
}

static __global__ void k_scan_apply(const uint32_t* in, uint32_t* out, uint64_t n, const uint32_t* partial) {
  __shared__ uint32_t sh[33];
  uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  uint32_t tot;
  uint32_t e = block_excl_scan<uint32_t>(s, sh, &tot) + partial[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k < n) out[base + k] = e;
    e += v[k];
  }
}

static void device_excl_scan(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* partial,
                             cudaStream_t s) {
  if (n == 0) return;
  const uint64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  PKD_LAUNCH(k_scan_reduce<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, partial));
  PKD_LAUNCH(k_scan_single<<<1, 1024, 0, s>>>(partial, nb));
  PKD_LAUNCH(k_scan_apply<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, partial));
}

// The same scan over n = min(nmax, *n_dev * mult) elements, a length only
// the device knows: a fixed grid of SCAN_BLOCKS blocks, each over a
// contiguous run of SCAN_TILE pieces (partial needs SCAN_BLOCKS words).
constexpr int SCAN_BLOCKS = 256;

__device__ __forceinline__ void scan_dev_range(const uint32_t* n_dev, uint32_t mult, uint64_t nmax, uint64_t& n,
                                               uint64_t& t0, uint64_t& t1) {
  n = min(nmax, (uint64_t)*n_dev * mult);
  const uint64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  const uint64_t per = (tiles + gridDim.x - 1) / gridDim.x;
  t0 = min(tiles, (uint64_t)blockIdx.x * per);
  t1 = min(tiles, t0 + per);
}

static __global__ void k_scan_reduce_dev(const uint32_t* in, const uint32_t* n_dev, uint32_t mult, uint64_t nmax,
                                         uint32_t* partial) {
  __shared__ uint32_t sh[33];
  uint64_t n, t0, t1;
  scan_dev_range(n_dev, mult, nmax, n, t0, t1);
  uint32_t s = 0;
  for (uint64_t i = t0 * SCAN_TILE + threadIdx.x; i < min(n, t1 * SCAN_TILE); i += SCAN_THREADS) s += in[i];
  uint32_t tot;
  block_excl_scan<uint32_t>(s, sh, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

static __global__ void k_scan_apply_dev(const uint32_t* in, uint32_t* out, const uint32_t* n_dev, uint32_t mult,
                                        uint64_t nmax, const uint32_t* partial) {
  __shared__ uint32_t sh[33];
  uint64_t n, t0, t1;
  scan_dev_range(n_dev, mult, nmax, n, t0, t1);
  uint32_t carry = partial[blockIdx.x];
  for (uint64_t t = t0; t < t1; ++t) {
    const uint64_t base = t * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
      v[k] = (base + k < n) ? in[base + k] : 0;
      s += v[k];
    }
    uint32_t tot;
    uint32_t e = block_excl_scan<uint32_t>(s, sh, &tot) + carry;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
      if (base + k < n) out[base + k] = e;
      e += v[k];
    }
    carry += tot;
  }
}

static void device_excl_scan_dev(const uint32_t* in, uint32_t* out, const uint32_t* n_dev, uint32_t mult,
                                 uint64_t nmax, uint32_t* partial, cudaStream_t s) {
  PKD_LAUNCH(k_scan_reduce_dev<<<SCAN_BLOCKS, SCAN_THREADS, 0, s>>>(in, n_dev, mult, nmax, partial));
  PKD_LAUNCH(k_scan_single<<<1, 1024, 0, s>>>(partial, SCAN_BLOCKS));
  PKD_LAUNCH(k_scan_apply_dev<<<SCAN_BLOCKS, SCAN_THREADS, 0, s>>>(in, out, n_dev, mult, nmax, partial));
}

// Streaming multiprocessors of the current device.
static inline int sm_count() {
  static int v = -1;
  if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) v = 1;
  }
  return v;
}

struct RoundDyn;

struct RoundArgs {
  Params p;
  int lam, NB, HN, TILE;
  Src src;
  Pts dst;
  Pts A;
  int dst_where;
  const Seg* big;
  const uint32_t* nbig;
  uint32_t* tile0;   // [nbig] first tile of each big segment
  uint64_t* excl;    // [nbig] points of the big segments before this one
  int2* skel;        // [nbig][HN]
  const uint32_t* skel_map;  // optional: big segment -> row of skel
  uint32_t* slots;   // [nbig][HN]
  uint32_t* nbk;     // [nbig] buckets
  uint8_t* exact;    // [nbig] 1: exact level on the points; 2: already handled
  uint32_t* hist;    // [tiles * NB]
  uint32_t* hscan;
  uint8_t* bkt;      // optional [tiles][TILE]: every point's bucket, written by
                     // the streaming count and read by the streaming scatter
                     // (NB <= 256), which then need not walk the skeleton again
  uint32_t* scnt;    // [nbig] samples
  uint32_t* sizes;   // [nbig][HN] skeleton subtree sizes
  Pts samp;          // sample buffer 0
  Seg* children;     // [nbig * NB]
  Node* nodes;
  uint8_t* ndim;
  uint32_t* shared_next;
  uint64_t shared_cap;
  DevStatus* st;
  long long wait_cycles;  // limit of a streaming kernel's waits (clock cycles)
  // rounds decided on the device: the round's entry of dyn (selected by
  // *sel) replaces src, dst, dst_where and children, and the tile count of
  // the round is *ntiles (null: the launch's own count)
  const RoundDyn* dyn;
  const uint32_t* sel;
  const uint32_t* ntiles;
};

// The per-round part of a build's arguments when its rounds are decided on
// the device: one entry for the first round, one for the odd rounds and one
// for the even rounds after the first (the point buffers alternate).
struct RoundDyn {
  Src src;
  Pts dst;
  int dst_where, src_where;
  const Seg* cur;  // segments of the round
  Seg* children;   // [big segments * NB] buckets of the round
};

__device__ __forceinline__ RoundArgs with_dyn(const RoundArgs& r0) {
  RoundArgs r = r0;
  if (r0.dyn) {
    const RoundDyn& d = r0.dyn[*r0.sel];
    r.src = d.src;
    r.dst = d.dst;
    r.dst_where = d.dst_where;
    r.children = d.children;
  }
  return r;
}

// The round's source and destination alone (hot kernels: no struct copy).
__device__ __forceinline__ Src round_src(const RoundArgs& r) { return r.dyn ? r.dyn[*r.sel].src : r.src; }
__device__ __forceinline__ Pts round_dst(const RoundArgs& r) { return r.dyn ? r.dyn[*r.sel].dst : r.dst; }

// Tiles of the round: the device count when there is one, else `host`.
__device__ __forceinline__ uint32_t round_tiles(const RoundArgs& r, uint32_t host) {
  return r.ntiles ? *r.ntiles : host;
}

__device__ __forceinline__ uint32_t seg_of_tile(const uint32_t* tile0, uint32_t nseg, uint32_t tile) {
  uint32_t lo = 0, hi = nseg;  // largest s with tile0[s] <= tile
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (tile0[mid] <= tile) lo = mid;
    else hi = mid;
  }
  return lo;
}

// tile0 / excl over the big segments (one block).
static __global__ void k_big_prefix(const Seg* big, const uint32_t* nbig, uint32_t tile, uint32_t* tile0,
                             uint64_t* excl) {
  __shared__ uint32_t sh32[33];
  __shared__ unsigned long long sh64[33];
  const uint32_t n = *nbig;
  uint32_t ct = 0;
  unsigned long long cl = 0;
  for (uint32_t base = 0; base < n; base += blockDim.x) {
    uint32_t i = base + threadIdx.x;
    uint32_t t = 0;
    unsigned long long l = 0;
    if (i < n) {
      t = (big[i].len + tile - 1) / tile;
      l = big[i].len;
    }
    uint32_t tt;
    unsigned long long tl;
    uint32_t et = block_excl_scan<uint32_t>(t, sh32, &tt);
    unsigned long long el = block_excl_scan<unsigned long long>(l, sh64, &tl);
    if (i < n) {
      tile0[i] = ct + et;
      excl[i] = cl + el;
    }
    ct += tt;
    cl += tl;
  }
}

struct SieveTile {
  uint32_t s;
  Seg seg;
  uint64_t first;
  int cnt;
  uint32_t t0, nt;
};

__device__ __forceinline__ bool sieve_tile(const RoundArgs& r, SieveTile& t, uint32_t tile) {
  const uint32_t nb = *r.nbig;
  t.s = seg_of_tile(r.tile0, nb, tile);
  t.seg = r.big[t.s];
  t.t0 = r.tile0[t.s];
  t.nt = (t.seg.len + r.TILE - 1) / r.TILE;
  t.first = (uint64_t)(tile - t.t0) * r.TILE;
  if (t.first >= t.seg.len) return false;
  t.cnt = (int)min((uint64_t)r.TILE, (uint64_t)t.seg.len - t.first);
  return true;
}

// Walk the heap skeleton held in shared memory (split, meta) to a bucket.
template <int D>
__device__ __forceinline__ int walk_bucket(const int2* sk, const int32_t* x, int lam) {
  int h = 1;
  for (int l = 0; l < lam; ++l) {
    const int2 e = sk[h];
    if (sk_state(e.y) != SK_INTERNAL) break;
    h = 2 * h + (x[sk_dim(e.y)] >= e.x);
  }
  return sk_bucket(sk[h].y);
}

template <int D>
__device__ __forceinline__ void count_tile(const RoundArgs& r, uint32_t tile) {
  SieveTile t;
  if (!sieve_tile(r, t, tile)) return;
  extern __shared__ __align__(16) uint8_t sm[];
  int2* sk = (int2*)sm;
  unsigned* lh = (unsigned*)(sk + r.HN);
  const int2* gsk = r.skel + (uint64_t)(r.skel_map ? r.skel_map[t.s] : t.s) * r.HN;
  for (int v = threadIdx.x; v < r.HN; v += blockDim.x) sk[v] = gsk[v];
  for (int b = threadIdx.x; b < r.NB; b += blockDim.x) lh[b] = 0;
  __syncthreads();
  const bool heavy = sk_state(sk[1].y) == SK_HEAVY;
  if (!heavy) {
    // all of this thread's loads first, then the walks (loads stay in flight)
    int32_t x[SIEVE_PER][D];
#pragma unroll
    for (int k = 0; k < SIEVE_PER; ++k) {
      const int i = k * SIEVE_THREADS + threadIdx.x;
      if (i < t.cnt) {
        const uint64_t g = t.seg.start + t.first + i;
#pragma unroll
        for (int j = 0; j < D; ++j) x[k][j] = r.src.x(D, j, g);
      }
    }
#pragma unroll
    for (int k = 0; k < SIEVE_PER; ++k) {
      const int i = k * SIEVE_THREADS + threadIdx.x;
      const int b = i < t.cnt ? walk_bucket<D>(sk, x[k], r.lam) : -1;
      if (b >= 0) atomicAdd(&lh[b], 1u);
    }
  }
  __syncthreads();
  const uint64_t hb = (uint64_t)t.t0 * r.NB;
  const uint32_t tl = tile - t.t0;
  for (int b = threadIdx.x; b < r.NB; b += blockDim.x) r.hist[hb + (uint64_t)b * t.nt + tl] = lh[b];
}

// One tile a block at a time (the grid strides over the round's tiles).
template <int D>
__global__ void __launch_bounds__(SIEVE_THREADS) k_count(RoundArgs r0) {
  const RoundArgs r = with_dyn(r0);
  const uint32_t nt = round_tiles(r, gridDim.x);
  for (uint32_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    count_tile<D>(r, tile);
    __syncthreads();
  }
}

template <int D>
__device__ __forceinline__ void scatter_tile(const RoundArgs& r, uint32_t tile) {
  SieveTile t;
  if (!sieve_tile(r, t, tile)) return;
  extern __shared__ __align__(16) uint8_t sm[];
  int2* sk = (int2*)sm;
  unsigned* cur = (unsigned*)(sk + r.HN);      // [NB] per-bucket counters, then starts
  unsigned* lstart = cur + r.NB;               // [NB]
  uint32_t* gbase = lstart + r.NB;             // [NB] (relative to the segment start)
  int32_t* stx = (int32_t*)(gbase + r.NB);     // [D][TILE]
  uint32_t* sid = (uint32_t*)(stx + (size_t)D * r.TILE);
  uint16_t* sb = (uint16_t*)(sid + r.TILE);
  const int2* gsk = r.skel + (uint64_t)(r.skel_map ? r.skel_map[t.s] : t.s) * r.HN;
  for (int v = threadIdx.x; v < r.HN; v += blockDim.x) sk[v] = gsk[v];
  for (int b = threadIdx.x; b < r.NB; b += blockDim.x) cur[b] = 0;
  __syncthreads();
  if (sk_state(sk[1].y) == SK_HEAVY) return;
  constexpr int PER = SIEVE_PER;
  int32_t x[PER][D];
  uint32_t id[PER];
  int bk[PER], rk[PER];
  // all of this thread's loads first, then the walks (loads stay in flight)
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int i = k * SIEVE_THREADS + threadIdx.x;
    if (i < t.cnt) {
      const uint64_t g = t.seg.start + t.first + i;
#pragma unroll
      for (int j = 0; j < D; ++j) x[k][j] = r.src.x(D, j, g);
      id[k] = r.src.id(g);
    }
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int i = k * SIEVE_THREADS + threadIdx.x;
    bk[k] = i < t.cnt ? walk_bucket<D>(sk, x[k], r.lam) : -1;
    const unsigned m = peer_mask(bk[k], r.lam);
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (bk[k] >= 0 && lane_id() == leader) base = atomicAdd(&cur[bk[k]], (unsigned)__popc(m));
    base = __shfl_sync(FULL_MASK, base, leader);
    rk[k] = (int)base + __popc(m & lanemask_lt());
  }
  __syncthreads();
  // bucket starts inside the tile, and global bases from the scan
  if (threadIdx.x < 32) {
    unsigned carry = 0;
    for (int b0 = 0; b0 < r.NB; b0 += 32) {
      const int b = b0 + lane_id();
      const unsigned c = b < r.NB ? cur[b] : 0;
      const unsigned incl = (unsigned)warp_incl_scan((int)c);
      if (b < r.NB) lstart[b] = carry + incl - c;
      carry += __shfl_sync(FULL_MASK, incl, 31);
    }
  }
  const uint64_t hb = (uint64_t)t.t0 * r.NB;
  const uint32_t tl = tile - t.t0;
  const uint32_t segbase = r.hscan[hb];
  for (int b = threadIdx.x; b < r.NB; b += blockDim.x)
    gbase[b] = r.hscan[hb + (uint64_t)b * t.nt + tl] - segbase;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    if (bk[k] >= 0) {
      const int pos = (int)lstart[bk[k]] + rk[k];
#pragma unroll
      for (int j = 0; j < D; ++j) stx[j * r.TILE + pos] = x[k][j];
      sid[pos] = id[k];
      sb[pos] = (uint16_t)bk[k];
    }
  }
  __syncthreads();
  // every bucket's run leaves the tile as one contiguous, coalesced range
  for (int pos = threadIdx.x; pos < t.cnt; pos += blockDim.x) {
    const int b = sb[pos];
    const uint64_t g = t.seg.start + gbase[b] + (uint64_t)(pos - (int)lstart[b]);
#pragma unroll
    for (int j = 0; j < D; ++j) r.dst.c[(uint64_t)j * r.dst.stride + g] = stx[j * r.TILE + pos];
    r.dst.id[g] = sid[pos];
  }
}

template <int D>
__global__ void __launch_bounds__(SIEVE_THREADS) k_scatter(RoundArgs r0) {
  if (pkd_failed_block(r0.st)) return;
  const RoundArgs r = with_dyn(r0);
  const uint32_t nt = round_tiles(r, gridDim.x);
  for (uint32_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    scatter_tile<D>(r, tile);
    __syncthreads();
  }
}

static size_t scatter_smem(int HN, int NB, int D, int tile) {
  return (size_t)HN * 8 + (size_t)NB * 12 + (size_t)D * tile * 4 + (size_t)tile * 4 + (size_t)tile * 2;
}

template <int D>
static void launch_count_tiles(const RoundArgs& r, uint32_t tiles, uint64_t pts, const char* fam, cudaStream_t s) {
  const size_t sm = (size_t)r.HN * 8 + (size_t)r.NB * 4;
  // with a device tile count, `tiles` is only a bound: a grid of resident blocks strides over the tiles
  const uint32_t grid = r.ntiles ? std::min<uint32_t>(tiles, (uint32_t)sm_count() * 2) : tiles;
  KTimer kt;
  ktimer_begin(kt, fam, pts, s);
  PKD_LAUNCH(k_count<D><<<grid, SIEVE_THREADS, sm, s>>>(r));
  ktimer_end(kt);
}

template <int D>
static void launch_scatter_tiles(const RoundArgs& r, uint32_t tiles, uint64_t pts, const char* fam,
                                 cudaStream_t s) {
  const size_t sm = scatter_smem(r.HN, r.NB, D, r.TILE);
  static bool set = false;
  if (!set) {
    cudaFuncSetAttribute(k_scatter<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    set = true;
  }
  const uint32_t grid = r.ntiles ? std::min<uint32_t>(tiles, (uint32_t)sm_count() * 2) : tiles;
  KTimer kt;
  ktimer_begin(kt, fam, pts, s);
  PKD_LAUNCH(k_scatter<D><<<grid, SIEVE_THREADS, sm, s>>>(r));
  ktimer_end(kt);
}

#define PKD_DISPATCH_D(d, F, ...) \
  switch (d) {                    \
    case 1: F<1>(__VA_ARGS__); break; \
    case 2: F<2>(__VA_ARGS__); break; \
    case 3: F<3>(__VA_ARGS__); break; \
    case 4: F<4>(__VA_ARGS__); break; \
    case 5: F<5>(__VA_ARGS__); break; \
    case 6: F<6>(__VA_ARGS__); break; \
    case 7: F<7>(__VA_ARGS__); break; \
    default: F<8>(__VA_ARGS__); break; \
  }

// Shift a structure-of-arrays view so that absolute arena positions index
// into a scratch allocation that only covers [base, base + extent).
static Pts shifted(const Pts& p, uint64_t base) {
  Pts q = p;
  q.c = p.c - base;
  q.id = p.id - base;
  return q;
}

struct Scratch {
  cudaStream_t s;
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  template <class T>
  int get(T** p, size_t n) {
    int e = dalloc(p, n, s);
    if (e == PKD_OK) ptrs.push_back(*p);
    return e;
  }
};

#define PKD_TRY(x)               \
  do {                           \
    int _r = (x);                \
    if (_r != PKD_OK) return _r; \
  } while (0)

}  // namespace pkd
