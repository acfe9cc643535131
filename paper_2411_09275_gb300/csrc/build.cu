// Pkd-tree construction on the GPU (Alg. 1 of "Parallel kd-tree with Batch
// Updates"), for a set of independent subproblems at once.
//
// A subproblem larger than one CTA's shared memory takes a global round:
//   sample    points whose hash passes the rate test at the subproblem's depth
//   skeleton  lambda levels of exact medians on the sample: device-wide radix
//             select while a skeleton node's sample exceeds one CTA, then one
//             CTA per node in shared memory
//   count     every point walks the skeleton (splitters in shared memory) to
//             its bucket; per-tile bucket histograms (warp-aggregated)
//   scan      bucket-major ("column-major") exclusive prefix sum of the
//             histograms = write offset of every (tile, bucket)
//   scatter   the tile is staged in shared memory in bucket order and every
//             bucket's run is written contiguously into the other buffer
//             (the two buffers swap each round instead of copying back, Sec. 5)
//   emit      skeleton nodes become tree nodes; every bucket becomes a child
//             subproblem at depth + its skeleton depth
// A subproblem that fits in shared memory is finished by one CTA
// (smem_build.cuh).  When a skeleton root is a bucket (too few or identical
// samples) the subproblem takes one exact level on its own points; when its
// points are all identical it becomes one heavy leaf.
#include <map>
#include <mutex>
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "sieve_tma.cuh"
#include "smem_sorted.cuh"

namespace pkd {


// ---------------------------------------------------------------------------
// Point sources
// ---------------------------------------------------------------------------


// ---------------------------------------------------------------------------
// Shared-memory kernels (build mode and skeleton mode)
// ---------------------------------------------------------------------------

struct SmemPtrs {
  int32_t* X;
  uint32_t* ID;
  uint16_t* perm0;
  uint16_t* perm1;
  uint8_t* flag;
  unsigned* whist;
  int* wred;
  Task* wstack;
  SmemCtl* ctl;
};

__device__ SmemPtrs carve(uint8_t* sm, int cap, int d) {
  const SmemLayout Lo = smem_layout(cap, d);
  SmemPtrs q;
  q.X = (int32_t*)(sm + Lo.X);
  q.ID = (uint32_t*)(sm + Lo.ID);
  q.perm0 = (uint16_t*)(sm + Lo.perm0);
  q.perm1 = (uint16_t*)(sm + Lo.perm1);
  q.flag = (uint8_t*)(sm + Lo.flag);
  q.whist = (unsigned*)(sm + Lo.whist);
  q.wred = (int*)(sm + Lo.wred);
  q.wstack = (Task*)(sm + Lo.wstack);
  q.ctl = (SmemCtl*)(sm + Lo.ctl);
  return q;
}

template <int D>
__device__ SmemCtx<D> make_ctx(const SmemArgs& a, const SmemPtrs& q, int cap) {
  SmemCtx<D> cx;
  cx.p = a.p;
  cx.s = SmemPts<D>{q.X, q.ID, q.flag, cap};
  cx.flag = q.flag;
  cx.perm[0] = q.perm0;
  cx.perm[1] = q.perm1;
  cx.ctl = q.ctl;
  cx.out = a.A;
  cx.start = 0;
  cx.slot_base = 0;
  cx.slot_limit = 0;
  cx.nodes = a.nodes;
  cx.ndim = a.ndim;
  cx.skel = nullptr;
  cx.lam = 0;
  cx.min_split = 0;
  cx.st = a.st;
  return cx;
}

// Load the points of a segment into shared memory (coordinates per
// dimension, ids) and set the identity index list.
template <int D>
__device__ void load_segment(const SmemArgs& a, const Seg& seg, int32_t* X, uint32_t* ID, uint16_t* perm,
                             int cap, int rank, int stride) {
  const int n = (int)seg.len;
  for (int i = rank; i < n; i += stride) {
    const uint64_t g = seg.start + (uint64_t)i;
    if (seg.where == IN_INPUT) {
#pragma unroll
      for (int j = 0; j < D; ++j) X[j * cap + i] = a.in_coords[g * (uint64_t)D + j];
      ID[i] = a.in_ids ? a.in_ids[g] : (uint32_t)g;
    } else {
      const Pts& S = seg.where == IN_A ? a.A : a.B;
#pragma unroll
      for (int j = 0; j < D; ++j) X[j * cap + i] = S.c[(uint64_t)j * S.stride + g];
      ID[i] = S.id[g];
    }
    perm[i] = (uint16_t)i;
  }
}

template <int D>
__global__ void __launch_bounds__(SM_THREADS, 1) k_smem_build(SmemArgs a) {
  if (blockIdx.x >= *a.nsegs) return;
  extern __shared__ __align__(16) uint8_t sm[];
  const Seg seg = a.segs[blockIdx.x];
  const int cap = a.cap, tid = threadIdx.x;
  SmemPtrs q = carve(sm, cap, D);
  if (seg.len > (uint32_t)cap) {
    if (tid == 0) set_error(a.st, DERR_CAPACITY, (int)blockIdx.x);
    return;
  }
  const int n = (int)seg.len;
  load_segment<D>(a, seg, q.X, q.ID, q.perm0, cap, tid, SM_THREADS);
  if (tid == 0) {
    q.ctl->next_slot = 0;
    q.ctl->maxd = 0;
  }
  if (tid < SM_NW) q.ctl->wsp[tid] = 0;
  __syncthreads();
  if (n == 0) {
    if (tid == 0) {
      a.nodes[seg.root] = Node{0, 0, (uint32_t)seg.start, 0};
      a.ndim[seg.root] = PKD_LEAF;
    }
    return;
  }
  SmemCtx<D> cx = make_ctx<D>(a, q, cap);
  cx.start = seg.start;
  cx.slot_base = (uint32_t)(a.shared_cap + 2 * seg.start);
  cx.slot_limit = 2 * n;
  Task root{0, (uint16_t)n, 0, 0, 0, seg.depth, seg.root};
  run_team_tasks<false, D>(cx, root, q.whist, q.wred, q.wstack, SM_NW);
  __syncthreads();
  if (tid == 0) atomicMax(&a.st->max_depth, q.ctl->maxd);
}

// The base case on presorted lists (one CTA per segment of at most cap
// points): load, sort every dimension once, then split by lookups and stable
// list partitions.  Instantiated for one CTA per SM (the largest capacity)
// and for two (half the shared memory and at most 64 registers a thread);
// the segment lists of the two launches are separated when the segments are
// classified.
template <int D, int MINB>
__global__ void __launch_bounds__(SS_THREADS, MINB) k_smem_sorted(SmemArgs a) {
  if (blockIdx.x >= *a.nsegs) return;
  extern __shared__ __align__(16) uint8_t sm[];
  const Seg seg = a.segs[blockIdx.x];
  const int cap = a.cap, tid = threadIdx.x;
  const SortedLayout Lo = sorted_layout(cap, D);
  int32_t* X = (int32_t*)(sm + Lo.X);
  uint32_t* ID = (uint32_t*)(sm + Lo.ID);
  int* sred = (int*)(sm + Lo.red);
  STask* wstack = (STask*)(sm + Lo.stack);
  SmemCtl* ctl = (SmemCtl*)(sm + Lo.ctl);
  if (seg.len > (uint32_t)cap) {
    if (tid == 0) set_error(a.st, DERR_CAPACITY, 400000 + (int)blockIdx.x);
    return;
  }
  const int n = (int)seg.len;
  if (n == 0) {
    if (tid == 0) {
      a.nodes[seg.root] = Node{0, 0, (uint32_t)seg.start, 0};
      a.ndim[seg.root] = PKD_LEAF;
    }
    return;
  }
  if (tid < D) {
    sred[tid] = INT32_MAX;
    sred[D + tid] = INT32_MIN;
  }
  if (tid == 0) {
    ctl->next_slot = 0;
    ctl->maxd = 0;
  }
  if (tid < SS_NW) ctl->wsp[tid] = 0;
  __syncthreads();
  int lmn[D], lmx[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    lmn[j] = INT32_MAX;
    lmx[j] = INT32_MIN;
  }
  // four points per thread in flight: every load of a batch before its stores
  constexpr int LU = 4;
  // the segment's arrays, offset once (32-bit indexing below)
  const bool aos = seg.where == IN_INPUT;
  const Pts& S = seg.where == IN_A ? a.A : a.B;
  const int32_t* src_c[D];
#pragma unroll
  for (int j = 0; j < D; ++j)
    src_c[j] = aos ? a.in_coords + seg.start * (uint64_t)D + j : S.c + (uint64_t)j * S.stride + seg.start;
  const uint32_t* src_id = aos ? (a.in_ids ? a.in_ids + seg.start : nullptr) : S.id + seg.start;
  const int cstep = aos ? D : 1;
  for (int i0 = tid; i0 < n; i0 += LU * SS_THREADS) {
    int32_t v[LU][D];
    uint32_t id[LU];
#pragma unroll
    for (int u = 0; u < LU; ++u) {
      const int i = i0 + u * SS_THREADS;
      if (i < n) {
#pragma unroll
        for (int j = 0; j < D; ++j) v[u][j] = src_c[j][i * cstep];
        id[u] = src_id ? src_id[i] : (uint32_t)(seg.start + (uint64_t)i);
      }
    }
#pragma unroll
    for (int u = 0; u < LU; ++u) {
      const int i = i0 + u * SS_THREADS;
      if (i < n) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
          X[j * cap + i] = v[u][j];
          lmn[j] = min(lmn[j], v[u][j]);
          lmx[j] = max(lmx[j], v[u][j]);
        }
        ID[i] = id[u];
      }
    }
  }
#pragma unroll
  for (int j = 0; j < D; ++j) {
    lmn[j] = warp_min(lmn[j]);
    lmx[j] = warp_max(lmx[j]);
  }
  if (lane_id() == 0) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      atomicMin(&sred[j], lmn[j]);
      atomicMax(&sred[D + j], lmx[j]);
    }
  }
  __syncthreads();
  int vmn[D], vmx[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    vmn[j] = sred[j];
    vmx[j] = sred[D + j];
  }
  __syncthreads();
  SCtx<D> cx;
  cx.p = a.p;
  cx.X = X;
  cx.ID = ID;
  cx.flag = sm + Lo.flag;
  cx.lists = (uint16_t*)(sm + Lo.lists);
  cx.cap = cap;
  cx.ctl = ctl;
  cx.out = a.A;
  cx.start = seg.start;
  cx.slot_base = (uint32_t)(a.shared_cap + 2 * seg.start);
  cx.slot_limit = 2 * n;
  cx.nodes = a.nodes;
  cx.ndim = a.ndim;
  cx.st = a.st;
  unsigned* hist = (unsigned*)wstack;  // the task stacks are not in use yet
#pragma unroll 1
  for (int k = 0; k < D; ++k)
    if (!presort_dim_msd<D>(cx, k, vmn[k], vmx[k], n, hist, sred + 2 * D))
      presort_dim<D>(cx, k, vmn[k], vmx[k], n, hist, sred + 2 * D);
  uint32_t map = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) map |= (uint32_t)k << (4 * k);
  srun_tasks<D>(cx, STask{0, (uint16_t)n, 0, 0, 0, seg.depth, seg.root, map, 0}, sred, wstack);
  __syncthreads();
  // every leaf left its points' indices in list 0: write the subproblem out
  // in leaf order, coalesced
  {
    const uint16_t* P = cx.list(0);
    int32_t* oc[D];
#pragma unroll
    for (int j = 0; j < D; ++j) oc[j] = a.A.c + (uint64_t)j * a.A.stride + seg.start;
    uint32_t* oid = a.A.id + seg.start;
    for (int i = tid; i < n; i += SS_THREADS) {
      const int p = P[i];
      if (p >= n) continue;  // only after a recorded error, when leaves are missing
#pragma unroll
      for (int j = 0; j < D; ++j) oc[j][i] = X[j * cap + p];
      oid[i] = ID[p];
    }
  }
  if (tid == 0) atomicMax(&a.st->max_depth, ctl->maxd);
}

template <int D>
__global__ void __launch_bounds__(SM_THREADS, 1) k_smem_skel(SmemArgs a) {
  if (blockIdx.x >= *a.njobs) return;
  extern __shared__ __align__(16) uint8_t sm[];
  const SkelJob jb = a.jobs[blockIdx.x];
  const int cap = a.cap, tid = threadIdx.x;
  SmemPtrs q = carve(sm, cap, D);
  if (jb.n > (uint32_t)cap) {
    if (tid == 0) set_error(a.st, DERR_CAPACITY, 200000 + (int)blockIdx.x);
    return;
  }
  const int n = (int)jb.n;
  const int32_t* S = a.sbuf[jb.buf];
  for (int i = tid; i < n; i += SM_THREADS) {
#pragma unroll
    for (int j = 0; j < D; ++j) q.X[j * cap + i] = S[(uint64_t)j * a.sstride + jb.a + i];
    q.ID[i] = 0;
    q.flag[i] = 0;
    q.perm0[i] = (uint16_t)i;
  }
  if (tid < SM_NW) q.ctl->wsp[tid] = 0;
  __syncthreads();
  SmemCtx<D> cx = make_ctx<D>(a, q, cap);
  cx.skel = a.skel + (uint64_t)jb.seg * a.heap_n;
  cx.lam = jb.lam;
  cx.min_split = (int)jb.min_split;
  Task root{0, (uint16_t)n, 0, 0, jb.j, 0, jb.h};
  run_team_tasks<true, D>(cx, root, q.whist, q.wred, q.wstack, SM_NW);
}

// One warp per small subproblem (a leaf rebuilt with a few new points, or a
// small bucket): every warp of the CTA owns its own shared-memory slice.
constexpr int WK_WARPS = 8;

struct WarpLayout {
  size_t X, ID, perm0, perm1, flag, hist, stack, ctl, per_warp;
};

__host__ __device__ inline WarpLayout warp_layout(int wcap, int d) {
  WarpLayout L;
  size_t o = 0;
  L.X = o;
  o = align_up(o + (size_t)4 * d * wcap, 16);
  L.ID = o;
  o = align_up(o + (size_t)4 * wcap, 16);
  L.perm0 = o;
  o = align_up(o + (size_t)2 * wcap, 16);
  L.perm1 = o;
  o = align_up(o + (size_t)2 * wcap, 16);
  L.flag = o;
  o = align_up(o + (size_t)wcap, 16);
  L.hist = o;
  o = align_up(o + 256 * 4, 16);
  L.stack = o;
  o = align_up(o + WSTK * sizeof(Task), 16);
  L.ctl = o;
  o = align_up(o + sizeof(SmemCtl), 16);
  L.per_warp = o;
  return L;
}

int warp_cap_for(int d) { return d <= 4 ? 512 : 256; }

template <int D>
__global__ void __launch_bounds__(WK_WARPS * 32, 4) k_smem_warp(SmemArgs a) {
  extern __shared__ __align__(16) uint8_t sm[];
  const int cap = a.cap, lane = lane_id();
  const WarpLayout Lo = warp_layout(cap, D);
  uint8_t* base = sm + (size_t)warp_id() * Lo.per_warp;
  SmemPtrs q;
  q.X = (int32_t*)(base + Lo.X);
  q.ID = (uint32_t*)(base + Lo.ID);
  q.perm0 = (uint16_t*)(base + Lo.perm0);
  q.perm1 = (uint16_t*)(base + Lo.perm1);
  q.flag = base + Lo.flag;
  q.whist = (unsigned*)(base + Lo.hist);
  q.wred = nullptr;
  q.wstack = (Task*)(base + Lo.stack);
  q.ctl = (SmemCtl*)(base + Lo.ctl);
  const uint32_t nsegs = *a.nsegs;
  if (lane == 0) q.ctl->maxd = 0;
  __syncwarp();
  // every warp takes segments in turn (a grid of a few CTAs per SM)
  for (uint32_t sid = blockIdx.x * WK_WARPS + warp_id(); sid < nsegs; sid += gridDim.x * WK_WARPS) {
    const Seg seg = a.segs[sid];
    if (seg.len > (uint32_t)cap) {
      if (lane == 0) set_error(a.st, DERR_CAPACITY, 250000);
      return;
    }
    const int n = (int)seg.len;
    if (n > 0 && n <= a.p.phi && seg.where == IN_A) {
      // a leaf whose points already sit at their final arena positions
      if (lane == 0) {
        a.nodes[seg.root] = Node{0, (uint32_t)n, (uint32_t)seg.start, 0};
        a.ndim[seg.root] = PKD_LEAF;
        q.ctl->maxd = max(q.ctl->maxd, seg.depth);
      }
      continue;
    }
    __syncwarp();
    load_segment<D>(a, seg, q.X, q.ID, q.perm0, cap, lane, 32);
    if (lane == 0) q.ctl->next_slot = 0;
    __syncwarp();
    if (n == 0) {
      if (lane == 0) {
        a.nodes[seg.root] = Node{0, 0, (uint32_t)seg.start, 0};
        a.ndim[seg.root] = PKD_LEAF;
      }
      continue;
    }
    SmemCtx<D> cx = make_ctx<D>(a, q, cap);
    cx.start = seg.start;
    cx.slot_base = (uint32_t)(a.shared_cap + 2 * seg.start);
    cx.slot_limit = 2 * n;
    const Team wt{warp_id(), 1, 0, q.whist, nullptr};
    warp_run<false, D>(wt, cx, Task{0, (uint16_t)n, 0, 0, 0, seg.depth, seg.root}, q.wstack, 0);
  }
  __syncwarp();
  if (lane == 0) atomicMax(&a.st->max_depth, q.ctl->maxd);
}

template <int D>
static void launch_smem_build(const SmemArgs& a, uint32_t nblocks, size_t smb, cudaStream_t s) {
  static int set = 0;
  if (set < (int)smb) {
    cudaFuncSetAttribute(k_smem_build<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    set = (int)smb;
  }
  PKD_LAUNCH(k_smem_build<D><<<nblocks, SM_THREADS, smb, s>>>(a));
}

template <int D>
static void launch_smem_sorted(const SmemArgs& a, uint32_t nblocks, size_t smb, cudaStream_t s) {
  static int set = 0;
  if (set < (int)smb) {
    cudaFuncSetAttribute(k_smem_sorted<D, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    set = (int)smb;
  }
  PKD_LAUNCH((k_smem_sorted<D, 1><<<nblocks, SS_THREADS, smb, s>>>(a)));
}
template <int D>
static void launch_smem_sorted2(const SmemArgs& a, uint32_t nblocks, size_t smb, cudaStream_t s) {
  static int set = 0;
  if (set < (int)smb) {
    cudaFuncSetAttribute(k_smem_sorted<D, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    set = (int)smb;
  }
  PKD_LAUNCH((k_smem_sorted<D, 2><<<nblocks, SS_THREADS, smb, s>>>(a)));
}

// A second stream of the current device, created on first use.
static cudaStream_t aux_stream() {
  static std::mutex mu;
  static std::map<int, cudaStream_t> streams;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = streams.find(dev);
  if (it != streams.end()) return it->second;
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  streams[dev] = st;
  return st;
}

// Largest capacity of the presorted base case that lets two CTAs share an
// SM (each gets half of the SM's shared memory, less the per-CTA reserve).
static int sorted_cap_two_per_sm(int d) {
  static int per_sm = -1;
  if (per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (per_sm <= 0) per_sm = 96 * 1024;
  }
  const size_t budget = (size_t)per_sm / 2 - 2048;
  int lo = 64, hi = 16384;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (sorted_layout(mid, d).total <= budget) lo = mid;
    else hi = mid - 1;
  }
  return lo & ~63;
}

template <int D>
static void launch_smem_skel(const SmemArgs& a, uint32_t nblocks, size_t smb, cudaStream_t s) {
  static int set = 0;
  if (set < (int)smb) {
    cudaFuncSetAttribute(k_smem_skel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    set = (int)smb;
  }
  PKD_LAUNCH(k_smem_skel<D><<<nblocks, SM_THREADS, smb, s>>>(a));
}

template <int D>
static void launch_smem_warp(const SmemArgs& a, uint32_t nblocks, size_t smb, cudaStream_t s) {
  static int set = 0;
  if (set < (int)smb) {
    cudaFuncSetAttribute(k_smem_warp<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    set = (int)smb;
  }
  PKD_LAUNCH(k_smem_warp<D><<<nblocks, WK_WARPS * 32, smb, s>>>(a));
}

// ---------------------------------------------------------------------------
// Scans
// ---------------------------------------------------------------------------


// ---------------------------------------------------------------------------
// Round bookkeeping
// ---------------------------------------------------------------------------



// Split a segment list into big segments (ctr[0], their tiles ctr[2], their
// points *pts) and segments finished in shared memory, appended to the
// persistent base lists: one CTA per SM (longer than cap2), two CTAs per SM
// (*nbase), one warp (*nwbase) and one warp with a small slice (*ntbase).
__global__ void k_classify(const Seg* segs, uint32_t nseg, uint32_t cap, Seg* big, uint32_t* ctr,
                           unsigned long long* pts, Seg* base, uint32_t* nbase, uint32_t base_cap,
                           Seg* wbase, uint32_t* nwbase, uint32_t wcap, Seg* tbase, uint32_t* ntbase,
                           uint32_t tcap, Seg* bbase, uint32_t* nbbase, uint32_t cap2, uint32_t tile,
                           uint32_t where, unsigned long long* base_pts, DevStatus* st) {
  if (pkd_failed_block(st)) return;  // uniform: before the block-wide reservations
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  Seg s{};
  int kind = -1;  // 0 big, 1 one CTA (two per SM), 2 one warp, 3 small slice, 4 one CTA per SM
  if (i < nseg) {
    s = segs[i];
    if (s.len != SEG_SKIP) {
      s.where = where;
      kind = s.len > cap ? 0 : (s.len > cap2 ? 4 : (s.len > wcap ? 1 : (s.len > tcap ? 2 : 3)));
    }
  }
  // the list counters and point sums are updated once per block
  const uint32_t c[6] = {kind == 0, kind == 1, kind == 2, kind == 3, kind == 4,
                         kind == 0 ? (s.len + tile - 1) / tile : 0u};
  uint32_t* const ctrs[6] = {&ctr[0], nbase, nwbase, ntbase, nbbase, &ctr[2]};
  uint32_t first[6];
  block_reserve<6>(c, ctrs, first);
  const unsigned long long len = kind >= 0 ? s.len : 0ull;
  const unsigned long long v[4] = {kind == 0 ? len : 0ull, (kind == 1 || kind == 4) ? len : 0ull,
                                   kind == 2 ? len : 0ull, kind == 3 ? len : 0ull};
  unsigned long long* const sums[4] = {pts, &base_pts[0], &base_pts[1], &base_pts[2]};
  block_add64<4>(v, sums);
  if (kind == 0) {
    big[first[0]] = s;
  } else if (kind > 0) {
    const uint32_t b = first[kind];
    if (b < base_cap) (kind == 1 ? base : (kind == 2 ? wbase : (kind == 3 ? tbase : bbase)))[b] = s;
    else set_error(st, DERR_CAPACITY, 300 + kind);
  }
}

// Sample: points whose hash at the segment's depth passes the rate test.
// Persistent CTAs, each over a contiguous run of tiles: a CTA hashes a
// tile's ids and appends the sampled positions to a shared list; once per
// run of tiles of one segment (or before the list could overflow) it
// reserves the list's slots in the segment's sample with one atomic and
// gathers their coordinates.  One atomic per CTA and segment instead of one
// per tile: the first round's tiles all belong to one segment.  The order of
// a sample is immaterial: only its multiset enters the skeleton.
constexpr int SAMPLE_THREADS = 256;
constexpr int SAMPLE_PER = 16;      // points per thread (tiles of up to 4096)
constexpr int SAMPLE_LIST = 8192;   // sampled positions held before a flush
constexpr int SAMPLE_CTAS_PER_SM = 4;

__device__ __forceinline__ void sample_flush(const RoundArgs& r, const Seg& seg, uint32_t s, const uint32_t* lst,
                                             int nl, uint32_t* base_sh) {
  if (threadIdx.x == 0) *base_sh = atomicAdd(&r.scnt[s], (uint32_t)nl);
  __syncthreads();
  const uint64_t o0 = seg.start + *base_sh;
  const int d = r.p.d;
  for (int i = threadIdx.x; i < nl; i += SAMPLE_THREADS) {
    const uint64_t g = seg.start + lst[i];
    for (int j = 0; j < d; ++j) r.samp.c[(uint64_t)j * r.samp.stride + o0 + i] = r.src.x(d, j, g);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(SAMPLE_THREADS) k_sample(RoundArgs r, uint32_t ntiles) {
  __shared__ uint32_t sh[33];
  __shared__ uint32_t base_sh;
  __shared__ uint32_t lst[SAMPLE_LIST];
  const uint32_t per_cta = (ntiles + gridDim.x - 1) / gridDim.x;
  const uint32_t tb = min(ntiles, blockIdx.x * per_cta), te = min(ntiles, tb + per_cta);
  if (tb >= te) return;
  const uint32_t nb = *r.nbig;
  uint32_t s = seg_of_tile(r.tile0, nb, tb);
  Seg seg = r.big[s];
  uint32_t t0 = r.tile0[s];
  int shift = sample_shift(r.p, seg.len);
  uint64_t key = sample_key(r.p.seed, seg.depth);
  int nl = 0;  // uniform
  for (uint32_t tile = tb; tile < te; ++tile) {
    if (s + 1 < nb && r.tile0[s + 1] <= tile) {  // the next segment with tiles
      if (nl) sample_flush(r, seg, s, lst, nl, &base_sh);
      nl = 0;
      do {
        ++s;
      } while (s + 1 < nb && r.tile0[s + 1] <= tile);
      seg = r.big[s];
      t0 = r.tile0[s];
      shift = sample_shift(r.p, seg.len);
      key = sample_key(r.p.seed, seg.depth);
    }
    const uint64_t first = (uint64_t)(tile - t0) * r.TILE;
    if (first >= seg.len) continue;
    const int cnt = (int)min((uint64_t)r.TILE, (uint64_t)seg.len - first);
    if (nl + cnt > SAMPLE_LIST) {
      sample_flush(r, seg, s, lst, nl, &base_sh);
      nl = 0;
    }
    uint32_t ids[SAMPLE_PER];
#pragma unroll
    for (int k = 0; k < SAMPLE_PER; ++k) {
      const int i = k * SAMPLE_THREADS + threadIdx.x;
      if (i < cnt) ids[k] = r.src.id(seg.start + first + (uint64_t)i);
    }
    unsigned fl = 0;
#pragma unroll
    for (int k = 0; k < SAMPLE_PER; ++k) {
      const int i = k * SAMPLE_THREADS + threadIdx.x;
      if (i < cnt && in_sample_k(key, ids[k], shift)) fl |= 1u << k;
    }
    uint32_t total;
    const uint32_t off = block_excl_scan<uint32_t>((uint32_t)__popc(fl), sh, &total);
    int q = 0;
#pragma unroll
    for (int k = 0; k < SAMPLE_PER; ++k)
      if (fl & (1u << k)) lst[nl + (int)off + q++] = (uint32_t)(first + (uint64_t)(k * SAMPLE_THREADS + threadIdx.x));
    nl += (int)total;
  }
  if (nl) sample_flush(r, seg, s, lst, nl, &base_sh);
}

// ---------------------------------------------------------------------------
// Device-wide skeleton levels for samples larger than one CTA
// ---------------------------------------------------------------------------

struct JobState {
  int mn[PKD_DMAX];
  int mx[PKD_DMAX];
  int split;       // 1: this node splits
  int dim;
  int k;
  unsigned prefix, mask;
  int less, eq;
  int x;
  int L;
  unsigned lcur, rcur;
  int fixmin;
};

struct JobArgs {
  Params p;
  int d;
  const SkelJob* jobs;
  const uint32_t* njobs;
  const uint32_t* jtile0;
  JobState* js;
  uint32_t* jhist;  // [job][256]
  Pts sb[2];        // sample buffers
  int2* skel;
  int HN;
  int scap;
  SkelJob* next_big;
  uint32_t* next_ctr;  // [0] big jobs, [1] their tiles, [2] small jobs
  SkelJob* small;
  uint32_t small_cap, big_cap;
  DevStatus* st;
};

__global__ void k_job_tiles(const SkelJob* jobs, const uint32_t* njobs, uint32_t* jtile0) {
  __shared__ uint32_t sh[33];
  const uint32_t n = *njobs;
  uint32_t c = 0;
  for (uint32_t base = 0; base < n; base += blockDim.x) {
    uint32_t i = base + threadIdx.x;
    uint32_t t = i < n ? (jobs[i].n + JOB_TILE - 1) / JOB_TILE : 0;
    uint32_t tot;
    uint32_t e = block_excl_scan<uint32_t>(t, sh, &tot);
    if (i < n) jtile0[i] = c + e;
    c += tot;
  }
}

__global__ void k_job_init(JobArgs a) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *a.njobs) return;
  JobState& s = a.js[i];
  for (int j = 0; j < PKD_DMAX; ++j) {
    s.mn[j] = INT32_MAX;
    s.mx[j] = INT32_MIN;
  }
  s.split = 0;
  s.lcur = s.rcur = 0;
  s.fixmin = INT32_MAX;
  for (int b = 0; b < 256; ++b) a.jhist[(uint64_t)i * 256 + b] = 0;
}

struct JobTile {
  uint32_t job;
  SkelJob jb;
  uint64_t first;
  int cnt;
};

__device__ __forceinline__ bool job_tile(const JobArgs& a, JobTile& t) {
  const uint32_t nj = *a.njobs;
  t.job = seg_of_tile(a.jtile0, nj, blockIdx.x);
  t.jb = a.jobs[t.job];
  t.first = (uint64_t)(blockIdx.x - a.jtile0[t.job]) * JOB_TILE;
  if (t.first >= t.jb.n) return false;
  t.cnt = (int)min((uint64_t)JOB_TILE, (uint64_t)t.jb.n - t.first);
  return true;
}

__global__ void __launch_bounds__(JOB_THREADS) k_job_stats(JobArgs a) {
  JobTile t;
  if (!job_tile(a, t)) return;
  __shared__ int smn[PKD_DMAX][JOB_THREADS / 32], smx[PKD_DMAX][JOB_THREADS / 32];
  const Pts& B = a.sb[t.jb.buf];
  const int d = a.d;
  for (int j = 0; j < d; ++j) {
    int mn = INT32_MAX, mx = INT32_MIN;
    for (int i = threadIdx.x; i < t.cnt; i += blockDim.x) {
      int v = B.c[(uint64_t)j * B.stride + t.jb.a + t.first + i];
      mn = min(mn, v);
      mx = max(mx, v);
    }
    mn = warp_min(mn);
    mx = warp_max(mx);
    if (lane_id() == 0) {
      smn[j][warp_id()] = mn;
      smx[j][warp_id()] = mx;
    }
  }
  __syncthreads();
  if (threadIdx.x < d) {
    const int j = threadIdx.x;
    int mn = INT32_MAX, mx = INT32_MIN;
    for (int w = 0; w < JOB_THREADS / 32; ++w) {
      mn = min(mn, smn[j][w]);
      mx = max(mx, smx[j][w]);
    }
    atomicMin(&a.js[t.job].mn[j], mn);
    atomicMax(&a.js[t.job].mx[j], mx);
  }
}

__global__ void k_job_choose(JobArgs a) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *a.njobs) return;
  const SkelJob jb = a.jobs[i];
  JobState& s = a.js[i];
  int dim = -1;
  if (jb.j < jb.lam && jb.n >= jb.min_split) dim = widest_dim_rt(s.mn, s.mx, a.d);
  s.split = dim >= 0;
  s.dim = dim < 0 ? 0 : dim;
  s.k = (int)(jb.n / 2);
  s.prefix = 0;
  s.mask = 0;
  s.less = 0;
  s.eq = 0;
}

__global__ void __launch_bounds__(JOB_THREADS) k_job_hist(JobArgs a, int pass) {
  JobTile t;
  if (!job_tile(a, t)) return;
  const JobState& s = a.js[t.job];
  if (!s.split) return;
  __shared__ unsigned h[256];
  for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const Pts& B = a.sb[t.jb.buf];
  const int shift = 24 - 8 * pass;
  const unsigned prefix = s.prefix, mask = s.mask;
  const int32_t* X = B.c + (uint64_t)s.dim * B.stride + t.jb.a + t.first;
  for (int i = threadIdx.x; i < t.cnt; i += blockDim.x) {
    unsigned v = (unsigned)X[i];
    if ((v & mask) == prefix) atomicAdd(&h[(v >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 256; b += blockDim.x)
    if (h[b]) atomicAdd(&a.jhist[(uint64_t)t.job * 256 + b], h[b]);
}

// One warp per job.
__global__ void k_job_pick(JobArgs a, int pass) {
  const uint32_t job = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (job >= *a.njobs) return;
  JobState& s = a.js[job];
  if (!s.split) return;
  unsigned* h = a.jhist + (uint64_t)job * 256;
  int digit, below, eq;
  warp_find_digit(h, s.k, digit, below, eq);
  __syncwarp();
  for (int b = lane_id(); b < 256; b += 32) h[b] = 0;
  if (lane_id() == 0) {
    const int shift = 24 - 8 * pass;
    s.prefix |= (unsigned)digit << shift;
    s.mask |= 255u << shift;
    s.k -= below;
    s.less += below;
    s.eq = eq;
  }
}

__global__ void __launch_bounds__(JOB_THREADS) k_job_minabove(JobArgs a) {
  JobTile t;
  if (!job_tile(a, t)) return;
  JobState& s = a.js[t.job];
  if (!s.split || s.less != 0) return;
  const Pts& B = a.sb[t.jb.buf];
  const int32_t* X = B.c + (uint64_t)s.dim * B.stride + t.jb.a + t.first;
  const int x = (int)s.prefix;
  int m = INT32_MAX;
  for (int i = threadIdx.x; i < t.cnt; i += blockDim.x) {
    int v = X[i];
    if (v > x) m = min(m, v);
  }
  m = warp_min(m);
  if (lane_id() == 0 && m != INT32_MAX) atomicMin(&s.fixmin, m);
}

__global__ void k_job_fix(JobArgs a) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *a.njobs) return;
  JobState& s = a.js[i];
  if (!s.split) return;
  if (s.less == 0) {
    // nothing strictly below the median: split at the next distinct value;
    // the left side is then exactly the copies of the minimum.
    s.x = s.fixmin;
    s.L = s.eq;
  } else {
    s.x = (int)s.prefix;
    s.L = s.less;
  }
}

__global__ void __launch_bounds__(JOB_THREADS) k_job_partition(JobArgs a) {
  JobTile t;
  if (!job_tile(a, t)) return;
  JobState& s = a.js[t.job];
  if (!s.split) return;
  __shared__ uint32_t sh[33];
  __shared__ uint32_t base_l, base_r;
  const Pts& B = a.sb[t.jb.buf];
  const Pts& O = a.sb[t.jb.buf ^ 1];
  const int d = a.d;
  const int x = s.x;
  const int32_t* X = B.c + (uint64_t)s.dim * B.stride + t.jb.a + t.first;
  // Each thread takes a contiguous run of the tile so one scan covers it.
  const int per = (t.cnt + JOB_THREADS - 1) / JOB_THREADS;
  const int i0 = min(t.cnt, (int)threadIdx.x * per), i1 = min(t.cnt, i0 + per);
  uint32_t nl = 0;
  for (int i = i0; i < i1; ++i) nl += X[i] < x;
  uint32_t tl;
  uint32_t el = block_excl_scan<uint32_t>(nl, sh, &tl);
  const uint32_t er = (uint32_t)i0 - el;
  if (threadIdx.x == 0) {
    base_l = atomicAdd(&s.lcur, tl);
    base_r = atomicAdd(&s.rcur, (uint32_t)t.cnt - tl);
  }
  __syncthreads();
  uint64_t pl = t.jb.a + base_l + el;
  uint64_t pr = t.jb.a + (uint64_t)s.L + base_r + er;
  for (int i = i0; i < i1; ++i) {
    const uint64_t src = t.jb.a + t.first + i;
    const bool left = X[i] < x;
    const uint64_t dst = left ? pl++ : pr++;
    for (int j = 0; j < d; ++j) O.c[(uint64_t)j * O.stride + dst] = B.c[(uint64_t)j * B.stride + src];
  }
}

__device__ void push_job(const JobArgs& a, const SkelJob& c) {
  int2* sk = a.skel + (uint64_t)c.seg * a.HN;
  if (c.j >= c.lam || c.n < c.min_split) {
    sk[c.h] = make_int2(0, sk_meta(SK_BUCKET, 0, 0));
    return;
  }
  if (c.n > (uint32_t)a.scap) {
    uint32_t k = atomicAdd(&a.next_ctr[0], 1u);
    if (k >= a.big_cap) {
      set_error(a.st, DERR_CAPACITY, 400);
      return;
    }
    a.next_big[k] = c;
    atomicAdd(&a.next_ctr[1], (c.n + JOB_TILE - 1) / JOB_TILE);
  } else {
    uint32_t k = atomicAdd(&a.next_ctr[2], 1u);
    if (k >= a.small_cap) {
      set_error(a.st, DERR_CAPACITY, 401);
      return;
    }
    a.small[k] = c;
  }
}

__global__ void k_job_children(JobArgs a) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *a.njobs) return;
  const SkelJob jb = a.jobs[i];
  const JobState& s = a.js[i];
  int2* sk = a.skel + (uint64_t)jb.seg * a.HN;
  if (!s.split) {
    sk[jb.h] = make_int2(0, sk_meta(SK_BUCKET, 0, 0));
    return;
  }
  if (s.L <= 0 || (uint32_t)s.L >= jb.n) {
    set_error(a.st, DERR_STATE, 500);
    return;
  }
  sk[jb.h] = make_int2(s.x, sk_meta(SK_INTERNAL, s.dim, 0));
  SkelJob l = jb, r = jb;
  l.h = 2 * jb.h;
  r.h = 2 * jb.h + 1;
  l.buf = r.buf = (uint8_t)(jb.buf ^ 1);
  l.j = r.j = (uint8_t)(jb.j + 1);
  l.n = (uint32_t)s.L;
  r.a = jb.a + (uint64_t)s.L;
  r.n = jb.n - (uint32_t)s.L;
  push_job(a, l);
  push_job(a, r);
}

// Root jobs: one per big segment, on its sample.
__global__ void k_root_jobs(RoundArgs r, JobArgs a, int exact_pass) {
  uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= *r.nbig) return;
  const Seg seg = r.big[s];
  SkelJob jb;
  jb.seg = s;
  jb.h = 1;
  jb.a = seg.start;
  jb.buf = 0;
  jb.j = 0;
  jb.pad = 0;
  jb.pad2 = 0;
  if (!exact_pass) {
    jb.n = r.scnt[s];
    jb.lam = (uint8_t)r.lam;
    jb.min_split = 2u * (uint32_t)r.p.sigma_os;
  } else {
    if (r.exact[s] != 1) return;
    jb.n = seg.len;  // every point of the segment was copied into the sample buffer
    jb.lam = 1;
    jb.min_split = 2;
  }
  push_job(a, jb);
}

// Segments whose skeleton root is a bucket take one exact level next.
__global__ void k_mark_exact(RoundArgs r, uint32_t* ctr) {
  uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= *r.nbig) return;
  const int m = r.skel[(uint64_t)s * r.HN + 1].y;
  if (r.exact[s] == 0 && sk_state(m) == SK_BUCKET) {
    r.exact[s] = 1;
    atomicAdd(ctr, 1u);
  }
}

__global__ void k_copy_exact(RoundArgs r) {
  const uint32_t nb = *r.nbig;
  const uint32_t s = seg_of_tile(r.tile0, nb, blockIdx.x);
  if (r.exact[s] != 1) return;
  const Seg seg = r.big[s];
  const uint64_t first = (uint64_t)(blockIdx.x - r.tile0[s]) * r.TILE;
  if (first >= seg.len) return;
  const int cnt = (int)min((uint64_t)r.TILE, (uint64_t)seg.len - first);
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const uint64_t g = seg.start + first + i;
    for (int j = 0; j < r.p.d; ++j) r.samp.c[(uint64_t)j * r.samp.stride + g] = r.src.x(r.p.d, j, g);
  }
}

// Number the buckets left to right, detect heavy segments, give every
// skeleton node a tree slot (root: the segment's own slot).
__global__ void k_finalize(RoundArgs r) {
  uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= *r.nbig) return;
  int2* sk = r.skel + (uint64_t)s * r.HN;
  uint32_t* sl = r.slots + (uint64_t)s * r.HN;
  const Seg seg = r.big[s];
  if (sk_state(sk[1].y) != SK_INTERNAL) {
    // exact level found no split: every point is identical
    sk[1] = make_int2(0, sk_meta(SK_HEAVY, 0, 0));
    r.nbk[s] = 0;
    sl[1] = seg.root;
    return;
  }
  // in-order walk of the heap
  int stack[12];
  int sp = 0, h = 1, nb = 0, ni = 0;
  while (sp > 0 || h != 0) {
    if (h != 0) {
      const int st = sk_state(sk[h].y);
      if (st == SK_INTERNAL) {
        stack[sp++] = h;
        h = 2 * h;
        continue;
      }
      if (st != SK_BUCKET) {
        set_error(r.st, DERR_STATE, 600);
        return;
      }
      sk[h].y = sk_meta(SK_BUCKET, 0, nb++);
      h = 0;
    } else {
      h = stack[--sp];
      ++ni;
      h = 2 * h + 1;
    }
  }
  r.nbk[s] = nb;
  const uint32_t need = (uint32_t)(ni - 1 + nb);
  const uint32_t b0 = atomicAdd(r.shared_next, need);
  if ((uint64_t)b0 + need > r.shared_cap) {
    set_error(r.st, DERR_SLOT, 601);
    return;
  }
  uint32_t k = b0;
  for (int v = 1; v < r.HN; ++v) {
    const int st = sk_state(sk[v].y);
    if (st == SK_NONE) continue;
    sl[v] = (v == 1) ? seg.root : k++;
  }
}

// ---------------------------------------------------------------------------
// Sieve: count and scatter
// ---------------------------------------------------------------------------




// Children segments, interior nodes and heavy leaves of every big segment.
__global__ void k_emit(RoundArgs r, uint32_t* heavy_ctr) {
  if (pkd_failed_block(r.st)) return;
  uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= *r.nbig) return;
  const Seg seg = r.big[s];
  const int2* sk = r.skel + (uint64_t)s * r.HN;
  const uint32_t* sl = r.slots + (uint64_t)s * r.HN;
  Seg* ch = r.children + (uint64_t)s * r.NB;
  const uint32_t nb = r.nbk[s];
  for (int b = (int)nb; b < r.NB; ++b) ch[b].len = SEG_SKIP;
  if (sk_state(sk[1].y) == SK_HEAVY) {
    r.nodes[seg.root] = Node{0, seg.len, (uint32_t)seg.start, 0};
    r.ndim[seg.root] = PKD_LEAF;
    atomicAdd(heavy_ctr, 1u);
    atomicMax(&r.st->max_depth, seg.depth);
    return;
  }
  const uint32_t nt = (seg.len + r.TILE - 1) / r.TILE;
  const uint64_t hb = (uint64_t)r.tile0[s] * r.NB;
  const uint32_t base = r.hscan[hb];
  // subtree sizes, children before parents (heap order reversed)
  uint32_t* size = r.sizes + (uint64_t)s * r.HN;
  for (int v = r.HN - 1; v >= 1; --v) {
    const int st = sk_state(sk[v].y);
    if (st == SK_BUCKET) {
      const int b = sk_bucket(sk[v].y);
      const uint32_t b0 = r.hscan[hb + (uint64_t)b * nt] - base;
      const uint32_t b1 = (b + 1 < (int)nb) ? r.hscan[hb + (uint64_t)(b + 1) * nt] - base : seg.len;
      size[v] = b1 - b0;
      Seg c;
      c.start = seg.start + b0;
      c.len = b1 - b0;
      c.depth = seg.depth + (31 - __clz(v));
      c.root = sl[v];
      c.where = (uint32_t)r.dst_where;
      ch[b] = c;
    } else if (st == SK_INTERNAL) {
      size[v] = size[2 * v] + size[2 * v + 1];
      r.nodes[sl[v]] = Node{sk[v].x, size[v], sl[2 * v], sl[2 * v + 1]};
      r.ndim[sl[v]] = (uint8_t)sk_dim(sk[v].y);
    }
  }
  if (size[1] != seg.len) set_error(r.st, DERR_STATE, 700);
}


// Heavy segments whose points are not yet in the arena.
__global__ void k_copy_heavy(RoundArgs r) {
  if (pkd_failed_block(r.st)) return;
  SieveTile t;
  if (!sieve_tile(r, t)) return;
  if (sk_state(r.skel[(uint64_t)t.s * r.HN + 1].y) != SK_HEAVY) return;
  for (int i = threadIdx.x; i < t.cnt; i += blockDim.x) {
    const uint64_t g = t.seg.start + t.first + i;
    for (int j = 0; j < r.p.d; ++j) r.A.c[(uint64_t)j * r.A.stride + g] = r.src.x(r.p.d, j, g);
    r.A.id[g] = r.src.id(g);
  }
}

// ---------------------------------------------------------------------------
// Host orchestration
// ---------------------------------------------------------------------------

static int smem_optin() {
  static int v = -1;
  if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (v <= 0) v = 48 * 1024;
  }
  return v;
}

static int num_sms() {
  static int v = -1;
  if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) v = 152;
  }
  return v;
}

static int cap_for_bytes(int d, size_t budget) {
  int lo = 64, hi = 65535;
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    if (smem_layout(mid, d).total <= budget) lo = mid;
    else hi = mid - 1;
  }
  return lo & ~63;
}

int base_cap_for(int d) {
  if (knobs().base_cap > 0) return knobs().base_cap;
  const size_t budget = (size_t)std::min(smem_optin(), 200 * 1024);
  if (knobs().base_kernel == 0) {
    int lo = 64, hi = 16384;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (sorted_layout(mid, d).total <= budget) lo = mid;
      else hi = mid - 1;
    }
    return lo & ~63;
  }
  return std::min(cap_for_bytes(d, budget), 16384);
}

int skel_cap_for(int d) {
  if (knobs().skel_cap > 0) return knobs().skel_cap;
  const size_t budget = (size_t)std::min(smem_optin(), 200 * 1024);
  return std::min(cap_for_bytes(d, budget), 16384);
}








// Run the job levels for skeleton nodes whose samples exceed one CTA, then
// finish every small node in shared memory.
static int run_skeleton_jobs(JobArgs ja, SkelJob* big0, uint32_t nbig_jobs, uint32_t big_tiles,
                             uint32_t nsmall_host, SmemArgs sa, uint32_t* hctr, uint32_t* dctr,
                             SkelJob* bigA, SkelJob* bigB, uint32_t* d_njobs, Scratch& sc,
                             cudaStream_t s) {
  (void)big0;
  SkelJob* cur = bigA;
  SkelJob* nxt = bigB;
  uint32_t njobs = nbig_jobs, tiles = big_tiles;
  JobState* js = nullptr;
  uint32_t* jhist = nullptr;
  uint32_t* jtile0 = nullptr;
  uint32_t cap_jobs = 0;
  while (njobs > 0) {
    if (njobs > cap_jobs) {
      cap_jobs = std::max(njobs, 64u);
      PKD_TRY(sc.get(&js, cap_jobs));
      PKD_TRY(sc.get(&jhist, (size_t)cap_jobs * 256));
      PKD_TRY(sc.get(&jtile0, cap_jobs));
    }
    PKD_CUDA(cudaMemcpyAsync(d_njobs, &njobs, 4, cudaMemcpyHostToDevice, s));
    ja.jobs = cur;
    ja.njobs = d_njobs;
    ja.jtile0 = jtile0;
    ja.js = js;
    ja.jhist = jhist;
    ja.next_big = nxt;
    const unsigned g1 = (njobs + 127) / 128;
    PKD_LAUNCH(k_job_tiles<<<1, 1024, 0, s>>>(cur, d_njobs, jtile0));
    PKD_LAUNCH(k_job_init<<<g1, 128, 0, s>>>(ja));
    PKD_CUDA(cudaMemsetAsync(dctr, 0, 8, s));  // next big jobs and tiles
    PKD_LAUNCH(k_job_stats<<<tiles, JOB_THREADS, 0, s>>>(ja));
    PKD_LAUNCH(k_job_choose<<<g1, 128, 0, s>>>(ja));
    for (int pass = 0; pass < 4; ++pass) {
      PKD_LAUNCH(k_job_hist<<<tiles, JOB_THREADS, 0, s>>>(ja, pass));
      PKD_LAUNCH(k_job_pick<<<(njobs * 32 + 127) / 128, 128, 0, s>>>(ja, pass));
    }
    PKD_LAUNCH(k_job_minabove<<<tiles, JOB_THREADS, 0, s>>>(ja));
    PKD_LAUNCH(k_job_fix<<<g1, 128, 0, s>>>(ja));
    PKD_LAUNCH(k_job_partition<<<tiles, JOB_THREADS, 0, s>>>(ja));
    PKD_LAUNCH(k_job_children<<<g1, 128, 0, s>>>(ja));
    PKD_CUDA(cudaMemcpyAsync(hctr, dctr, 12, cudaMemcpyDeviceToHost, s));
    PKD_CUDA(cudaStreamSynchronize(s));
    njobs = hctr[0];
    tiles = hctr[1];
    std::swap(cur, nxt);
  }
  // small jobs: the count lives in dctr[2]
  PKD_CUDA(cudaMemcpyAsync(hctr, dctr, 12, cudaMemcpyDeviceToHost, s));
  PKD_CUDA(cudaStreamSynchronize(s));
  const uint32_t nsmall = hctr[2];
  (void)nsmall_host;
  if (nsmall > 0) {
    sa.jobs = ja.small;
    sa.njobs = dctr + 2;
    const int d = sa.p.d;
    sa.cap = skel_cap_for(d);
    const size_t smb = smem_layout(sa.cap, d).total;
    PKD_DISPATCH_D(d, launch_smem_skel, sa, nsmall, smb, s);
  }
  return PKD_OK;
}

int run_build(TreeMem& t, const BuildJob& job, cudaStream_t s) {
  const Params& p = t.p;
  const int d = p.d;
  const int lam = p.lambda;
  const int NB = 1 << lam, HN = 2 << lam;
  const int TILE = std::min(std::max(knobs().tile, 256), 4096);
  const uint32_t cap = (uint32_t)base_cap_for(d);
  const int scap = skel_cap_for(d);
  const uint64_t base = job.base, extent = std::max<uint64_t>(job.extent, 1);
  Scratch sc{s, {}};

  // scratch point buffer B and two sample buffers over [base, base + extent)
  int32_t *bc, *s0c, *s1c;
  uint32_t* bid;
  PKD_TRY(sc.get(&bc, (size_t)d * extent));
  PKD_TRY(sc.get(&bid, extent));
  PKD_TRY(sc.get(&s0c, (size_t)d * extent));
  PKD_TRY(sc.get(&s1c, (size_t)d * extent));
  const Pts B = shifted(Pts{bc, bid, extent}, base);
  Pts S0 = shifted(Pts{s0c, bid, extent}, base), S1 = shifted(Pts{s1c, bid, extent}, base);
  S0.id = S1.id = nullptr;

  // device counters: [0] big segs, [2] their tiles, [3] exact, [4] heavy,
  // [8..10] skeleton jobs; [12] base list length; u64 at [14] big points
  // u32: [12] CTA list, [13] warp list, [24] tiny list, [25] one-CTA-per-SM list;
  // u64: [14] big points, [16] CTA points, [18] warp points, [20] tiny points
  uint32_t* dctr;
  PKD_TRY(sc.get(&dctr, 32));
  unsigned long long* dpts = (unsigned long long*)(dctr + 14);
  unsigned long long* dbase_pts = (unsigned long long*)(dctr + 16);
  uint32_t* d_nbase = dctr + 12;
  PinnedBlock hblk(s);  // 128 bytes of host counters
  uint32_t* hctr = (uint32_t*)hblk.p;
  if (!hctr) return PKD_ENOMEM;
  PKD_CUDA(cudaMemsetAsync(dctr, 0, 32 * 4, s));

  const uint64_t nroots = job.dsegs ? job.dsegs_n : job.segs.size();
  Seg* cur;
  if (job.dsegs) {
    cur = const_cast<Seg*>(job.dsegs);
  } else {
    PKD_TRY(sc.get(&cur, std::max<uint64_t>(nroots, 1)));
    PKD_CUDA(cudaMemcpyAsync(cur, job.segs.data(), nroots * sizeof(Seg), cudaMemcpyHostToDevice, s));
  }
  uint64_t ncur = nroots;
  const uint32_t wcap = (uint32_t)warp_cap_for(d);
  // every base segment is a root or a non-empty bucket: at most extent + roots
  const uint64_t base_cap_segs = extent + nroots + 16;
  Seg *base_list, *wbase_list, *tbase_list, *bbase_list;
  PKD_TRY(sc.get(&base_list, base_cap_segs));
  PKD_TRY(sc.get(&wbase_list, base_cap_segs));
  PKD_TRY(sc.get(&tbase_list, base_cap_segs));
  PKD_TRY(sc.get(&bbase_list, base_cap_segs));
  const uint32_t tcap = 128;
  // the presorted base case runs two CTAs per SM up to cap2 points
  const uint32_t cap2 =
      knobs().base_kernel == 0 ? std::min<uint32_t>(cap, (uint32_t)sorted_cap_two_per_sm(d)) : cap;

  Src src{};
  int src_where;
  if (job.input_coords) {
    src.aos = job.input_coords;
    src.aos_ids = job.input_ids;
    src.is_aos = 1;
    src_where = IN_INPUT;
  } else {
    src.soa = t.A;
    src.is_aos = 0;
    src_where = IN_A;
  }

  SmemArgs sa{};
  sa.p = p;
  sa.A = t.A;
  sa.B = B;
  sa.in_coords = job.input_coords;
  sa.in_ids = job.input_ids;
  sa.nodes = t.nodes;
  sa.ndim = t.ndim;
  sa.st = t.st;
  sa.sbuf[0] = S0.c;
  sa.sbuf[1] = S1.c;
  sa.sstride = extent;
  sa.heap_n = HN;
  sa.shared_cap = t.shared_cap;

  uint32_t* d_nj;
  PKD_TRY(sc.get(&d_nj, 4));

  for (int round = 0; ncur > 0; ++round) {
    if (round > 64) return PKD_EINTERNAL;
    Seg* big;
    PKD_TRY(sc.get(&big, ncur));
    PKD_CUDA(cudaMemsetAsync(dctr, 0, 12 * 4, s));
    PKD_CUDA(cudaMemsetAsync(dpts, 0, 8, s));
    PKD_LAUNCH(k_classify<<<(unsigned)((ncur + 255) / 256), 256, 0, s>>>(
        cur, (uint32_t)ncur, cap, big, dctr, dpts, base_list, d_nbase, (uint32_t)base_cap_segs,
        wbase_list, d_nbase + 1, wcap, tbase_list, dctr + 24, tcap, bbase_list, dctr + 25, cap2, (uint32_t)TILE,
        (uint32_t)src_where,
        dbase_pts, t.st));
    PKD_CUDA(cudaMemcpyAsync(hctr, dctr, 16 * 4, cudaMemcpyDeviceToHost, s));
    PKD_CUDA(cudaStreamSynchronize(s));
    const uint32_t nbig = hctr[0], tiles = hctr[2];
    const uint64_t pts_big = *(unsigned long long*)(hctr + 14);
    if (nbig == 0) break;

    RoundArgs r{};
    r.wait_cycles = knobs().wait_cycles;
    r.p = p;
    r.lam = lam;
    r.NB = NB;
    r.HN = HN;
    r.TILE = TILE;
    r.src = src;
    const bool dst_is_A = (src_where == IN_B);
    r.dst = dst_is_A ? t.A : B;
    r.dst_where = dst_is_A ? IN_A : IN_B;
    r.A = t.A;
    r.big = big;
    r.nbig = dctr;
    PKD_TRY(sc.get(&r.tile0, nbig));
    PKD_TRY(sc.get(&r.excl, nbig));
    PKD_TRY(sc.get(&r.skel, (size_t)nbig * HN));
    PKD_TRY(sc.get(&r.slots, (size_t)nbig * HN));
    PKD_TRY(sc.get(&r.sizes, (size_t)nbig * HN));
    PKD_TRY(sc.get(&r.nbk, nbig));
    PKD_TRY(sc.get(&r.exact, nbig));
    PKD_TRY(sc.get(&r.hist, (size_t)tiles * NB));
    PKD_TRY(sc.get(&r.hscan, (size_t)tiles * NB));
    r.bkt = nullptr;
    if (record_buckets(NB)) PKD_TRY(sc.get(&r.bkt, (size_t)tiles * TILE));
    PKD_TRY(sc.get(&r.scnt, nbig));
    PKD_TRY(sc.get(&r.children, (size_t)nbig * NB));
    r.samp = S0;
    r.nodes = t.nodes;
    r.ndim = t.ndim;
    r.shared_next = t.shared_next;
    r.shared_cap = t.shared_cap;
    r.st = t.st;
    PKD_CUDA(cudaMemsetAsync(r.skel, 0, (size_t)nbig * HN * sizeof(int2), s));
    PKD_CUDA(cudaMemsetAsync(r.scnt, 0, (size_t)nbig * 4, s));
    PKD_CUDA(cudaMemsetAsync(r.exact, 0, nbig, s));
    PKD_LAUNCH(k_big_prefix<<<1, 1024, 0, s>>>(big, dctr, (uint32_t)TILE, r.tile0, r.excl));

    // 1. sample
    {
      KTimer kt;
      ktimer_begin(kt, "sample", pts_big, s);
      const uint32_t sgrid = std::min<uint32_t>(tiles, (uint32_t)stream_sm_count() * SAMPLE_CTAS_PER_SM);
      PKD_LAUNCH(k_sample<<<sgrid, SAMPLE_THREADS, 0, s>>>(r, tiles));
      ktimer_end(kt);
    }

    // 2. skeletons (and, for segments whose skeleton root is a bucket, one
    //    exact level on their own points)
    JobArgs ja{};
    ja.p = p;
    ja.d = d;
    ja.sb[0] = S0;
    ja.sb[1] = S1;
    ja.skel = r.skel;
    ja.HN = HN;
    ja.scap = scap;
    ja.st = t.st;
    const uint32_t small_cap = nbig * (uint32_t)NB + 16;
    const uint32_t big_cap = (uint32_t)std::min<uint64_t>(pts_big / (uint64_t)scap + nbig + 16, 1u << 30);
    SkelJob *bigA, *bigB, *small;
    PKD_TRY(sc.get(&bigA, big_cap));
    PKD_TRY(sc.get(&bigB, big_cap));
    PKD_TRY(sc.get(&small, small_cap));
    ja.small = small;
    ja.small_cap = small_cap;
    ja.big_cap = big_cap;
    uint32_t* jctr = dctr + 8;
    ja.next_ctr = jctr;
    sa.skel = r.skel;
    for (int exact_pass = 0; exact_pass < 2; ++exact_pass) {
      if (exact_pass == 1) {
        PKD_LAUNCH(k_mark_exact<<<(nbig + 127) / 128, 128, 0, s>>>(r, dctr + 3));
        PKD_CUDA(cudaMemcpyAsync(hctr + 3, dctr + 3, 4, cudaMemcpyDeviceToHost, s));
        PKD_CUDA(cudaStreamSynchronize(s));
        if (hctr[3] == 0) break;
        PKD_LAUNCH(k_copy_exact<<<tiles, 256, 0, s>>>(r));
      }
      PKD_CUDA(cudaMemsetAsync(jctr, 0, 12, s));
      ja.next_big = bigA;
      PKD_LAUNCH(k_root_jobs<<<(nbig + 127) / 128, 128, 0, s>>>(r, ja, exact_pass));
      PKD_CUDA(cudaMemcpyAsync(hctr + 8, jctr, 12, cudaMemcpyDeviceToHost, s));
      PKD_CUDA(cudaStreamSynchronize(s));
      PKD_TRY(run_skeleton_jobs(ja, bigA, hctr[8], hctr[9], 0, sa, hctr + 8, jctr, bigA, bigB, d_nj,
                                sc, s));
    }

    // 3. finalize skeletons, count, scan, emit, scatter
    PKD_LAUNCH(k_finalize<<<(nbig + 127) / 128, 128, 0, s>>>(r));
    PKD_DISPATCH_D(d, launch_count, r, tiles, pts_big, "count", s);
    uint32_t* partial;
    const uint64_t nh = (uint64_t)tiles * NB;
    PKD_TRY(sc.get(&partial, (nh + SCAN_TILE - 1) / SCAN_TILE + 1));
    device_excl_scan(r.hist, r.hscan, nh, partial, s);
    PKD_LAUNCH(k_emit<<<(nbig + 63) / 64, 64, 0, s>>>(r, dctr + 4));
    PKD_DISPATCH_D(d, launch_scatter, r, tiles, pts_big, "scatter", s);
    PKD_LAUNCH(k_copy_heavy<<<tiles, 256, 0, s>>>(r));

    // 4. the buckets, now in the destination buffer, are the next round
    cur = r.children;
    ncur = (uint64_t)nbig * NB;
    src.soa = r.dst;
    src.is_aos = 0;
    src_where = r.dst_where;
  }

  // 5. every small subproblem, one CTA each, in shared memory
  PKD_CUDA(cudaMemcpyAsync(hctr + 12, d_nbase, 14 * 4, cudaMemcpyDeviceToHost, s));
  PKD_CUDA(cudaStreamSynchronize(s));
  if (job.before_base) job.before_base();
  const uint64_t cta_pts = *(unsigned long long*)(hctr + 16), warp_pts = *(unsigned long long*)(hctr + 18);
  const uint64_t tiny_pts = *(unsigned long long*)(hctr + 20);
  const uint32_t nbase = std::min<uint32_t>(hctr[12], (uint32_t)base_cap_segs);
  const uint32_t nwbase = std::min<uint32_t>(hctr[13], (uint32_t)base_cap_segs);
  const uint32_t ntbase = std::min<uint32_t>(hctr[24], (uint32_t)base_cap_segs);
  const uint32_t nbbase = std::min<uint32_t>(hctr[25], (uint32_t)base_cap_segs);
  for (int pass = 0; pass < 2; ++pass) {
    const uint32_t nw = pass == 0 ? nwbase : ntbase;
    if (nw == 0) continue;
    SmemArgs wa = sa;
    wa.segs = pass == 0 ? wbase_list : tbase_list;
    wa.nsegs = pass == 0 ? d_nbase + 1 : dctr + 24;
    wa.cap = pass == 0 ? (int)wcap : (int)tcap;
    const size_t smb = warp_layout(wa.cap, d).per_warp * WK_WARPS;
    KTimer kt;
    ktimer_begin(kt, "smem_warp", pass == 0 ? warp_pts : tiny_pts, s);
    const uint32_t blocks = std::min<uint32_t>((nw + WK_WARPS - 1) / WK_WARPS, (uint32_t)(num_sms() * 8));
    PKD_DISPATCH_D(d, launch_smem_warp, wa, blocks, smb, s);
    ktimer_end(kt);
  }
  if (nbase + nbbase > 0) {
    KTimer kt;
    ktimer_begin(kt, "smem_build", cta_pts, s);
    if (knobs().base_kernel == 0) {
      // the one-CTA-per-SM segments run beside the two-CTA launch, on a
      // second stream, so their long CTAs do not form a tail of their own
      cudaStream_t sb = s;
      cudaEvent_t fork = nullptr, join = nullptr;
      if (nbase > 0 && nbbase > 0) {
        sb = aux_stream();
        PKD_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        PKD_CUDA(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
        PKD_CUDA(cudaEventRecord(fork, s));
        PKD_CUDA(cudaStreamWaitEvent(sb, fork, 0));
      }
      if (nbbase > 0) {
        SmemArgs s1 = sa;
        s1.segs = bbase_list;
        s1.nsegs = dctr + 25;
        s1.cap = (int)cap;
        PKD_DISPATCH_D(d, launch_smem_sorted, s1, nbbase, sorted_layout((int)cap, d).total, sb);
      }
      if (nbase > 0) {
        SmemArgs s2 = sa;
        s2.segs = base_list;
        s2.nsegs = d_nbase;
        s2.cap = (int)cap2;
        PKD_DISPATCH_D(d, launch_smem_sorted2, s2, nbase, sorted_layout((int)cap2, d).total, s);
      }
      if (join) {
        PKD_CUDA(cudaEventRecord(join, sb));
        PKD_CUDA(cudaStreamWaitEvent(s, join, 0));
        cudaEventDestroy(fork);
        cudaEventDestroy(join);
      }
    } else {
      sa.segs = base_list;
      sa.nsegs = d_nbase;
      sa.cap = (int)cap;
      PKD_DISPATCH_D(d, launch_smem_build, sa, nbase, smem_layout((int)cap, d).total, s);
    }
    ktimer_end(kt);
  }
  PKD_CUDA(cudaGetLastError());
  return PKD_OK;
}

}  // namespace pkd
