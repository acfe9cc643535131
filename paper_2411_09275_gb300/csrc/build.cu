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
#include <chrono>
#include <map>
#include <mutex>
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "flow.cuh"
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

// The entries of a list, one per CTA at a time, from a persistent grid:
// every CTA takes the next entry from the grab counter (zeroed before the
// launch) until the list is done, so a grid of resident CTAs serves a list
// whose length only the device knows (the skeleton jobs of a graph's loop
// bodies).  The entry's work `f` may return early but only uniformly over
// the CTA.
// The list length is re-read for every entry, so that nothing stays live
// across an entry's work.
__device__ __forceinline__ uint32_t list_len(const uint32_t* n, uint32_t cap) { return min(*n, cap); }

template <class F>
__device__ __forceinline__ void for_each_entry(const uint32_t* n, uint32_t cap, uint32_t* grab, F&& f) {
  __shared__ uint32_t nxt;
  for (;;) {
    __syncthreads();  // the previous entry is done with shared memory
    if (threadIdx.x == 0) nxt = atomicAdd(grab, 1u);
    __syncthreads();
    const uint32_t i = nxt;
    if (i >= list_len(n, cap)) return;
    f(i);
  }
}

template <int D>
__device__ __forceinline__ void smem_build_one(const SmemArgs& a, uint32_t sid) {
  extern __shared__ __align__(16) uint8_t sm[];
  const Seg seg = a.segs[sid];
  const int cap = a.cap, tid = threadIdx.x;
  SmemPtrs q = carve(sm, cap, D);
  if (seg.len > (uint32_t)cap) {
    if (tid == 0) set_error(a.st, DERR_CAPACITY, (int)sid);
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

template <int D>
__global__ void __launch_bounds__(SM_THREADS, 1) k_smem_build(SmemArgs a) {
  if (blockIdx.x < list_len(a.nsegs, a.list_cap)) smem_build_one<D>(a, blockIdx.x);
}

// The base case on presorted lists (one CTA per segment of at most cap
// points): load, sort every dimension once, then split by lookups and stable
// list partitions.  Instantiated for one CTA per SM (the largest capacity)
// and for two (half the shared memory and at most 64 registers a thread);
// the segment lists of the two launches are separated when the segments are
// classified.
template <int D>
__device__ __forceinline__ void smem_sorted_one(const SmemArgs& a, uint32_t sid) {
  extern __shared__ __align__(16) uint8_t sm[];
  const Seg seg = a.segs[sid];
  const int cap = a.cap, tid = threadIdx.x;
  const SortedLayout Lo = sorted_layout(cap, D);
  int32_t* X = (int32_t*)(sm + Lo.X);
  uint32_t* ID = (uint32_t*)(sm + Lo.ID);
  int* sred = (int*)(sm + Lo.red);
  STask* wstack = (STask*)(sm + Lo.stack);
  SmemCtl* ctl = (SmemCtl*)(sm + Lo.ctl);
  if (seg.len > (uint32_t)cap) {
    if (tid == 0) set_error(a.st, DERR_CAPACITY, 400000 + (int)sid);
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

// One CTA per entry of the list (a persistent loop around this body costs
// registers the two-CTAs-per-SM form does not have: it would spill).
template <int D, int MINB>
__global__ void __launch_bounds__(SS_THREADS, MINB) k_smem_sorted(SmemArgs a) {
  if (blockIdx.x < list_len(a.nsegs, a.list_cap)) smem_sorted_one<D>(a, blockIdx.x);
}

template <int D>
__device__ __forceinline__ void smem_skel_one(const SmemArgs& a, uint32_t ji) {
  extern __shared__ __align__(16) uint8_t sm[];
  const SkelJob jb = a.jobs[ji];
  const int cap = a.cap, tid = threadIdx.x;
  SmemPtrs q = carve(sm, cap, D);
  if (jb.n > (uint32_t)cap) {
    if (tid == 0) set_error(a.st, DERR_CAPACITY, 200000 + (int)ji);
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

template <int D>
__global__ void __launch_bounds__(SM_THREADS, 1) k_smem_skel(SmemArgs a) {
  for_each_entry(a.njobs, a.list_cap, a.grab, [&](uint32_t ji) { smem_skel_one<D>(a, ji); });
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
  const uint32_t nsegs = list_len(a.nsegs, a.list_cap);
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

// Launch of a shared-memory kernel with its dynamic shared memory.
template <class K>
static void launch_with_smem(K kern, int* set, uint32_t nblocks, int threads, size_t smb, cudaStream_t s,
                             const SmemArgs& a) {
  if (*set < (int)smb) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    *set = (int)smb;
  }
  if (nblocks == 0) return;
  PKD_LAUNCH(kern<<<nblocks, threads, smb, s>>>(a));
}

template <int D>
static void launch_smem_build(const SmemArgs& a, uint32_t nblocks, size_t smb, cudaStream_t s) {
  static int set = 0;
  launch_with_smem(k_smem_build<D>, &set, nblocks, SM_THREADS, smb, s, a);
}

template <int D>
static void launch_smem_sorted(const SmemArgs& a, uint32_t nblocks, size_t smb, cudaStream_t s) {
  static int set = 0;
  launch_with_smem(k_smem_sorted<D, 1>, &set, nblocks, SS_THREADS, smb, s, a);
}
template <int D>
static void launch_smem_sorted2(const SmemArgs& a, uint32_t nblocks, size_t smb, cudaStream_t s) {
  static int set = 0;
  launch_with_smem(k_smem_sorted<D, 2>, &set, nblocks, SS_THREADS, smb, s, a);
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
__global__ void k_classify(const RoundDyn* dyn, const uint32_t* sel, const uint32_t* ncur, uint32_t cur_cap,
                           uint32_t cap, Seg* big, uint32_t big_cap, uint32_t* ctr,
                           unsigned long long* pts, Seg* base, uint32_t* nbase, uint32_t base_cap,
                           Seg* wbase, uint32_t* nwbase, uint32_t wcap, Seg* tbase, uint32_t* ntbase,
                           uint32_t tcap, Seg* bbase, uint32_t* nbbase, uint32_t cap2, uint32_t tile,
                           unsigned long long* base_pts, DevStatus* st) {
  if (pkd_failed_block(st)) return;  // uniform: before the block-wide reservations
  const RoundDyn& dy = dyn[*sel];
  const Seg* segs = dy.cur;
  const uint32_t where = (uint32_t)dy.src_where;
  const uint32_t nseg = min(*ncur, cur_cap);
  // the grid strides over the segments, a block-uniform loop
  for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < nseg; i0 += gridDim.x * blockDim.x) {
    const uint32_t i = i0 + threadIdx.x;
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
      if (first[0] < big_cap) big[first[0]] = s;
    } else if (kind > 0) {
      const uint32_t b = first[kind];
      if (b < base_cap) (kind == 1 ? base : (kind == 2 ? wbase : (kind == 3 ? tbase : bbase)))[b] = s;
      else set_error(st, DERR_CAPACITY, 300 + kind);
    }
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

__device__ __forceinline__ void sample_flush(const RoundArgs& r, const Src& src, const Seg& seg, uint32_t s, const uint32_t* lst,
                                             int nl, uint32_t* base_sh) {
  if (threadIdx.x == 0) *base_sh = atomicAdd(&r.scnt[s], (uint32_t)nl);
  __syncthreads();
  const uint64_t o0 = seg.start + *base_sh;
  const int d = r.p.d;
  for (int i = threadIdx.x; i < nl; i += SAMPLE_THREADS) {
    const uint64_t g = seg.start + lst[i];
    for (int j = 0; j < d; ++j) r.samp.c[(uint64_t)j * r.samp.stride + o0 + i] = src.x(d, j, g);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(SAMPLE_THREADS) k_sample(RoundArgs r, uint32_t ntiles_host) {
  __shared__ uint32_t sh[33];
  __shared__ uint32_t base_sh;
  __shared__ uint32_t lst[SAMPLE_LIST];
  const Src src = round_src(r);
  const uint32_t ntiles = round_tiles(r, ntiles_host);
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
      if (nl) sample_flush(r, src, seg, s, lst, nl, &base_sh);
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
      sample_flush(r, src, seg, s, lst, nl, &base_sh);
      nl = 0;
    }
    uint32_t ids[SAMPLE_PER];
#pragma unroll
    for (int k = 0; k < SAMPLE_PER; ++k) {
      const int i = k * SAMPLE_THREADS + threadIdx.x;
      if (i < cnt) ids[k] = src.id(seg.start + first + (uint64_t)i);
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
  if (nl) sample_flush(r, src, seg, s, lst, nl, &base_sh);
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
  const uint32_t* jtiles;  // tiles of the current level's jobs (written by k_job_tiles)
};

// Grid-stride loop over i in [0, n).
#define PKD_FOR(i, n) for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += gridDim.x * blockDim.x)

__global__ void k_job_tiles(const SkelJob* jobs, const uint32_t* njobs, uint32_t* jtile0, uint32_t* total) {
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
  if (threadIdx.x == 0) *total = c;
}

__global__ void k_job_init(JobArgs a) {
  PKD_FOR(i, *a.njobs) {
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
}

struct JobTile {
  uint32_t job;
  SkelJob jb;
  uint64_t first;
  int cnt;
};

__device__ __forceinline__ bool job_tile(const JobArgs& a, JobTile& t, uint32_t tile) {
  const uint32_t nj = *a.njobs;
  t.job = seg_of_tile(a.jtile0, nj, tile);
  t.jb = a.jobs[t.job];
  t.first = (uint64_t)(tile - a.jtile0[t.job]) * JOB_TILE;
  if (t.first >= t.jb.n) return false;
  t.cnt = (int)min((uint64_t)JOB_TILE, (uint64_t)t.jb.n - t.first);
  return true;
}

// The grid strides over the level's tiles, one tile per block at a time.
#define PKD_JOB_TILE_KERNEL(name, body_fn)                                  \
  __global__ void __launch_bounds__(JOB_THREADS) name(JobArgs a) {          \
    const uint32_t nt = *a.jtiles;                                          \
    for (uint32_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {        \
      body_fn(a, tile);                                                     \
      __syncthreads();                                                      \
    }                                                                       \
  }

__device__ __forceinline__ void job_stats_tile(const JobArgs& a, uint32_t tile) {
  JobTile t;
  if (!job_tile(a, t, tile)) return;
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
PKD_JOB_TILE_KERNEL(k_job_stats, job_stats_tile)

__global__ void k_job_choose(JobArgs a) {
  PKD_FOR(i, *a.njobs) {
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
}

__device__ __forceinline__ void job_hist_tile(const JobArgs& a, uint32_t tile, int pass) {
  JobTile t;
  if (!job_tile(a, t, tile)) return;
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

__global__ void __launch_bounds__(JOB_THREADS) k_job_hist(JobArgs a, int pass) {
  const uint32_t nt = *a.jtiles;
  for (uint32_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    job_hist_tile(a, tile, pass);
    __syncthreads();
  }
}

// One warp per job.
__global__ void k_job_pick(JobArgs a, int pass) {
  const uint32_t nj = *a.njobs;
  for (uint32_t job = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; job < nj; job += (gridDim.x * blockDim.x) >> 5) {
  JobState& s = a.js[job];
  if (!s.split) continue;
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
}

__device__ __forceinline__ void job_minabove_tile(const JobArgs& a, uint32_t tile) {
  JobTile t;
  if (!job_tile(a, t, tile)) return;
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
PKD_JOB_TILE_KERNEL(k_job_minabove, job_minabove_tile)

__global__ void k_job_fix(JobArgs a) {
  PKD_FOR(i, *a.njobs) {
  JobState& s = a.js[i];
  if (!s.split) continue;
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
}

__device__ __forceinline__ void job_partition_tile(const JobArgs& a, uint32_t tile) {
  JobTile t;
  if (!job_tile(a, t, tile)) return;
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
PKD_JOB_TILE_KERNEL(k_job_partition, job_partition_tile)

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
  PKD_FOR(i, *a.njobs) {
  const SkelJob jb = a.jobs[i];
  const JobState& s = a.js[i];
  int2* sk = a.skel + (uint64_t)jb.seg * a.HN;
  if (!s.split) {
    sk[jb.h] = make_int2(0, sk_meta(SK_BUCKET, 0, 0));
    continue;
  }
  if (s.L <= 0 || (uint32_t)s.L >= jb.n) {
    set_error(a.st, DERR_STATE, 500);
    continue;
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
}

// Root jobs: one per big segment, on its sample.
__global__ void k_root_jobs(RoundArgs r, JobArgs a, int exact_pass) {
  PKD_FOR(s, *r.nbig) {
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
    if (r.exact[s] != 1) continue;
    jb.n = seg.len;  // every point of the segment was copied into the sample buffer
    jb.lam = 1;
    jb.min_split = 2;
  }
  push_job(a, jb);
  }
}

// Segments whose skeleton root is a bucket take one exact level next.
__global__ void k_mark_exact(RoundArgs r, uint32_t* ctr) {
  PKD_FOR(s, *r.nbig) {
    const int m = r.skel[(uint64_t)s * r.HN + 1].y;
    if (r.exact[s] == 0 && sk_state(m) == SK_BUCKET) {
      r.exact[s] = 1;
      atomicAdd(ctr, 1u);
    }
  }
}

__global__ void k_copy_exact(RoundArgs r0, uint32_t ntiles_host) {
  const RoundArgs r = with_dyn(r0);
  const uint32_t nb = *r.nbig, nt = round_tiles(r, ntiles_host);
  for (uint32_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    const uint32_t s = seg_of_tile(r.tile0, nb, tile);
    if (r.exact[s] != 1) continue;
    const Seg seg = r.big[s];
    const uint64_t first = (uint64_t)(tile - r.tile0[s]) * r.TILE;
    if (first >= seg.len) continue;
    const int cnt = (int)min((uint64_t)r.TILE, (uint64_t)seg.len - first);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const uint64_t g = seg.start + first + i;
      for (int j = 0; j < r.p.d; ++j) r.samp.c[(uint64_t)j * r.samp.stride + g] = r.src.x(r.p.d, j, g);
    }
  }
}

// Number the buckets left to right, detect heavy segments, give every
// skeleton node a tree slot (root: the segment's own slot).  One warp per
// segment: a bucket's number is the count of buckets whose first position
// on level lambda lies left of its own (a bitmap of those positions), and
// the slots follow heap order (a running count of the occupied positions).
constexpr int FIN_WARPS = 4;
__device__ __forceinline__ void finalize_warp(const RoundArgs& r, uint32_t s, uint32_t* bits, uint32_t* pre) {
  const int lane = lane_id();
  int2* sk = r.skel + (uint64_t)s * r.HN;
  uint32_t* sl = r.slots + (uint64_t)s * r.HN;
  const Seg seg = r.big[s];
  if (sk_state(sk[1].y) != SK_INTERNAL) {  // warp-uniform
    // exact level found no split: every point is identical
    if (lane == 0) {
      sk[1] = make_int2(0, sk_meta(SK_HEAVY, 0, 0));
      r.nbk[s] = 0;
      sl[1] = seg.root;
    }
    return;
  }
  bits[lane] = 0;
  __syncwarp();
  // every child of an interior node is interior or a bucket; buckets mark
  // their first position
  bool bad = false;
  uint32_t occ = 0;
  for (int v = 1 + lane; v < r.HN; v += 32) {
    const int st = sk_state(sk[v].y);
    if (st == SK_NONE) continue;
    ++occ;
    if (st == SK_INTERNAL) {
      if (2 * v + 1 >= r.HN) {
        bad = true;
      } else {
        const int a = sk_state(sk[2 * v].y), b = sk_state(sk[2 * v + 1].y);
        bad |= (a != SK_INTERNAL && a != SK_BUCKET) || (b != SK_INTERNAL && b != SK_BUCKET);
      }
    } else if (st == SK_BUCKET) {
      const int j = 31 - __clz(v);
      const uint32_t lo = (uint32_t)(v - (1 << j)) << (r.lam - j);
      atomicOr(&bits[lo >> 5], 1u << (lo & 31));
    } else {
      bad = true;
    }
  }
  if (__any_sync(FULL_MASK, bad)) {
    if (lane == 0) set_error(r.st, DERR_STATE, 600);
    return;
  }
  __syncwarp();
  const uint32_t wc = (uint32_t)__popc(bits[lane]);
  const uint32_t incl = (uint32_t)warp_incl_scan((int)wc);
  pre[lane] = incl - wc;
  const uint32_t nb = __shfl_sync(FULL_MASK, incl, 31);
  __syncwarp();
  for (int v = 1 + lane; v < r.HN; v += 32) {
    if (sk_state(sk[v].y) != SK_BUCKET) continue;
    const int j = 31 - __clz(v);
    const uint32_t lo = (uint32_t)(v - (1 << j)) << (r.lam - j);
    const uint32_t num = pre[lo >> 5] + (uint32_t)__popc(bits[lo >> 5] & ((1u << (lo & 31)) - 1u));
    sk[v].y = sk_meta(SK_BUCKET, 0, (int)num);
  }
  const uint32_t need = (uint32_t)warp_sum((int)occ) - 1;  // the root keeps the segment's slot
  uint32_t b0 = 0;
  if (lane == 0) {
    r.nbk[s] = nb;
    b0 = atomicAdd(r.shared_next, need);
  }
  b0 = __shfl_sync(FULL_MASK, b0, 0);
  if ((uint64_t)b0 + need > r.shared_cap) {
    if (lane == 0) set_error(r.st, DERR_SLOT, 601);
    return;
  }
  uint32_t k = b0;
  for (int v0 = 1; v0 < r.HN; v0 += 32) {
    const int v = v0 + lane;
    const bool on = v < r.HN && sk_state(sk[v].y) != SK_NONE;
    const bool takes = on && v != 1;
    const unsigned m = __ballot_sync(FULL_MASK, takes);
    if (on) sl[v] = v == 1 ? seg.root : k + (uint32_t)__popc(m & lanemask_lt());
    k += (uint32_t)__popc(m);
  }
}

__global__ void __launch_bounds__(FIN_WARPS * 32) k_finalize(RoundArgs r) {
  __shared__ uint32_t bits_sh[FIN_WARPS][32], pre_sh[FIN_WARPS][32];
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < *r.nbig; s += nw)
    finalize_warp(r, s, bits_sh[warp_id()], pre_sh[warp_id()]);
}

// ---------------------------------------------------------------------------
// Sieve: count and scatter
// ---------------------------------------------------------------------------




// Children segments, interior nodes and heavy leaves of every big segment:
// one warp per segment.  The buckets (at any level of the skeleton) are
// independent, so their ranges are read by all lanes at once; the interior
// nodes then take their sizes level by level from the deepest.
__device__ __forceinline__ void emit_warp(const RoundArgs& r, uint32_t* heavy_ctr, uint32_t s) {
  const int lane = lane_id();
  const Seg seg = r.big[s];
  const int2* sk = r.skel + (uint64_t)s * r.HN;
  const uint32_t* sl = r.slots + (uint64_t)s * r.HN;
  Seg* ch = r.children + (uint64_t)s * r.NB;
  const uint32_t nb = r.nbk[s];
  for (int b = (int)nb + lane; b < r.NB; b += 32) ch[b].len = SEG_SKIP;
  if (sk_state(sk[1].y) == SK_HEAVY) {  // warp-uniform
    if (lane == 0) {
      r.nodes[seg.root] = Node{0, seg.len, (uint32_t)seg.start, 0};
      r.ndim[seg.root] = PKD_LEAF;
      atomicAdd(heavy_ctr, 1u);
      atomicMax(&r.st->max_depth, seg.depth);
    }
    return;
  }
  const uint32_t nt = (seg.len + r.TILE - 1) / r.TILE;
  const uint64_t hb = (uint64_t)r.tile0[s] * r.NB;
  const uint32_t base = r.hscan[hb];
  uint32_t* size = r.sizes + (uint64_t)s * r.HN;
  for (int v = 1 + lane; v < r.HN; v += 32) {
    const int m = sk[v].y;
    if (sk_state(m) != SK_BUCKET) continue;
    const int b = sk_bucket(m);
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
  }
  __syncwarp();
  for (int j = r.lam - 1; j >= 0; --j) {  // interior nodes sit above level lambda
    for (int v = (1 << j) + lane; v < (2 << j); v += 32) {
      const int2 e = sk[v];
      if (sk_state(e.y) != SK_INTERNAL) continue;
      const uint32_t sz = size[2 * v] + size[2 * v + 1];
      size[v] = sz;
      r.nodes[sl[v]] = Node{e.x, sz, sl[2 * v], sl[2 * v + 1]};
      r.ndim[sl[v]] = (uint8_t)sk_dim(e.y);
    }
    __syncwarp();
  }
  if (lane == 0 && size[1] != seg.len) set_error(r.st, DERR_STATE, 700);
}

__global__ void k_emit(RoundArgs r0, uint32_t* heavy_ctr) {
  if (pkd_failed_block(r0.st)) return;
  const RoundArgs r = with_dyn(r0);
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < *r.nbig; s += nw) emit_warp(r, heavy_ctr, s);
}


// Heavy segments whose points are not yet in the arena.
// (nheavy: the round's heavy segments, counted by the emission; none is
// the common case, and then no tile is looked at)
__global__ void k_copy_heavy(RoundArgs r0, uint32_t ntiles_host, const uint32_t* nheavy) {
  if (pkd_failed_block(r0.st) || *nheavy == 0) return;
  const RoundArgs r = with_dyn(r0);
  const uint32_t nt = round_tiles(r, ntiles_host);
  for (uint32_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    SieveTile t;
    if (!sieve_tile(r, t, tile)) continue;
    if (sk_state(r.skel[(uint64_t)t.s * r.HN + 1].y) != SK_HEAVY) continue;
    for (int i = threadIdx.x; i < t.cnt; i += blockDim.x) {
      const uint64_t g = t.seg.start + t.first + i;
      for (int j = 0; j < r.p.d; ++j) r.A.c[(uint64_t)j * r.A.stride + g] = r.src.x(r.p.d, j, g);
      r.A.id[g] = r.src.id(g);
    }
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








// ---------------------------------------------------------------------------
// Round control on the device
// ---------------------------------------------------------------------------

// Words of a build's device control block.
enum : int {
  C_NBIG = 0,      // big segments of the round
  C_TILES = 2,     // their tiles
  C_EXACT = 3,     // segments that take an exact level
  C_HEAVY = 4,     // heavy segments
  C_JNEXT = 8,     // [8] jobs pushed for the next level, [9] their tiles, [10] small jobs
  C_JSMALL = 10,
  C_NBASE = 12,    // base lists: two CTAs per SM, one warp
  C_NWBASE = 13,
  C_PTS = 14,      // u64: points of the big segments
  C_BASE_PTS = 16, // u64 x3: points of the CTA, warp and small-slice lists
  C_NTBASE = 24,   // base lists: small slice, one CTA per SM
  C_NBBASE = 25,
  C_ROUND = 26,    // rounds done
  C_SEL = 27,      // entry of the round arguments (0 first round, 1 odd, 2 even)
  C_NCUR = 28,     // segments of the round
  C_GO = 29,       // another round
  C_JN = 30,       // jobs of the current skeleton level
  C_JTILES = 31,   // their tiles
  C_JLEVEL = 32,   // skeleton levels done in this pass
  C_JGO = 33,      // another skeleton level
  C_GRAB = 36,     // grab counter of the persistent small-job launch
  C_WORDS = 48
};
constexpr uint32_t MAX_ROUNDS = 64;
constexpr uint32_t MAX_JOB_LEVELS = 64;

__global__ void k_ctl_init(uint32_t* c, uint32_t nroots) {
  for (int i = threadIdx.x; i < C_WORDS; i += blockDim.x) c[i] = i == C_NCUR ? nroots : 0u;
}

// After a round's segments were classified: whether the round has work.
// The counts are within the buffers by construction (every big segment
// holds more than cap points); a count past them stops the build with an
// error instead of reaching past a buffer.
__global__ void k_round_go(uint32_t* c, uint32_t big_cap, uint32_t tiles_cap, DevStatus* st) {
  const bool more = c[C_NBIG] > 0;
  if (c[C_NBIG] > big_cap || c[C_TILES] > tiles_cap) {
    set_error(st, DERR_CAPACITY, 802);
    c[C_NBIG] = c[C_TILES] = 0;
    c[C_GO] = 0;
  } else if (more && c[C_ROUND] >= MAX_ROUNDS) {
    set_error(st, DERR_STATE, 800);
    c[C_GO] = 0;
  } else {
    c[C_GO] = more ? 1u : 0u;
  }
}

// End of a round: its buckets are the next round's segments.
__global__ void k_round_next(uint32_t* c, uint32_t NB) {
  const uint32_t r = c[C_ROUND] + 1;
  c[C_ROUND] = r;
  c[C_SEL] = (r & 1) ? 1u : 2u;
  c[C_NCUR] = c[C_NBIG] * NB;
  for (int i = 0; i < 12; ++i) c[i] = 0;
  c[C_PTS] = c[C_PTS + 1] = 0;
}

// Per-big-segment state of the round, cleared.
__global__ void k_round_clear(RoundArgs r) {
  const uint32_t nb = *r.nbig;
  PKD_FOR(i, nb * (uint32_t)r.HN) {
    r.skel[i] = make_int2(0, 0);
    if (i < nb) {
      r.scnt[i] = 0;
      r.exact[i] = 0;
    }
  }
}

// Start of a skeleton pass: no pushed jobs, no levels, no small jobs.
__global__ void k_jobs_reset(uint32_t* c) {
  c[C_JNEXT] = c[C_JNEXT + 1] = c[C_JSMALL] = 0;
  c[C_JLEVEL] = 0;
  c[C_GRAB] = 0;
}

// The jobs pushed by the last step become the current level (one block).
__global__ void k_job_advance(SkelJob* cur, const SkelJob* next, uint32_t* c, uint32_t cap, DevStatus* st) {
  const uint32_t n = min(c[C_JNEXT], cap);
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) cur[i] = next[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    c[C_JN] = n;
    c[C_JNEXT] = c[C_JNEXT + 1] = 0;
    const uint32_t lvl = c[C_JLEVEL] + 1;
    c[C_JLEVEL] = lvl;
    if (n > 0 && lvl > MAX_JOB_LEVELS) {
      set_error(st, DERR_STATE, 801);
      c[C_JGO] = 0;
    } else {
      c[C_JGO] = n > 0 ? 1u : 0u;
    }
  }
}

// ---------------------------------------------------------------------------
// Device-decided graphs: streams, capture lock, retired executables
// ---------------------------------------------------------------------------

bool& flow_capturing() {
  static thread_local bool v = false;
  return v;
}

std::mutex& flow_mutex() {
  static std::mutex m;
  return m;
}

cudaStream_t flow_stream(int level) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, cudaStream_t> streams;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_pair(dev, level);
  auto it = streams.find(key);
  if (it != streams.end()) return it->second;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  streams[key] = st;
  return st;
}

// The launch shape of a base-case kernel node, set on the device from the
// length of its list just before it runs (a graph's kernel nodes are
// recorded with a placeholder grid; the lists' lengths exist only on the
// device).
struct BaseShape {
  cudaGraphDeviceNode_t node;
  const uint32_t* count;  // list length
  uint32_t cap;           // entries the list can hold
  uint32_t per_block;     // entries per block
  uint32_t max_blocks;    // 0: no limit
  uint32_t pad;
};
constexpr int MAX_SHAPES = 4;

// Recorded builds, reused: a graph's kernels take every pointer and size as
// an argument, so a build whose arguments are all equal to an earlier one's
// (the same tree memory, scratch and input at the same addresses: repeated
// builds of one size, which the stream-ordered pool tends to place at the
// same addresses) launches that graph again instead of recording a new one.
// The key lists every value the recorded kernels take.  An evicted entry
// is destroyed once its last launch has completed (checked without waiting
// at later builds), so eviction never blocks the host.
struct GraphEntry {
  std::vector<uint64_t> key;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  cudaEvent_t done = nullptr;  // after the entry's last launch
  cudaEvent_t base = nullptr;  // external event: the base cases may start
  BaseShape shapes[MAX_SHAPES];
  uint64_t used = 0;
};
constexpr int GRAPH_CACHE = 16;
static std::vector<GraphEntry> g_graphs;   // guarded by flow_mutex()
static std::vector<GraphEntry> g_retired;  // evicted, maybe still running
static uint64_t g_graph_clock = 0;

static void graph_entry_destroy(GraphEntry& e) {
  if (e.exec) cudaGraphExecDestroy(e.exec);
  if (e.graph) cudaGraphDestroy(e.graph);
  if (e.done) cudaEventDestroy(e.done);
  if (e.base) cudaEventDestroy(e.base);
  e = GraphEntry{};
}

// Destroys the evicted entries whose last launch has completed.
static void graph_reap() {
  std::vector<GraphEntry> keep;
  for (GraphEntry& e : g_retired) {
    if (!e.done || cudaEventQuery(e.done) == cudaSuccess) graph_entry_destroy(e);
    else keep.push_back(e);
  }
  cudaGetLastError();  // a pending event's query status is not an error
  g_retired.swap(keep);
}

static GraphEntry* graph_find(const std::vector<uint64_t>& key) {
  for (GraphEntry& e : g_graphs)
    if (e.key == key) {
      e.used = ++g_graph_clock;
      return &e;
    }
  return nullptr;
}

static GraphEntry* graph_slot() {
  if ((int)g_graphs.size() < GRAPH_CACHE) {
    g_graphs.emplace_back();
    return &g_graphs.back();
  }
  GraphEntry* lru = &g_graphs[0];
  for (GraphEntry& e : g_graphs)
    if (e.used < lru->used) lru = &e;
  g_retired.push_back(*lru);
  *lru = GraphEntry{};
  return lru;
}

static int g_graph_builds = 0;  // builds whose rounds ran from one graph launch
static int g_graph_reuses = 0;  // ... of them, launches of a recorded graph


__global__ void k_base_shapes(const BaseShape* sh, int n) {
  if (threadIdx.x != 0) return;
  for (int i = 0; i < n; ++i) {
    const BaseShape b = sh[i];
    const uint32_t c = min(*b.count, b.cap);
    uint32_t blocks = (c + b.per_block - 1) / b.per_block;
    if (b.max_blocks && blocks > b.max_blocks) blocks = b.max_blocks;
    if (blocks == 0) {
      cudaGraphKernelNodeSetEnabled(b.node, false);
    } else {
      cudaGraphKernelNodeSetEnabled(b.node, true);
      cudaGraphKernelNodeSetGridDim(b.node, dim3(blocks, 1, 1));
    }
  }
}

// The kernel node a launch just recorded on a capturing stream.
static cudaGraphNode_t last_node(cudaStream_t st) {
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &nd) != cudaSuccess || nd != 1)
    return nullptr;
  return deps[0];
}

// Makes a recorded kernel node device-updatable; its device handle, or null.
static cudaGraphDeviceNode_t make_updatable(cudaGraphNode_t node) {
  if (!node) return nullptr;
  cudaKernelNodeAttrValue v{};
  v.deviceUpdatableKernelNode.deviceUpdatable = 1;
  if (cudaGraphKernelNodeSetAttribute(node, cudaKernelNodeAttributeDeviceUpdatableKernelNode, &v) != cudaSuccess)
    return nullptr;
  cudaKernelNodeAttrValue o{};
  if (cudaGraphKernelNodeGetAttribute(node, cudaKernelNodeAttributeDeviceUpdatableKernelNode, &o) != cudaSuccess)
    return nullptr;
  return o.deviceUpdatableKernelNode.devNode;
}

// ---------------------------------------------------------------------------
// Host orchestration
// ---------------------------------------------------------------------------

// Every buffer a build needs, sized for the worst case so that no step
// depends on a count the host has not seen:
//   big segments of a round   <= extent / (cap + 1)  (each holds > cap points)
//   their tiles               <= extent / TILE + big segments
//   big skeleton jobs a level <= extent / (scap + 1) (disjoint sample ranges)
struct BuildBufs {
  uint64_t nbig, ncur, tiles, big_jobs, jtiles, small_jobs;
  Seg* big;
  uint32_t *tile0, *slots, *sizes, *nbk, *hist, *hscan, *scnt, *partial;
  uint64_t* excl;
  int2* skel;
  uint8_t *exact, *bkt;
  Seg* children[2];
  SkelJob *jcur, *jnext, *jsmall;
  JobState* js;
  uint32_t *jhist, *jtile0;
  RoundDyn* dyn;
};

int run_build(TreeMem& t, const BuildJob& job, cudaStream_t s) {
  const Params& p = t.p;
  const int d = p.d;
  const int lam = p.lambda;
  const int NB = 1 << lam, HN = 2 << lam;
  const int TILE = std::min(std::max(knobs().tile, 256), 4096);
  const uint32_t cap = (uint32_t)base_cap_for(d);
  const int scap = skel_cap_for(d);
  const uint64_t base = job.base, extent = std::max<uint64_t>(job.extent, 1);
  const int nsm = num_sms();
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

  uint32_t* dctr;
  PKD_TRY(sc.get(&dctr, C_WORDS));
  PinnedBlock hblk(s);  // host copy of the control block
  uint32_t* hctr = (uint32_t*)hblk.p;
  if (!hctr) return PKD_ENOMEM;
  static_assert(C_WORDS * 4 <= PINNED_BLOCK, "control block");
  memset(hctr, 0, C_WORDS * 4);

  const uint64_t nroots = job.dsegs ? job.dsegs_n : job.segs.size();
  if (nroots >= 0xFFFFFFFFull) return PKD_EINVAL;
  Seg* roots;
  if (job.dsegs) {
    roots = const_cast<Seg*>(job.dsegs);
  } else {
    PKD_TRY(sc.get(&roots, std::max<uint64_t>(nroots, 1)));
    PKD_TRY(dev_store(roots, job.segs.data(), nroots * sizeof(Seg), s));
  }
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

  // worst-case round buffers
  BuildBufs bb{};
  bb.nbig = extent / (cap + 1) + 1;
  bb.ncur = std::max<uint64_t>(nroots, bb.nbig * NB);
  bb.tiles = (extent + TILE - 1) / TILE + bb.nbig;
  bb.big_jobs = extent / ((uint64_t)scap + 1) + bb.nbig + 16;
  bb.jtiles = (extent + JOB_TILE - 1) / JOB_TILE + bb.big_jobs;
  bb.small_jobs = bb.nbig * NB + 16;
  if (bb.ncur >= 0xFFFFFFFFull || bb.tiles * NB >= 0xFFFFFFFFull) return PKD_EINVAL;
  PKD_TRY(sc.get(&bb.big, bb.nbig));
  PKD_TRY(sc.get(&bb.tile0, bb.nbig));
  PKD_TRY(sc.get(&bb.excl, bb.nbig));
  PKD_TRY(sc.get(&bb.skel, bb.nbig * HN));
  PKD_TRY(sc.get(&bb.slots, bb.nbig * HN));
  PKD_TRY(sc.get(&bb.sizes, bb.nbig * HN));
  PKD_TRY(sc.get(&bb.nbk, bb.nbig));
  PKD_TRY(sc.get(&bb.exact, bb.nbig));
  PKD_TRY(sc.get(&bb.scnt, bb.nbig));
  PKD_TRY(sc.get(&bb.hist, bb.tiles * NB));
  PKD_TRY(sc.get(&bb.hscan, bb.tiles * NB));
  PKD_TRY(sc.get(&bb.partial, SCAN_BLOCKS + 1));
  bb.bkt = nullptr;
  if (record_buckets(NB)) PKD_TRY(sc.get(&bb.bkt, bb.tiles * TILE));
  PKD_TRY(sc.get(&bb.children[0], bb.nbig * NB));
  PKD_TRY(sc.get(&bb.children[1], bb.nbig * NB));
  PKD_TRY(sc.get(&bb.jcur, bb.big_jobs));
  PKD_TRY(sc.get(&bb.jnext, bb.big_jobs));
  PKD_TRY(sc.get(&bb.jsmall, bb.small_jobs));
  PKD_TRY(sc.get(&bb.js, bb.big_jobs));
  PKD_TRY(sc.get(&bb.jhist, bb.big_jobs * 256));
  PKD_TRY(sc.get(&bb.jtile0, bb.big_jobs));
  PKD_TRY(sc.get(&bb.dyn, 3));

  // the arguments of the three kinds of rounds: the first reads the input
  // (or the arena), the odd ones B, the even ones after the first the arena
  {
    RoundDyn hd[3];
    Src in{};
    if (job.input_coords) {
      in.aos = job.input_coords;
      in.aos_ids = job.input_ids;
      in.is_aos = 1;
    } else {
      in.soa = t.A;
    }
    Src fromB{};
    fromB.soa = B;
    Src fromA{};
    fromA.soa = t.A;
    hd[0] = RoundDyn{in, B, (int)IN_B, job.input_coords ? (int)IN_INPUT : (int)IN_A, roots, bb.children[0]};
    hd[1] = RoundDyn{fromB, t.A, (int)IN_A, (int)IN_B, bb.children[0], bb.children[1]};
    hd[2] = RoundDyn{fromA, B, (int)IN_B, (int)IN_A, bb.children[1], bb.children[0]};
    static_assert(sizeof(hd) % 4 == 0, "round arguments");
    PKD_TRY(dev_store(bb.dyn, hd, sizeof(hd), s));
  }

  RoundArgs r{};
  r.wait_cycles = knobs().wait_cycles;
  r.p = p;
  r.lam = lam;
  r.NB = NB;
  r.HN = HN;
  r.TILE = TILE;
  r.A = t.A;
  r.big = bb.big;
  r.nbig = dctr + C_NBIG;
  r.tile0 = bb.tile0;
  r.excl = bb.excl;
  r.skel = bb.skel;
  r.slots = bb.slots;
  r.sizes = bb.sizes;
  r.nbk = bb.nbk;
  r.exact = bb.exact;
  r.hist = bb.hist;
  r.hscan = bb.hscan;
  r.bkt = bb.bkt;
  r.scnt = bb.scnt;
  r.samp = S0;
  r.nodes = t.nodes;
  r.ndim = t.ndim;
  r.shared_next = t.shared_next;
  r.shared_cap = t.shared_cap;
  r.st = t.st;
  r.dyn = bb.dyn;
  r.sel = dctr + C_SEL;
  r.ntiles = dctr + C_TILES;

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
  sa.skel = bb.skel;

  JobArgs ja{};
  ja.p = p;
  ja.d = d;
  ja.sb[0] = S0;
  ja.sb[1] = S1;
  ja.skel = bb.skel;
  ja.HN = HN;
  ja.scap = scap;
  ja.st = t.st;
  ja.jobs = bb.jcur;
  ja.njobs = dctr + C_JN;
  ja.jtile0 = bb.jtile0;
  ja.js = bb.js;
  ja.jhist = bb.jhist;
  ja.next_big = bb.jnext;
  ja.next_ctr = dctr + C_JNEXT;
  ja.small = bb.jsmall;
  ja.small_cap = (uint32_t)bb.small_jobs;
  ja.big_cap = (uint32_t)bb.big_jobs;
  ja.jtiles = dctr + C_JTILES;

  // launch shapes: grids of resident blocks that stride over device counts
  auto grid_for = [&](uint64_t items, int per_block, int per_sm) {
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((items + per_block - 1) / per_block,
                                                              (uint64_t)nsm * per_sm));
  };
  const unsigned g_seg128 = grid_for(bb.nbig, 128, 8);
  const unsigned g_clear = grid_for(bb.nbig * HN, 256, 8);
  const unsigned g_cls = grid_for(bb.ncur, 256, 8);
  const unsigned g_tiles = grid_for(bb.tiles, 1, 8);
  const unsigned g_job = grid_for(bb.big_jobs, 128, 8);
  const unsigned g_jobw = grid_for(bb.big_jobs * 32, 128, 8);
  const unsigned g_jtiles = grid_for(bb.jtiles, 1, 8);
  const unsigned g_sample = grid_for(bb.tiles, 1, SAMPLE_CTAS_PER_SM);

  const bool graph = knobs().graph_rounds != 0;
  Flow f;
  f.dctl = dctr;
  f.hctl = hctr;
  f.nctl = C_WORDS;
  f.s = s;

  auto classify = [&](Flow& g) {
    PKD_LAUNCH(k_classify<<<g_cls, 256, 0, g.s>>>(
        bb.dyn, dctr + C_SEL, dctr + C_NCUR, (uint32_t)bb.ncur, cap, bb.big, (uint32_t)bb.nbig, dctr,
        (unsigned long long*)(dctr + C_PTS), base_list, dctr + C_NBASE, (uint32_t)base_cap_segs, wbase_list,
        dctr + C_NWBASE, wcap, tbase_list, dctr + C_NTBASE, tcap, bbase_list, dctr + C_NBBASE, cap2,
        (uint32_t)TILE, (unsigned long long*)(dctr + C_BASE_PTS), t.st));
    PKD_LAUNCH(k_round_go<<<1, 1, 0, g.s>>>(dctr, (uint32_t)bb.nbig, (uint32_t)bb.tiles, t.st));
    return PKD_OK;
  };

  // one skeleton level of the jobs whose samples exceed one CTA
  auto job_level = [&](Flow& g) {
    cudaStream_t q = g.s;
    PKD_LAUNCH(k_job_tiles<<<1, 1024, 0, q>>>(bb.jcur, dctr + C_JN, bb.jtile0, dctr + C_JTILES));
    PKD_LAUNCH(k_job_init<<<g_job, 128, 0, q>>>(ja));
    PKD_LAUNCH(k_job_stats<<<g_jtiles, JOB_THREADS, 0, q>>>(ja));
    PKD_LAUNCH(k_job_choose<<<g_job, 128, 0, q>>>(ja));
    for (int pass = 0; pass < 4; ++pass) {
      PKD_LAUNCH(k_job_hist<<<g_jtiles, JOB_THREADS, 0, q>>>(ja, pass));
      PKD_LAUNCH(k_job_pick<<<g_jobw, 128, 0, q>>>(ja, pass));
    }
    PKD_LAUNCH(k_job_minabove<<<g_jtiles, JOB_THREADS, 0, q>>>(ja));
    PKD_LAUNCH(k_job_fix<<<g_job, 128, 0, q>>>(ja));
    PKD_LAUNCH(k_job_partition<<<g_jtiles, JOB_THREADS, 0, q>>>(ja));
    PKD_LAUNCH(k_job_children<<<g_job, 128, 0, q>>>(ja));
    PKD_LAUNCH(k_job_advance<<<1, 1024, 0, q>>>(bb.jcur, bb.jnext, dctr, (uint32_t)bb.big_jobs, t.st));
    return PKD_OK;
  };

  // the skeletons of every big segment: root jobs, device-wide levels while
  // a node's sample exceeds one CTA, then every small node in shared memory
  auto skeleton_pass = [&](Flow& g, int exact_pass) {
    if (exact_pass) PKD_LAUNCH(k_copy_exact<<<g_tiles, 256, 0, g.s>>>(r, 0));
    PKD_LAUNCH(k_jobs_reset<<<1, 1, 0, g.s>>>(dctr));
    PKD_LAUNCH(k_root_jobs<<<g_seg128, 128, 0, g.s>>>(r, ja, exact_pass));
    PKD_LAUNCH(k_job_advance<<<1, 1024, 0, g.s>>>(bb.jcur, bb.jnext, dctr, (uint32_t)bb.big_jobs, t.st));
    PKD_TRY(flow_while(g, C_JGO, job_level));
    SmemArgs ka = sa;
    ka.jobs = bb.jsmall;
    ka.njobs = dctr + C_JSMALL;
    ka.list_cap = (uint32_t)bb.small_jobs;
    ka.grab = dctr + C_GRAB;
    ka.cap = scap;
    const size_t smb = smem_layout(ka.cap, d).total;
    PKD_DISPATCH_D(d, launch_smem_skel, ka, (uint32_t)nsm, smb, g.s);
    return PKD_OK;
  };

  auto round = [&](Flow& g) {
    cudaStream_t q = g.s;
    const uint64_t pts_big = g.graph ? 0 : *(unsigned long long*)(g.hctl + C_PTS);
    PKD_LAUNCH(k_round_clear<<<g_clear, 256, 0, q>>>(r));
    PKD_LAUNCH(k_big_prefix<<<1, 1024, 0, q>>>(bb.big, dctr + C_NBIG, (uint32_t)TILE, bb.tile0, bb.excl));
    {
      KTimer kt;
      ktimer_begin(kt, "sample", pts_big, q);
      PKD_LAUNCH(k_sample<<<g_sample, SAMPLE_THREADS, 0, q>>>(r, 0));
      ktimer_end(kt);
    }
    PKD_TRY(skeleton_pass(g, 0));
    // segments whose skeleton root is a bucket take one exact level on their own points
    PKD_LAUNCH(k_mark_exact<<<g_seg128, 128, 0, q>>>(r, dctr + C_EXACT));
    PKD_TRY(flow_if(g, C_EXACT, [&](Flow& h) { return skeleton_pass(h, 1); }));
    PKD_LAUNCH(k_finalize<<<grid_for(bb.nbig * 32, FIN_WARPS * 32, 8), FIN_WARPS * 32, 0, q>>>(r));
    PKD_DISPATCH_D(d, launch_count, r, (uint32_t)bb.tiles, pts_big, "count", q);
    device_excl_scan_dev(bb.hist, bb.hscan, dctr + C_TILES, (uint32_t)NB, bb.tiles * NB, bb.partial, q);
    PKD_LAUNCH(k_emit<<<grid_for(bb.nbig * 32, 128, 8), 128, 0, q>>>(r, dctr + C_HEAVY));
    PKD_DISPATCH_D(d, launch_scatter, r, (uint32_t)bb.tiles, pts_big, "scatter", q);
    PKD_LAUNCH(k_copy_heavy<<<g_tiles, 256, 0, q>>>(r, 0, dctr + C_HEAVY));
    // the buckets, now in the destination buffer, are the next round
    PKD_LAUNCH(k_round_next<<<1, 1, 0, q>>>(dctr, (uint32_t)NB));
    return classify(g);
  };

  // 5. every small subproblem, in shared memory, one CTA (or warp) per
  //    entry of the base lists: `q` is the stream, `list_blocks(w, per,
  //    max)` the grid of the list whose length is control word w.
  auto base_stage = [&](cudaStream_t q, cudaStream_t aux, auto&& list_blocks, auto&& recorded) {
    const uint64_t cta_pts = *(unsigned long long*)(hctr + C_BASE_PTS);
    const uint64_t warp_pts = *(unsigned long long*)(hctr + C_BASE_PTS + 2);
    const uint64_t tiny_pts = *(unsigned long long*)(hctr + C_BASE_PTS + 4);
    for (int pass = 0; pass < 2; ++pass) {
      SmemArgs wa = sa;
      const int w = pass == 0 ? C_NWBASE : C_NTBASE;
      wa.segs = pass == 0 ? wbase_list : tbase_list;
      wa.nsegs = dctr + w;
      wa.list_cap = (uint32_t)base_cap_segs;
      wa.cap = pass == 0 ? (int)wcap : (int)tcap;
      const size_t smb = warp_layout(wa.cap, d).per_warp * WK_WARPS;
      const uint32_t blocks = list_blocks(w, WK_WARPS, (uint32_t)(nsm * 8));
      if (blocks == 0) continue;
      KTimer kt;
      ktimer_begin(kt, "smem_warp", pass == 0 ? warp_pts : tiny_pts, q);
      PKD_DISPATCH_D(d, launch_smem_warp, wa, blocks, smb, q);
      ktimer_end(kt);
      PKD_TRY(recorded(q, w, (uint32_t)WK_WARPS, (uint32_t)(nsm * 8)));
    }
    KTimer kt;
    ktimer_begin(kt, "smem_build", cta_pts, q);
    if (knobs().base_kernel == 0) {
      // the one-CTA-per-SM segments run beside the two-CTA launch, on a
      // second stream, so their long CTAs do not form a tail of their own
      cudaEvent_t fork = nullptr, join = nullptr;
      PKD_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
      PKD_CUDA(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
      PKD_CUDA(cudaEventRecord(fork, q));
      PKD_CUDA(cudaStreamWaitEvent(aux, fork, 0));
      SmemArgs s1 = sa;
      s1.segs = bbase_list;
      s1.nsegs = dctr + C_NBBASE;
      s1.list_cap = (uint32_t)base_cap_segs;
      s1.cap = (int)cap;
      const uint32_t b1 = list_blocks(C_NBBASE, 1, 0);
      if (b1) {
        PKD_DISPATCH_D(d, launch_smem_sorted, s1, b1, sorted_layout((int)cap, d).total, aux);
        PKD_TRY(recorded(aux, C_NBBASE, 1u, 0u));
      }
      SmemArgs s2 = sa;
      s2.segs = base_list;
      s2.nsegs = dctr + C_NBASE;
      s2.list_cap = (uint32_t)base_cap_segs;
      s2.cap = (int)cap2;
      const uint32_t b2 = list_blocks(C_NBASE, 1, 0);
      if (b2) {
        PKD_DISPATCH_D(d, launch_smem_sorted2, s2, b2, sorted_layout((int)cap2, d).total, q);
        PKD_TRY(recorded(q, C_NBASE, 1u, 0u));
      }
      PKD_CUDA(cudaEventRecord(join, aux));
      PKD_CUDA(cudaStreamWaitEvent(q, join, 0));
      cudaEventDestroy(fork);
      cudaEventDestroy(join);
    } else {
      SmemArgs s2 = sa;
      s2.segs = base_list;
      s2.nsegs = dctr + C_NBASE;
      s2.list_cap = (uint32_t)base_cap_segs;
      s2.cap = (int)cap;
      const uint32_t b2 = list_blocks(C_NBASE, 1, 0);
      if (b2) {
        PKD_DISPATCH_D(d, launch_smem_build, s2, b2, smem_layout((int)cap, d).total, q);
        PKD_TRY(recorded(q, C_NBASE, 1u, 0u));
      }
    }
    ktimer_end(kt);
    return PKD_OK;
  };

  PKD_LAUNCH(k_ctl_init<<<1, 64, 0, s>>>(dctr, (uint32_t)nroots));
  if (!graph) {
    PKD_TRY(classify(f));
    PKD_TRY(flow_while(f, C_GO, round));
    // the counts come back once more: every list gets its exact grid
    PKD_TRY(flow_read(f));
    if (job.before_base) job.before_base(nullptr);
    auto host_blocks = [&](int w, uint32_t per, uint32_t mx) {
      const uint32_t c = (uint32_t)std::min<uint64_t>(hctr[w], base_cap_segs);
      const uint32_t b = (c + per - 1) / per;
      return mx ? std::min(b, mx) : b;
    };
    auto none = [](cudaStream_t, int, uint32_t, uint32_t) { return PKD_OK; };
    PKD_TRY(base_stage(s, aux_stream(), host_blocks, none));
  } else {
    // One graph: WHILE(another round) { ... WHILE(another skeleton level)
    // { ... } ... IF(exact levels) { ... } ... }, then the base cases as
    // device-updatable kernel nodes whose grids k_base_shapes sets from the
    // lists' lengths (a node with an empty list is disabled).
    std::lock_guard<std::mutex> lk(flow_mutex());
    const auto rec0 = std::chrono::steady_clock::now();
    cudaStream_t cs = flow_stream(0);
    if (!cs) return PKD_ECUDA;
    BaseShape* dshape;
    PKD_TRY(sc.get(&dshape, MAX_SHAPES));
    PinnedBlock shblk(s);
    if (!shblk.p) return PKD_ENOMEM;
    static_assert(MAX_SHAPES * sizeof(BaseShape) <= PINNED_BLOCK, "shape block");
    BaseShape* hshape = (BaseShape*)shblk.p;

    // every value the recorded kernels take as an argument
    std::vector<uint64_t> key;
    {
      auto put = [&](uint64_t v) { key.push_back(v); };
      auto putp = [&](const void* q) { key.push_back((uint64_t)(uintptr_t)q); };
      int dev = 0;
      cudaGetDevice(&dev);
      put((uint64_t)dev);
      for (void* q : sc.ptrs) putp(q);  // every scratch buffer, in allocation order
      putp(t.A.c), putp(t.A.id), put(t.A.stride), putp(t.nodes), putp(t.ndim), putp(t.st), putp(t.shared_next);
      put(t.shared_cap);
      putp(job.input_coords), putp(job.input_ids), put(job.base), put(job.extent), putp(roots), put(nroots);
      put((uint64_t)p.d), put((uint64_t)p.phi), put((uint64_t)p.lambda), put((uint64_t)p.sigma_log2);
      put((uint64_t)p.sigma_os), put((uint64_t)p.count_mode), put((uint64_t)p.alpha_num), put((uint64_t)p.alpha_den);
      put(p.seed);
      put((uint64_t)TILE), put(cap), put((uint64_t)scap), put(cap2), put(wcap), put((uint64_t)nsm);
      put((uint64_t)knobs().sieve_kernel), put((uint64_t)knobs().base_kernel), put((uint64_t)knobs().wait_cycles);
      put((uint64_t)record_buckets(NB));
    }
    graph_reap();
    GraphEntry* ent = graph_find(key);
    if (ent) {
      memcpy(hshape, ent->shapes, sizeof(ent->shapes));
      PKD_TRY(dev_store(dshape, hshape, sizeof(ent->shapes), s));
      PKD_CUDA(cudaGraphLaunch(ent->exec, s));
      PKD_CUDA(cudaEventRecord(ent->done, s));
      ++g_graph_builds;
      ++g_graph_reuses;
      stat_host_ms("graph_record",
                   std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - rec0).count(), 0);
      if (job.before_base) job.before_base(ent->base);
      PKD_CUDA(cudaGetLastError());
      return PKD_OK;
    }

    int nshape = 0;
    cudaGraphNode_t shape_nodes[MAX_SHAPES] = {};
    cudaEvent_t ready = nullptr, done = nullptr, base_ev = nullptr;
    PKD_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    PKD_CUDA(cudaEventCreateWithFlags(&base_ev, cudaEventDisableTiming));
    // the capture stream starts after the work queued so far on s
    PKD_CUDA(cudaEventRecord(ready, s));
    PKD_CUDA(cudaStreamWaitEvent(cs, ready, 0));
    cudaEventDestroy(ready);
    PKD_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    flow_capturing() = true;
    Flow g = f;
    g.s = cs;
    g.graph = true;
    int e = classify(g);
    if (e == PKD_OK) e = flow_while(g, C_GO, round);
    if (e == PKD_OK) {
      PKD_LAUNCH(k_base_shapes<<<1, 32, 0, cs>>>(dshape, MAX_SHAPES));
      if (cudaEventRecordWithFlags(base_ev, cs, cudaEventRecordExternal) != cudaSuccess) e = PKD_ECUDA;
    }
    auto dev_blocks = [](int, uint32_t, uint32_t) { return 1u; };  // placeholders
    auto record_shape = [&](cudaStream_t q, int w, uint32_t per, uint32_t mx) {
      if (nshape >= MAX_SHAPES) return PKD_EINTERNAL;
      shape_nodes[nshape] = last_node(q);
      if (!shape_nodes[nshape]) return PKD_ECUDA;
      hshape[nshape] = BaseShape{nullptr, dctr + w, (uint32_t)base_cap_segs, per, mx, 0};
      ++nshape;
      return PKD_OK;
    };
    if (e == PKD_OK) e = base_stage(cs, aux_stream(), dev_blocks, record_shape);
    flow_capturing() = false;
    cudaGraph_t graph_h = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph_h);
    if (e == PKD_OK && ce != cudaSuccess) e = PKD_ECUDA;
    // the recorded base-case nodes become device-updatable (the shape
    // kernel walks MAX_SHAPES entries: unused ones repeat the first update)
    for (int k = 0; e == PKD_OK && k < nshape; ++k) {
      hshape[k].node = make_updatable(shape_nodes[k]);
      if (!hshape[k].node) e = PKD_ECUDA;
    }
    if (e == PKD_OK && nshape == 0) e = PKD_EINTERNAL;
    for (int k = nshape; e == PKD_OK && k < MAX_SHAPES; ++k) hshape[k] = hshape[0];
    cudaGraphExec_t exec = nullptr;
    if (e == PKD_OK) e = dev_store(dshape, hshape, MAX_SHAPES * sizeof(BaseShape), s);
    if (e == PKD_OK && cudaGraphInstantiate(&exec, graph_h, 0) != cudaSuccess) e = PKD_ECUDA;
    if (e == PKD_OK && cudaGraphUpload(exec, s) != cudaSuccess) e = PKD_ECUDA;
    if (e == PKD_OK && cudaGraphLaunch(exec, s) != cudaSuccess) e = PKD_ECUDA;
    if (e == PKD_OK && cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) e = PKD_ECUDA;
    if (e == PKD_OK && cudaEventRecord(done, s) != cudaSuccess) e = PKD_ECUDA;
    if (e != PKD_OK) {
      cudaGetLastError();
      cudaStreamSynchronize(s);
      if (exec) cudaGraphExecDestroy(exec);
      if (graph_h) cudaGraphDestroy(graph_h);
      if (done) cudaEventDestroy(done);
      cudaEventDestroy(base_ev);
      return e;
    }
    ent = graph_slot();
    ent->key = std::move(key);
    ent->exec = exec;
    ent->graph = graph_h;
    ent->done = done;
    ent->base = base_ev;
    memcpy(ent->shapes, hshape, sizeof(ent->shapes));
    ent->used = ++g_graph_clock;
    ++g_graph_builds;
    stat_host_ms("graph_record",
                 std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - rec0).count(), 1);
    // work that overlaps the base cases starts at the graph's event
    if (job.before_base) job.before_base(base_ev);
  }
  PKD_CUDA(cudaGetLastError());
  return PKD_OK;
}

int graph_builds() { return g_graph_builds; }
int graph_reuses() { return g_graph_reuses; }

}  // namespace pkd
