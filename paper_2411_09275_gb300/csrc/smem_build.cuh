// One CTA finishes a whole subproblem in shared memory (the base case of
// Alg. 1: "the base case fits into the cache"), and the same frame builds
// the skeleton of a sample that fits in shared memory.
//
// Points stay where they were loaded; only 16-bit index lists move.  A task
// is one node: either the root of a Build(P, t) call (j == 0) or a skeleton
// node at local depth j whose sample is the flagged subset of its points.
// Because the sample of every skeleton node below a Build root is drawn at
// that root's depth, one flag byte per point serves all its skeleton levels,
// and partitioning the points level by level yields exactly the buckets a
// sieve over the finished skeleton would (shared-memory traffic is cheap, so
// the sieve's one-pass data movement buys nothing here).
//
// Scheduling: the root task is processed by all 16 warps of the CTA; at
// every split the team halves and each half takes one child (a child much
// smaller than its sibling is deferred to the stack of the team's first warp
// instead), down to single warps, which finish their subtrees depth first
// with a stack that always continues with the smaller child (so it stays
// within log2(cap) entries).  Teams synchronise on their own named barrier.
#pragma once

#include "team.cuh"

namespace pkd {

constexpr int SM_NW = 16;
constexpr int SM_THREADS = SM_NW * 32;
constexpr int WSTK = 32;
constexpr int DEFER_MAX = 96;  // children this small are deferred instead of splitting a team

struct Task {
  uint16_t lo, hi, ns;
  uint8_t buf, j;
  uint32_t t;     // tree depth of this node (build mode) / unused
  uint32_t slot;  // node slot (build mode) / heap index (skeleton mode)
};
static_assert(sizeof(Task) == 16, "Task layout");

struct SmemCtl {
  int next_slot;
  unsigned maxd;   // deepest leaf written by this CTA (or warp)
  int wsp[SM_NW];  // per-warp stack depth
};

// A skeleton node whose sample is still to be split: the node at heap index
// h of segment `seg`, with n samples at a.. in sample buffer `buf`.
struct SkelJob {
  uint32_t seg;
  uint32_t h;
  uint64_t a;
  uint32_t n;
  uint8_t buf, j, lam, pad;
  uint32_t min_split;  // split only with at least this many samples
  uint32_t pad2;
};
static_assert(sizeof(SkelJob) == 32, "SkelJob layout");

// Heap skeleton entry: split value and meta = state | dim << 8 | bucket << 16.
enum SkState : int { SK_NONE = 0, SK_INTERNAL = 1, SK_BUCKET = 2, SK_HEAVY = 3 };
__host__ __device__ __forceinline__ int sk_meta(int state, int dim, int bucket) {
  return state | (dim << 8) | (bucket << 16);
}
__host__ __device__ __forceinline__ int sk_state(int meta) { return meta & 0xFF; }
__host__ __device__ __forceinline__ int sk_dim(int meta) { return (meta >> 8) & 0xFF; }
__host__ __device__ __forceinline__ int sk_bucket(int meta) { return (meta >> 16) & 0xFFFF; }

// Arguments of the shared-memory kernels.
struct SmemArgs {
  Params p;
  int cap;  // point capacity of the shared arrays
  // build mode
  Pts A, B;
  const int32_t* in_coords;  // point-major input for IN_INPUT
  const uint32_t* in_ids;    // NULL -> ids are input positions
  Node* nodes;
  uint8_t* ndim;
  const Seg* segs;
  const uint32_t* nsegs;  // device count of segs
  // skeleton mode
  const SkelJob* jobs;
  const uint32_t* njobs;
  const int32_t* sbuf[2];  // sample coordinate buffers (SoA, stride = sstride)
  uint64_t sstride;
  int2* skel;              // [seg][heap]
  int heap_n;              // 2^(lambda+1)
  uint64_t shared_cap;     // first per-position node slot
  DevStatus* st;
  uint32_t list_cap;       // entries segs / jobs can hold (bounds the device count)
  uint32_t* grab;          // persistent launches: next entry to take (zeroed before the launch)
};

struct SmemLayout {
  size_t X, ID, perm0, perm1, flag, whist, wred, wstack, ctl, total;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Shared memory of one CTA with `warps` warps holding up to `cap` points.
__host__ __device__ inline SmemLayout smem_layout(int cap, int d, int warps = SM_NW) {
  SmemLayout L;
  size_t o = 0;
  L.X = o;
  o = align_up(o + (size_t)4 * d * cap, 16);
  L.ID = o;
  o = align_up(o + (size_t)4 * cap, 16);
  L.perm0 = o;
  o = align_up(o + (size_t)2 * cap, 16);
  L.perm1 = o;
  o = align_up(o + (size_t)2 * cap, 16);
  L.flag = o;
  o = align_up(o + (size_t)cap, 16);
  L.whist = o;
  o = align_up(o + (size_t)warps * 256 * 4, 16);
  L.wred = o;
  o = align_up(o + (size_t)warps * RED_INTS * 4, 16);
  L.wstack = o;
  o = align_up(o + (size_t)warps * WSTK * sizeof(Task), 16);
  L.ctl = o;
  o = align_up(o + sizeof(SmemCtl), 16);
  L.total = o;
  return L;
}

template <int D>
struct SmemCtx {
  Params p;
  SmemPts<D> s;
  uint8_t* flag;
  uint16_t* perm[2];
  SmemCtl* ctl;
  // build mode
  Pts out;
  uint64_t start;
  uint32_t slot_base;
  int slot_limit;
  Node* nodes;
  uint8_t* ndim;
  // skeleton mode
  int2* skel;  // this segment's heap
  int lam;
  int min_split;
  DevStatus* st;
};

// ---------------------------------------------------------------------------
// Build mode
// ---------------------------------------------------------------------------

template <int D>
__device__ __forceinline__ void emit_leaf(const Team& tm, const SmemCtx<D>& cx, const Task& tk) {
  const uint16_t* P = cx.perm[tk.buf];
  for (int i = tk.lo + tm.rank(); i < tk.hi; i += tm.size()) {
    const int p = P[i];
    const uint64_t g = cx.start + (uint64_t)i;
#pragma unroll
    for (int j = 0; j < D; ++j) cx.out.c[(uint64_t)j * cx.out.stride + g] = cx.s.x(j, p);
    cx.out.id[g] = cx.s.ID[p];
  }
  if (tm.leader()) {
    Node nd;
    nd.split = 0;
    nd.size = (uint32_t)(tk.hi - tk.lo);
    nd.a = (uint32_t)(cx.start + tk.lo);
    nd.b = 0;
    cx.nodes[tk.slot] = nd;
    cx.ndim[tk.slot] = PKD_LEAF;
    atomicMax(&cx.ctl->maxd, tk.t);  // published once per CTA / warp
  }
}

// A Build root of at most 128 points handled by one warp entirely in
// registers (each lane holds up to 4 points): min/max, the sample count,
// the element of rank floor(n/2) by broadcast rank counting, and the stable
// partition by ballots.  Returns -1 when the rules call for a skeleton split
// on the sample (the generic path then takes over), otherwise the number of
// children like process_build.
constexpr int REG_MAX = 128;

template <int D>
__device__ __forceinline__ int warp_small_build(const Team& tm, const SmemCtx<D>& cx, const Task& tk, Task* ch) {
  constexpr int Q = REG_MAX / 32;
  const int lane = lane_id();
  const int lo = tk.lo, hi = tk.hi, n = hi - lo;
  const uint16_t* P = cx.perm[tk.buf];
  uint16_t* Qp = cx.perm[tk.buf ^ 1];
  int p[Q];
  int32_t x[Q][D];
  bool valid[Q];
  int mn[D], mx[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    mn[j] = INT32_MAX;
    mx[j] = INT32_MIN;
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int i = lo + q * 32 + lane;
    valid[q] = i < hi;
    p[q] = valid[q] ? P[i] : 0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      x[q][j] = valid[q] ? cx.s.x(j, p[q]) : 0;
      if (valid[q]) {
        mn[j] = min(mn[j], x[q][j]);
        mx[j] = max(mx[j], x[q][j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < D; ++j) {
    mn[j] = warp_min(mn[j]);
    mx[j] = warp_max(mx[j]);
  }
  int vmin, vmax;
  const int wd = widest_dim<D>(mn, mx, vmin, vmax);
  if (wd < 0) {  // heavy leaf
    emit_leaf<D>(tm, cx, tk);
    return 0;
  }
  if (n >= 2 * cx.p.sigma_os) {
    // draw the sample; with enough samples the node is a skeleton node
    const int shift = sample_shift(cx.p, (uint64_t)n);
    int ns = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const bool f = valid[q] && in_sample(cx.p.seed, tk.t, cx.s.ID[p[q]], shift);
      if (valid[q]) cx.flag[p[q]] = f;
      ns += __popc(__ballot_sync(FULL_MASK, f));
    }
    __syncwarp();
    if (ns >= 2 * cx.p.sigma_os) return -1;
  }
  // element of rank k = floor(n/2) on dimension wd
  int key[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    int v = x[q][0];
#pragma unroll
    for (int j = 1; j < D; ++j)
      if (j == wd) v = x[q][j];
    key[q] = valid[q] ? v : INT32_MAX;
  }
  int less[Q], leq[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) less[q] = leq[q] = 0;
#pragma unroll
  for (int qs = 0; qs < Q; ++qs) {
    if (qs * 32 >= n) break;
    for (int sl = 0; sl < 32; ++sl) {
      const int v = __shfl_sync(FULL_MASK, key[qs], sl);
      const bool ok = qs * 32 + sl < n;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        less[q] += ok && v < key[q];
        leq[q] += ok && v <= key[q];
      }
    }
  }
  const int k = n / 2;
  int cand = INT32_MAX, cless = 0;
#pragma unroll
  for (int q = 0; q < Q; ++q)
    if (valid[q] && less[q] <= k && k < leq[q]) {
      cand = key[q];
      cless = less[q];
    }
  int xsplit = warp_min(cand);
  int count_less = warp_max(cand == xsplit ? cless : -1);
  if (count_less == 0) {  // nothing strictly below: the next distinct value
    int m = INT32_MAX;
#pragma unroll
    for (int q = 0; q < Q; ++q)
      if (valid[q] && key[q] > xsplit) m = min(m, key[q]);
    xsplit = warp_min(m);
  }
  // stable partition: left (key < xsplit) first, original order kept
  int L = 0;
#pragma unroll
  for (int q = 0; q < Q; ++q) L += __popc(__ballot_sync(FULL_MASK, valid[q] && key[q] < xsplit));
  int lpos = lo, rpos = lo + L;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const bool left = valid[q] && key[q] < xsplit;
    const unsigned bl = __ballot_sync(FULL_MASK, left);
    const unsigned br = __ballot_sync(FULL_MASK, valid[q] && !left);
    if (left) Qp[lpos + __popc(bl & lanemask_lt())] = (uint16_t)p[q];
    else if (valid[q]) Qp[rpos + __popc(br & lanemask_lt())] = (uint16_t)p[q];
    lpos += __popc(bl);
    rpos += __popc(br);
  }
  __syncwarp();
  int b = 0;
  if (lane == 0) b = atomicAdd(&cx.ctl->next_slot, 2);
  b = __shfl_sync(FULL_MASK, b, 0);
  if (b + 2 > cx.slot_limit || L <= 0 || L >= n) {
    if (lane == 0) set_error(cx.st, b + 2 > cx.slot_limit ? DERR_SLOT : DERR_STATE, 150 + L);
    return 0;
  }
  const uint32_t sl = cx.slot_base + (uint32_t)b, sr = sl + 1;
  if (lane == 0) {
    cx.nodes[tk.slot] = Node{xsplit, (uint32_t)n, sl, sr};
    cx.ndim[tk.slot] = (uint8_t)wd;
  }
  const uint8_t nb = (uint8_t)(tk.buf ^ 1);
  ch[0] = Task{(uint16_t)lo, (uint16_t)(lo + L), 0, nb, 0, tk.t + 1, sl};
  ch[1] = Task{(uint16_t)(lo + L), (uint16_t)hi, 0, nb, 0, tk.t + 1, sr};
  return 2;
}

// Process one node; returns the number of children written to ch (0 or 2).
template <int D>
__device__ int process_build(const Team& tm, const SmemCtx<D>& cx, Task tk, Task* ch) {
  for (;;) {
    const int lo = tk.lo, hi = tk.hi, n = hi - lo;
    if (tm.nw == 1 && tk.j == 0 && n > cx.p.phi && n <= REG_MAX) {
      const int r = warp_small_build<D>(tm, cx, tk, ch);
      if (r >= 0) return r;
    }
    uint16_t* P = cx.perm[tk.buf];
    uint16_t* Q = cx.perm[tk.buf ^ 1];
    int dim = 0, x = 0;
    bool on_sample;
    if (tk.j == 0) {
      // Build(P, t): leaf wrap, heavy leaf, then sample and skeleton root.
      if (n <= cx.p.phi) {
        emit_leaf<D>(tm, cx, tk);
        return 0;
      }
      int mn[D], mx[D];
      team_minmax<D>(tm, cx.s, P, lo, hi, false, mn, mx);
      int vmin, vmax;
      const int wd = widest_dim<D>(mn, mx, vmin, vmax);
      if (wd < 0) {
        emit_leaf<D>(tm, cx, tk);
        return 0;
      }
      // A subproblem with fewer than 2*sigma_os points cannot reach the
      // split threshold whatever its sample: no need to draw it.
      int ns = 0;
      if (n >= 2 * cx.p.sigma_os) {
        const int shift = sample_shift(cx.p, (uint64_t)n);
        ns = team_draw_sample<D>(tm, cx.s, cx.flag, P, lo, hi, cx.p.seed, tk.t, shift);
      }
      tk.ns = (uint16_t)ns;
      bool skel = false;
      if (ns >= 2 * cx.p.sigma_os)
        skel = team_split_rule<D>(tm, cx.s, P, lo, hi, true, ns, nullptr, nullptr, dim, x);
      if (skel) {
        on_sample = true;
      } else {
        // Too few (or identical) samples: one exact level on P itself.
        on_sample = false;
        dim = wd;
        int less, eq;
        x = team_select<D>(tm, cx.s, P, lo, hi, false, dim, n / 2, vmin, vmax, less, eq);
        if (less == 0) x = team_min_above<D>(tm, cx.s, P, lo, hi, false, dim, x);
      }
    } else {
      // Skeleton node: bucket when deep enough, too few samples or identical.
      if (tk.j >= cx.p.lambda || tk.ns < 2 * cx.p.sigma_os) {
        tk.j = 0;
        continue;
      }
      if (!team_split_rule<D>(tm, cx.s, P, lo, hi, true, tk.ns, nullptr, nullptr, dim, x)) {
        tk.j = 0;
        continue;
      }
      on_sample = true;
    }
    int L, SL, SR;
    team_partition<D>(tm, cx.s, P, Q, lo, hi, dim, x, L, SL, SR);
    int b = 0;
    if (tm.leader()) b = atomicAdd(&cx.ctl->next_slot, 2);
    b = tm.bcast(b);
    if (b + 2 > cx.slot_limit) {
      if (tm.leader()) set_error(cx.st, DERR_SLOT, b);
      return 0;
    }
    if (L <= 0 || L >= n) {
      if (tm.leader()) set_error(cx.st, DERR_STATE, 100 + L);
      return 0;
    }
    const uint32_t sl = cx.slot_base + (uint32_t)b, sr = sl + 1;
    if (tm.leader()) {
      Node nd;
      nd.split = x;
      nd.size = (uint32_t)n;
      nd.a = sl;
      nd.b = sr;
      cx.nodes[tk.slot] = nd;
      cx.ndim[tk.slot] = (uint8_t)dim;
    }
    const uint8_t nj = on_sample ? (uint8_t)(tk.j + 1) : (uint8_t)0;
    const uint8_t nb = (uint8_t)(tk.buf ^ 1);
    ch[0] = Task{(uint16_t)lo, (uint16_t)(lo + L), (uint16_t)SL, nb, nj, tk.t + 1, sl};
    ch[1] = Task{(uint16_t)(lo + L), (uint16_t)hi, (uint16_t)SR, nb, nj, tk.t + 1, sr};
    return 2;
  }
}

// ---------------------------------------------------------------------------
// Skeleton mode: every loaded point is a sample; nodes become heap entries.
// ---------------------------------------------------------------------------

template <int D>
__device__ int process_skel(const Team& tm, const SmemCtx<D>& cx, Task tk, Task* ch) {
  const int lo = tk.lo, hi = tk.hi, n = hi - lo;
  uint16_t* P = cx.perm[tk.buf];
  uint16_t* Q = cx.perm[tk.buf ^ 1];
  int dim, x;
  const bool split = tk.j < cx.lam && n >= cx.min_split &&
                     team_split_rule<D>(tm, cx.s, P, lo, hi, false, n, nullptr, nullptr, dim, x);
  if (!split) {
    if (tm.leader()) cx.skel[tk.slot] = make_int2(0, sk_meta(SK_BUCKET, 0, 0));
    return 0;
  }
  int L, SL, SR;
  team_partition<D>(tm, cx.s, P, Q, lo, hi, dim, x, L, SL, SR);
  if (tm.leader()) cx.skel[tk.slot] = make_int2(x, sk_meta(SK_INTERNAL, dim, 0));
  const uint8_t nb = (uint8_t)(tk.buf ^ 1);
  const uint8_t nj = (uint8_t)(tk.j + 1);
  ch[0] = Task{(uint16_t)lo, (uint16_t)(lo + L), 0, nb, nj, 0, 2 * tk.slot};
  ch[1] = Task{(uint16_t)(lo + L), (uint16_t)hi, 0, nb, nj, 0, 2 * tk.slot + 1};
  return 2;
}

template <bool SKEL, int D>
__device__ __forceinline__ int process_task(const Team& tm, const SmemCtx<D>& cx, const Task& tk, Task* ch) {
  if (SKEL) return process_skel<D>(tm, cx, tk, ch);
  return process_build<D>(tm, cx, tk, ch);
}

// One warp finishes its subtree depth first; `stk` holds sp0 deferred tasks.
template <bool SKEL, int D>
__device__ void warp_run(const Team& wt, const SmemCtx<D>& cx, Task tk, Task* stk, int sp0) {
  int sp = sp0;
  for (int iter = 1;; ++iter) {
    Task ch[2];
    const int nch = process_task<SKEL, D>(wt, cx, tk, ch);
    if ((iter & 63) == 0) {  // another CTA's failure ends this one early
      const int err = *(volatile int*)&cx.st->err;
      if (__shfl_sync(FULL_MASK, err, 0)) return;  // warp-uniform exit
    }
    if (nch == 2) {
      const int s0 = ch[0].hi - ch[0].lo, s1 = ch[1].hi - ch[1].lo;
      const Task big = s0 >= s1 ? ch[0] : ch[1];
      const Task small = s0 >= s1 ? ch[1] : ch[0];
      if (sp >= WSTK) {
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

// Drive the warps of a CTA over one root task (see the scheduling note at
// the top).  Every branch below is uniform within the team that takes it.
template <bool SKEL, int D>
__device__ void run_team_tasks(const SmemCtx<D>& cx, Task root, unsigned* whist, int* wred, Task* wstack,
                               int cta_warps) {
  const int w = warp_id();
  int f = 0, nw = cta_warps;
  Task tk = root;
  bool have_task = true;
  while (nw > 1) {
    const Team tm{f, nw, team_barrier(f, nw, cta_warps), whist + f * 256, wred + f * RED_INTS};
    Task ch[2];
    const int nch = process_task<SKEL, D>(tm, cx, tk, ch);
    if (nch == 0) {  // this team's subtree is finished (deferred tasks remain)
      have_task = false;
      break;
    }
    const int s0 = ch[0].hi - ch[0].lo, s1 = ch[1].hi - ch[1].lo;
    const int big = s0 >= s1 ? 0 : 1;
    const int small_n = min(s0, s1);
    // a tiny child goes to the first warp's stack; the team keeps the other
    tm.sync();
    const bool defer = small_n <= DEFER_MAX && small_n * 8 <= max(s0, s1) && cx.ctl->wsp[f] < WSTK;
    tm.sync();
    if (defer) {
      if (tm.leader()) {
        wstack[f * WSTK + cx.ctl->wsp[f]] = ch[big ^ 1];
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
    tk = wstack[w * WSTK + --sp0];
  }
  __syncwarp();
  const Team wt{w, 1, 0, whist + w * 256, wred + w * RED_INTS};
  warp_run<SKEL, D>(wt, cx, tk, wstack + w * WSTK, sp0);
}

}  // namespace pkd
