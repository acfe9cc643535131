// Batch updates of a Pkd-tree: BatchInsert (Alg. 2, Sec. 4.1) and the
// two-round BatchDelete (Sec. 4.2).
//
//  route    the batch is sieved through the tree lambda levels at a time: the
//           "skeleton at T" is fetched from the existing nodes (cut at
//           leaves), and the same count / scan / scatter kernels as the build
//           move every batch point to its external node.  Internal external
//           nodes become the next round's items; leaves collect "leaf groups".
//  match    (delete only) every stored point of a reached leaf is compared
//           with the batch points routed there; matches are marked dead and
//           points that match nothing are discarded (round 1 of Sec. 4.2).
//  count    exact per-node counts of inserted / deleted points, aggregated
//           bottom-up over the recorded skeletons.
//  decide   top-down over every skeleton: a node that receives updates stays
//           (its size is rewritten in place) when it is still alpha-balanced,
//           otherwise it is rebuilt with Build on all its (live) points plus
//           the new ones, and nothing below it is looked at.  A reached leaf
//           is rebuilt (insert: Build(leaf + new)) or compacted (delete).
//  rebuild  old subtrees are flattened by a parallel breadth-first walk into
//           fresh arena ranges, new points appended, and every rebuild item
//           becomes a root segment of one multi-segment build (build.cu).
#include <algorithm>
#include <cstdio>
#include <vector>

#include "sieve_tma.cuh"
#include "tree_impl.hpp"

namespace pkd {

constexpr uint32_t LINK_NONE = 0xFFFFFFFFu;
constexpr uint32_t LINK_LEAF = 0x80000000u;

struct LeafGroup {
  uint32_t slot;   // the leaf's node slot
  uint32_t depth;  // its tree depth
  uint64_t start;  // first routed batch point (position in the batch buffers)
  uint32_t len;    // routed batch points
  uint32_t found;  // insert: len; delete: stored points removed
  uint32_t flag;   // 1: inside a subtree that is rebuilt
  uint32_t pad;
};

struct RebuildItem {
  uint32_t slot;
  uint32_t depth;
  uint32_t size;    // points after the update
  uint32_t old_live;
  uint64_t ws, we;  // batch points (insert) in the final batch buffer
  uint64_t pos;     // arena position assigned
};

struct UpdArgs {
  Params p;
  int lam, NB, HN, TILE;
  int insert;
  const Node* nodes;
  const uint8_t* ndim;
  // this round
  const Seg* items;
  const uint32_t* nitems;
  int2* skel;
  uint32_t* slots;
  uint32_t* nbk;
  const uint32_t* tile0;
  const uint32_t* hscan;
  uint64_t* bstart;  // [item][NB]
  uint32_t* blen;    // [item][NB]
  uint32_t* link;    // [item][NB]
  uint32_t* fnd;     // [item][HN]
  uint32_t* nsz;     // [item][HN] new size of a node that stays, or ~0 (applied at the end)
  uint32_t* iflag;   // [item]
  // next round
  Seg* next;
  uint32_t* next_ctr;  // [0] items, [1] tiles of big items, [2] big items, [3] small items,
                       // [16] points of the big items
  Seg* next_big;       // big items (more than SMALL_ITEM points) and their item index
  uint32_t* next_bigmap;
  uint32_t* next_small;  // item index of the small items
  uint32_t* next_iflag;
  const uint32_t* next_fnd;  // found counts of the next round (aggregation)
  int next_HN;
  // leaf groups
  LeafGroup* groups;
  uint32_t* ngroups;
  uint32_t group_cap;
  // rebuild items
  RebuildItem* items_out;
  uint32_t* nitems_out;
  unsigned long long* items_total;
  uint32_t items_cap;
  uint32_t* aux;  // [node slot] deleted points below (delete only)
  DevStatus* st;
};

// The per-item kernels (fetch, emit, aggregate, decide) give each item one
// warp, whose lanes take the heap entries of one skeleton level at a time
// (levels are ordered by __syncwarp); each CTA holds ITEM_WARPS items.
constexpr int ITEM_WARPS = 4;
__host__ __device__ inline unsigned item_blocks(uint64_t n) { return (unsigned)((n + ITEM_WARPS - 1) / ITEM_WARPS); }
__device__ __forceinline__ uint32_t item_of_warp() { return blockIdx.x * ITEM_WARPS + warp_id(); }

// The skeleton at each item: its node and lambda levels below, cut at leaves;
// the external nodes are numbered left to right (the item's buckets).
// The skeleton is assembled in shared memory (one level's node loads in
// flight at a time, both of a node's records at once) and written out at
// the end.
__global__ void __launch_bounds__(ITEM_WARPS * 32) k_fetch(UpdArgs a) {
  extern __shared__ __align__(16) uint8_t fetch_sm[];
  __shared__ uint32_t bits_sh[ITEM_WARPS][32], pre_sh[ITEM_WARPS][32];
  const uint32_t i = item_of_warp();
  if (i >= *a.nitems) return;  // warp-uniform
  const int lane = lane_id();
  uint32_t* bits = bits_sh[warp_id()];
  uint32_t* pre = pre_sh[warp_id()];
  int2* sk = reinterpret_cast<int2*>(fetch_sm) + (size_t)warp_id() * a.HN;
  uint32_t* sl = reinterpret_cast<uint32_t*>(reinterpret_cast<int2*>(fetch_sm) + (size_t)ITEM_WARPS * a.HN) +
                 (size_t)warp_id() * a.HN;
  for (int v = lane; v < a.HN; v += 32) {
    sk[v] = make_int2(0, sk_meta(SK_NONE, 0, 0));
    sl[v] = 0xFFFFFFFFu;
  }
  bits[lane] = 0;
  __syncwarp();
  if (lane == 0) {
    sl[1] = a.items[i].root;
    sk[1] = make_int2(0, sk_meta(SK_BUCKET, 0, 0));  // provisional: marks "defined"
  }
  __syncwarp();
  for (int j = 0; j <= a.lam; ++j) {
    for (int v = (1 << j) + lane; v < (2 << j); v += 32) {
      if (sk_state(sk[v].y) == SK_NONE) continue;
      const uint32_t slot = sl[v];
      uint8_t dm = (uint8_t)PKD_LEAF;
      Node nd{};
      if (j < a.lam) {  // both loads issued together
        dm = a.ndim[slot];
        nd = a.nodes[slot];
      }
      if (dm == PKD_LEAF) {
        // external: bit (its first position on level lambda) in the bitmap
        const uint32_t lo = (uint32_t)(v - (1 << j)) << (a.lam - j);
        atomicOr(&bits[lo >> 5], 1u << (lo & 31));
        continue;
      }
      sk[v] = make_int2(nd.split, sk_meta(SK_INTERNAL, dm, 0));
      sl[2 * v] = nd.a;
      sl[2 * v + 1] = nd.b;
      sk[2 * v] = make_int2(0, sk_meta(SK_BUCKET, 0, 0));
      sk[2 * v + 1] = make_int2(0, sk_meta(SK_BUCKET, 0, 0));
    }
    __syncwarp();
  }
  // left-to-right number of an external node = set bits before its position
  const uint32_t wc = (uint32_t)__popc(bits[lane]);
  const uint32_t incl = (uint32_t)warp_incl_scan((int)wc);
  pre[lane] = incl - wc;
  __syncwarp();
  for (int j = 0; j <= a.lam; ++j) {
    for (int v = (1 << j) + lane; v < (2 << j); v += 32) {
      if (sk_state(sk[v].y) != SK_BUCKET) continue;
      const uint32_t lo = (uint32_t)(v - (1 << j)) << (a.lam - j);
      const uint32_t nbk = pre[lo >> 5] + (uint32_t)__popc(bits[lo >> 5] & ((1u << (lo & 31)) - 1u));
      sk[v].y = sk_meta(SK_BUCKET, 0, (int)nbk);
    }
  }
  __syncwarp();
  int2* gsk = a.skel + (uint64_t)i * a.HN;
  uint32_t* gsl = a.slots + (uint64_t)i * a.HN;
  for (int v = lane; v < a.HN; v += 32) {
    gsk[v] = sk[v];
    gsl[v] = sl[v];
  }
  if (lane == 31) a.nbk[i] = incl;
}

constexpr uint32_t SMALL_ITEM = 256;  // items up to this many points: one warp routes them

// Bucket ranges of the big items from the bucket-major scan of the tile
// histograms: one warp per item, its lanes over the buckets.
__global__ void k_bucket_ranges(RoundArgs r, uint64_t* bstart, uint32_t* blen, const uint32_t* nbk) {
  if (pkd_failed_block(r.st)) return;
  const uint32_t s = (uint32_t)(((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (s >= *r.nbig) return;  // warp-uniform
  const Seg it = r.big[s];
  const uint32_t k = r.skel_map[s];
  const uint32_t nb = nbk[k];
  const uint32_t nt = (it.len + r.TILE - 1) / r.TILE;
  const uint64_t hb = (uint64_t)r.tile0[s] * r.NB;
  const uint32_t base = r.hscan[hb];
  for (uint32_t b = lane_id(); b < (uint32_t)r.NB; b += 32) {
    uint32_t b0 = it.len, b1 = it.len;
    if (b < nb) {
      b0 = r.hscan[hb + (uint64_t)b * nt] - base;
      b1 = (b + 1 < nb) ? r.hscan[hb + (uint64_t)(b + 1) * nt] - base : it.len;
    }
    bstart[(uint64_t)k * r.NB + b] = it.start + b0;
    blen[(uint64_t)k * r.NB + b] = b1 - b0;
  }
}

// Small items: one warp walks every point through the item's skeleton,
// counts and ranks the buckets in shared memory, and scatters the item in
// one pass (no global histogram: the warp owns the whole item).  Points
// also go to the final batch buffer F (see k_copy_round).
template <int D>
__global__ void __launch_bounds__(256, (D <= 3 ? 6 : 1)) k_route_small(RoundArgs r, const uint32_t* small, const uint32_t* nsmall,
                                                     const Seg* items, const uint32_t* nbk, uint64_t* bstart,
                                                     uint32_t* blen, Pts F) {
  if (pkd_failed_block(r.st)) return;
  extern __shared__ unsigned cnt_sm[];
  const uint32_t gw = blockIdx.x * (blockDim.x / 32) + warp_id();
  if (gw >= *nsmall) return;  // warp-uniform
  unsigned* cnt = cnt_sm + (size_t)warp_id() * r.NB;
  const uint32_t k = small[gw];
  const Seg it = items[k];
  const int2* sk = r.skel + (uint64_t)k * r.HN;
  const uint32_t nb = nbk[k];
  for (int b = lane_id(); b < r.NB; b += 32) cnt[b] = 0;
  __syncwarp();
  constexpr int PER = SMALL_ITEM / 32;
  int32_t x[PER][D];
  uint32_t id[PER];
  int bk[PER], rk[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const uint32_t i = q * 32 + lane_id();
    bk[q] = -1;
    rk[q] = 0;
    if (i < it.len) {
      const uint64_t g = it.start + i;
#pragma unroll
      for (int j = 0; j < D; ++j) x[q][j] = r.src.x(D, j, g);
      id[q] = r.src.id(g);
      int h = 1;
      for (int l = 0; l < r.lam; ++l) {
        const int2 e = sk[h];
        if (sk_state(e.y) != SK_INTERNAL) break;
        h = 2 * h + (x[q][sk_dim(e.y)] >= e.x);
      }
      bk[q] = sk_bucket(sk[h].y);
    }
    const unsigned m = peer_mask(bk[q], r.lam);
    const int leader = __ffs(m) - 1;
    unsigned b0 = 0;
    if (bk[q] >= 0 && lane_id() == leader) b0 = atomicAdd(&cnt[bk[q]], (unsigned)__popc(m));
    rk[q] = (int)__shfl_sync(FULL_MASK, b0, leader) + __popc(m & lanemask_lt());
  }
  __syncwarp();
  // bucket starts: exclusive scan of the counts, 32 buckets at a time
  unsigned carry = 0;
  for (int b0 = 0; b0 < r.NB; b0 += 32) {
    const int b = b0 + lane_id();
    const unsigned c = b < r.NB ? cnt[b] : 0;
    const unsigned incl = (unsigned)warp_incl_scan((int)c);
    if (b < r.NB) {
      const uint64_t o = (uint64_t)k * r.NB + b;
      bstart[o] = it.start + carry + incl - c;
      blen[o] = (uint32_t)b < nb ? c : 0;
    }
    __syncwarp();
    if (b < r.NB) cnt[b] = carry + incl - c;
    carry += __shfl_sync(FULL_MASK, incl, 31);
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    if (bk[q] < 0) continue;
    const uint64_t g = it.start + cnt[bk[q]] + (uint32_t)rk[q];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      r.dst.c[(uint64_t)j * r.dst.stride + g] = x[q][j];
      F.c[(uint64_t)j * F.stride + g] = x[q][j];
    }
    r.dst.id[g] = id[q];
    F.id[g] = id[q];
  }
}

template <int D>
static void launch_route_small(const RoundArgs& ra, const uint32_t* small, const uint32_t* nsmall, const Seg* items,
                               const uint32_t* nbk, uint64_t* bstart, uint32_t* blen, Pts F, uint32_t n,
                               cudaStream_t s) {
  const size_t smb = (size_t)8 * ra.NB * 4;
  PKD_LAUNCH(k_route_small<D><<<(n + 7) / 8, 256, smb, s>>>(ra, small, nsmall, items, nbk, bstart, blen, F));
}

// Next-round items and leaf groups from the bucket ranges.  Each lane takes
// EMIT_PER heap positions at a time (v = v0 + 32u + lane): the loads of all
// of them are issued before the first counter update, and the warp reserves
// its outputs with one atomic per counter for all of them (warp scans give
// each lane its offsets).
constexpr int EMIT_PER = 4;
__global__ void __launch_bounds__(ITEM_WARPS * 32) k_route_emit(UpdArgs a) {
  if (pkd_failed_block(a.st)) return;
  const uint32_t i = item_of_warp();
  if (i >= *a.nitems) return;  // warp-uniform
  const int lane = lane_id();
  const Seg it = a.items[i];
  const int2* sk = a.skel + (uint64_t)i * a.HN;
  const uint32_t* sl = a.slots + (uint64_t)i * a.HN;
  const uint64_t kb0 = (uint64_t)i * a.NB;
  for (int b = lane; b < a.NB; b += 32) a.link[kb0 + b] = LINK_NONE;
  __syncwarp();
  for (int v0 = 1; v0 < a.HN; v0 += 32 * EMIT_PER) {
    int bkt[EMIT_PER];
#pragma unroll
    for (int u = 0; u < EMIT_PER; ++u) {
      const int v = v0 + 32 * u + lane;
      bkt[u] = -1;
      if (v < a.HN) {
        const int m = sk[v].y;
        if (sk_state(m) == SK_BUCKET) bkt[u] = sk_bucket(m);
      }
    }
    uint32_t cnt[EMIT_PER], slot[EMIT_PER];
    uint64_t b0[EMIT_PER];
#pragma unroll
    for (int u = 0; u < EMIT_PER; ++u) {
      cnt[u] = 0;
      slot[u] = 0;
      b0[u] = 0;
      if (bkt[u] >= 0) {
        cnt[u] = a.blen[kb0 + bkt[u]];
        b0[u] = a.bstart[kb0 + bkt[u]];
        slot[u] = sl[v0 + 32 * u + lane];
      }
    }
    bool leaf[EMIT_PER], big[EMIT_PER];
    uint32_t nL = 0, nN = 0, nB = 0, tiles = 0, bigpts = 0;
#pragma unroll
    for (int u = 0; u < EMIT_PER; ++u) {
      const bool reached = cnt[u] != 0;
      leaf[u] = reached && a.ndim[slot[u]] == PKD_LEAF;
      const bool inner = reached && !leaf[u];
      big[u] = inner && cnt[u] > SMALL_ITEM;
      nL += leaf[u];
      nN += inner;
      nB += big[u];
      if (big[u]) {
        tiles += (cnt[u] + a.TILE - 1) / a.TILE;
        bigpts += cnt[u];
      }
    }
    // one update of each counter per warp and batch
    const uint32_t iL = (uint32_t)warp_incl_scan((int)nL);
    const uint32_t iN = (uint32_t)warp_incl_scan((int)nN);
    const uint32_t iB = (uint32_t)warp_incl_scan((int)nB);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      tiles += __shfl_xor_sync(FULL_MASK, tiles, o);
      bigpts += __shfl_xor_sync(FULL_MASK, bigpts, o);
    }
    const uint32_t tL = __shfl_sync(FULL_MASK, iL, 31), tN = __shfl_sync(FULL_MASK, iN, 31);
    const uint32_t tB = __shfl_sync(FULL_MASK, iB, 31);
    uint32_t gB = 0, qB = 0, kB = 0, sB = 0;
    if (lane == 0) {
      if (tL) gB = atomicAdd(a.ngroups, tL);
      if (tN) qB = atomicAdd(&a.next_ctr[0], tN);
      if (tB) {
        kB = atomicAdd(&a.next_ctr[2], tB);
        atomicAdd(&a.next_ctr[1], tiles);
        atomicAdd(&a.next_ctr[16], bigpts);
      }
      if (tN > tB) sB = atomicAdd(&a.next_ctr[3], tN - tB);
    }
    uint32_t g = __shfl_sync(FULL_MASK, gB, 0) + iL - nL;
    uint32_t q = __shfl_sync(FULL_MASK, qB, 0) + iN - nN;
    uint32_t kb = __shfl_sync(FULL_MASK, kB, 0) + iB - nB;
    uint32_t sb = __shfl_sync(FULL_MASK, sB, 0) + (iN - iB) - (nN - nB);
#pragma unroll
    for (int u = 0; u < EMIT_PER; ++u) {
      if (!cnt[u]) continue;
      const int v = v0 + 32 * u + lane;
      const uint64_t k = kb0 + bkt[u];
      const uint32_t depth = it.depth + (31 - __clz(v));
      if (leaf[u]) {
        if (g >= a.group_cap) {
          set_error(a.st, DERR_CAPACITY, 800);
        } else {
          a.groups[g] = LeafGroup{slot[u], depth, b0[u], cnt[u], a.insert ? cnt[u] : 0u, 0u, 0u};
          a.link[k] = LINK_LEAF | g;
        }
        ++g;
        continue;
      }
      const Seg c{b0[u], cnt[u], depth, slot[u], IN_B};
      a.next[q] = c;
      if (big[u]) {
        a.next_big[kb] = c;
        a.next_bigmap[kb] = q;
        ++kb;
      } else {
        a.next_small[sb] = q;
        ++sb;
      }
      a.link[k] = q;
      ++q;
    }
  }
}

// Copy every point this round moved into the final batch buffer F.  Points
// that go on to a deeper round are overwritten there later, so F ends with
// every point at its final position (the points of a leaf group are never
// moved again).  Same tiling as the sieve kernels: one block per tile.
__global__ void k_copy_round(RoundArgs r, Pts F) {
  if (pkd_failed_block(r.st)) return;
  SieveTile t;
  if (!sieve_tile(r, t, blockIdx.x)) return;
  const int d = r.p.d;
  for (int i = threadIdx.x; i < t.cnt; i += blockDim.x) {
    const uint64_t p = t.seg.start + t.first + (uint64_t)i;
    for (int j = 0; j < d; ++j) F.c[(uint64_t)j * F.stride + p] = r.dst.c[(uint64_t)j * r.dst.stride + p];
    F.id[p] = r.dst.id[p];
  }
}

// The per-leaf kernels below give each warp UPW leaves (or rebuild items):
// lanes 0..UPW-1 fetch the descriptors together, and for leaves of at most
// 32 points every load of the UPW leaves is issued before the first store,
// so a warp keeps UPW dependent chains in flight instead of one.
constexpr int UPW = 4;
constexpr int UPW_WARPS = 8;  // warps per CTA
static_assert(32 % UPW == 0, "lanes split evenly between a warp's leaves");
__host__ __device__ inline unsigned upw_blocks(uint32_t n) {
  return (unsigned)(((uint64_t)n + UPW * UPW_WARPS - 1) / (UPW * UPW_WARPS));
}

// Deletion round 1 at the leaves: mark stored points equal to a routed batch
// point (coordinates and id); count them.
template <int D>
__global__ void __launch_bounds__(UPW_WARPS * 32, (D <= 3 ? 8 : 1)) k_match(LeafGroup* groups, const uint32_t* ngroups,
                                                          const Node* nodes, Pts A, Pts F, uint8_t* dead,
                                                          uint32_t* aux) {
  const uint32_t n = *ngroups;
  const uint32_t k0 = (blockIdx.x * UPW_WARPS + warp_id()) * UPW;
  if (k0 >= n) return;
  const int lane = lane_id();
  uint32_t slot = 0, a = 0, sz = 0, glen = 0;
  unsigned long long gst = 0;
  if (lane < UPW && k0 + lane < n) {
    const LeafGroup G = groups[k0 + lane];
    const Node leaf = nodes[G.slot];
    slot = G.slot;
    gst = G.start;
    glen = G.len;
    a = leaf.a;
    sz = leaf.size;
  }
  {
    // common case: every leaf of the warp holds at most 32 points and
    // receives at most 32 / UPW batch points; all loads are issued at once
    constexpr int PER = 32 / UPW;
    uint32_t qa[UPW], qsz[UPW], qlen[UPW];
    bool small = true;
#pragma unroll
    for (int q = 0; q < UPW; ++q) {
      qa[q] = __shfl_sync(FULL_MASK, a, q);
      qsz[q] = __shfl_sync(FULL_MASK, sz, q);
      qlen[q] = __shfl_sync(FULL_MASK, glen, q);
      small &= qsz[q] <= 32 && qlen[q] <= (uint32_t)PER;
    }
    if (small) {
      int32_t x[UPW][D];
      uint32_t id[UPW];
#pragma unroll
      for (int q = 0; q < UPW; ++q) {
        id[q] = 0;
        if ((uint32_t)lane < qsz[q]) {
#pragma unroll
          for (int j = 0; j < D; ++j) x[q][j] = A.c[(uint64_t)j * A.stride + qa[q] + lane];
          id[q] = A.id[(uint64_t)qa[q] + lane];
        }
      }
      // lane q * PER + e holds batch point e of leaf q
      const int mq = lane / PER, me = lane % PER;
      const unsigned long long myst = __shfl_sync(FULL_MASK, gst, mq);
      const uint32_t mylen = __shfl_sync(FULL_MASK, glen, mq);
      int32_t fx[D];
      uint32_t fid = 0xFFFFFFFFu;
      if ((uint32_t)me < mylen) {
        const uint64_t r = myst + (uint64_t)me;
#pragma unroll
        for (int j = 0; j < D; ++j) fx[j] = F.c[(uint64_t)j * F.stride + r];
        fid = F.id[r];
      }
#pragma unroll
      for (int q = 0; q < UPW; ++q) {
        bool hit = false;
        for (int t = 0; t < (int)qlen[q]; ++t) {
          const int src = q * PER + t;
          bool same = __shfl_sync(FULL_MASK, fid, src) == id[q];
#pragma unroll
          for (int j = 0; j < D; ++j) same &= __shfl_sync(FULL_MASK, fx[j], src) == x[q][j];
          hit |= same;
        }
        hit &= (uint32_t)lane < qsz[q];
        if (hit) dead[(uint64_t)qa[q] + lane] = 1;
        const int found = __popc(__ballot_sync(FULL_MASK, hit));
        const uint32_t qslot = __shfl_sync(FULL_MASK, slot, q);
        if (lane == 0 && k0 + q < n) {
          groups[k0 + q].found = (uint32_t)found;
          aux[qslot] = (uint32_t)found;
        }
      }
      return;
    }
  }
#pragma unroll
  for (int q = 0; q < UPW; ++q) {
    if (k0 + q >= n) break;
    const uint32_t qa = __shfl_sync(FULL_MASK, a, q), qsz = __shfl_sync(FULL_MASK, sz, q);
    const uint32_t qlen = __shfl_sync(FULL_MASK, glen, q), qslot = __shfl_sync(FULL_MASK, slot, q);
    const unsigned long long qst = __shfl_sync(FULL_MASK, gst, q);
    int found = 0;
    for (uint32_t base = 0; base < qsz; base += 32) {
      const uint32_t i = base + lane;
      bool hit = false;
      int32_t x[D];
      uint32_t id = 0;
      if (i < qsz) {
        const uint64_t p = (uint64_t)qa + i;
#pragma unroll
        for (int j = 0; j < D; ++j) x[j] = A.c[(uint64_t)j * A.stride + p];
        id = A.id[p];
      }
      // the routed batch points, 32 at a time, broadcast lane by lane
      for (uint32_t b0 = 0; b0 < qlen; b0 += 32) {
        const uint32_t rb = b0 + lane;
        int32_t fx[D];
        uint32_t fid = 0xFFFFFFFFu;
        if (rb < qlen) {
          const uint64_t r = qst + rb;
#pragma unroll
          for (int j = 0; j < D; ++j) fx[j] = F.c[(uint64_t)j * F.stride + r];
          fid = F.id[r];
        }
        const int cnt = (int)min(32u, qlen - b0);
        for (int t = 0; t < cnt; ++t) {
          bool same = __shfl_sync(FULL_MASK, fid, t) == id;
#pragma unroll
          for (int j = 0; j < D; ++j) same &= __shfl_sync(FULL_MASK, fx[j], t) == x[j];
          hit |= same;
        }
      }
      hit &= i < qsz;
      if (hit) dead[(uint64_t)qa + i] = 1;
      found += __popc(__ballot_sync(FULL_MASK, hit));
    }
    if (lane == 0) {
      groups[k0 + q].found = (uint32_t)found;
      aux[qslot] = (uint32_t)found;
    }
  }
}

// Exact counts per skeleton node, bottom-up (rounds in reverse order).  The
// item's states and bucket counts are loaded first, AGG_PER heap positions
// per lane at a time with all their loads in flight together; the interior
// sums are then formed level by level in shared memory, from the deepest,
// and the counts are written out at the end.
constexpr int AGG_PER = 4;
__global__ void __launch_bounds__(ITEM_WARPS * 32) k_aggregate(UpdArgs a) {
  if (pkd_failed_block(a.st)) return;
  extern __shared__ __align__(16) int agg_sm[];
  const uint32_t i = item_of_warp();
  if (i >= *a.nitems) return;  // warp-uniform
  const int lane = lane_id();
  int* ms = agg_sm + (size_t)warp_id() * 2 * a.HN;
  uint32_t* fs = reinterpret_cast<uint32_t*>(ms + a.HN);
  const int2* sk = a.skel + (uint64_t)i * a.HN;
  const uint32_t* sl = a.slots + (uint64_t)i * a.HN;
  uint32_t* f = a.fnd + (uint64_t)i * a.HN;
  const uint64_t kb0 = (uint64_t)i * a.NB;
  for (int v0 = 1; v0 < a.HN; v0 += 32 * AGG_PER) {
    int m[AGG_PER];
#pragma unroll
    for (int u = 0; u < AGG_PER; ++u) {
      const int v = v0 + 32 * u + lane;
      m[u] = v < a.HN ? sk[v].y : sk_meta(SK_NONE, 0, 0);
    }
    uint32_t L[AGG_PER];
#pragma unroll
    for (int u = 0; u < AGG_PER; ++u)
      L[u] = sk_state(m[u]) == SK_BUCKET ? a.link[kb0 + sk_bucket(m[u])] : LINK_NONE;
#pragma unroll
    for (int u = 0; u < AGG_PER; ++u) {
      uint32_t c = 0;
      if (L[u] != LINK_NONE)
        c = (L[u] & LINK_LEAF) ? a.groups[L[u] & ~LINK_LEAF].found : a.next_fnd[(uint64_t)L[u] * a.next_HN + 1];
      const int v = v0 + 32 * u + lane;
      if (v < a.HN) {
        ms[v] = m[u];
        fs[v] = c;
      }
    }
  }
  __syncwarp();
  for (int j = a.lam - 1; j >= 0; --j) {  // interior nodes sit above level lambda
    for (int v = (1 << j) + lane; v < (2 << j); v += 32)
      if (sk_state(ms[v]) == SK_INTERNAL) fs[v] = fs[2 * v] + fs[2 * v + 1];
    __syncwarp();
  }
  for (int v = 1 + lane; v < a.HN; v += 32) {
    if (sk_state(ms[v]) == SK_NONE) continue;
    const uint32_t c = fs[v];
    f[v] = c;
    if (!a.insert && c) a.aux[sl[v]] = c;
  }
}

__device__ void push_rebuild(const UpdArgs& a, uint32_t slot, uint32_t depth, uint32_t size,
                             uint32_t old_live, uint64_t ws, uint64_t we) {
  const uint32_t k = atomicAdd(a.nitems_out, 1u);
  if (k >= a.items_cap) {
    set_error(a.st, DERR_CAPACITY, 810);
    return;
  }
  a.items_out[k] = RebuildItem{slot, depth, size, old_live, ws, we, 0};
  atomicAdd(a.items_total, (unsigned long long)size);
}

// Top-down alpha test over every skeleton (rounds in forward order; within a
// skeleton, level by level from the root).  under: one bit per heap node
// inside a subtree that is rebuilt.
// The item's skeleton, slots, counts and the nodes' current sizes are staged
// in shared memory first (DEC_PER heap positions per lane at a time, their
// loads in flight together); the levels then read shared memory only.
constexpr int DEC_PER = 4;
__global__ void __launch_bounds__(ITEM_WARPS * 32) k_decide(UpdArgs a) {
  if (pkd_failed_block(a.st)) return;
  extern __shared__ __align__(16) uint8_t dec_sm[];
  __shared__ uint32_t under_sh[ITEM_WARPS][64];
  const uint32_t i = item_of_warp();
  if (i >= *a.nitems) return;  // warp-uniform
  const int lane = lane_id();
  uint32_t* under = under_sh[warp_id()];
  const Seg it = a.items[i];
  int2* sk = reinterpret_cast<int2*>(dec_sm) + (size_t)warp_id() * a.HN;
  uint32_t* sl = reinterpret_cast<uint32_t*>(reinterpret_cast<int2*>(dec_sm) + (size_t)ITEM_WARPS * a.HN) +
                 (size_t)warp_id() * a.HN;
  uint32_t* f = sl + (size_t)ITEM_WARPS * a.HN;
  uint32_t* osz = f + (size_t)ITEM_WARPS * a.HN;
  {
    const int2* gsk = a.skel + (uint64_t)i * a.HN;
    const uint32_t* gsl = a.slots + (uint64_t)i * a.HN;
    const uint32_t* gf = a.fnd + (uint64_t)i * a.HN;
    for (int v0 = 1; v0 < a.HN; v0 += 32 * DEC_PER) {
      int2 e[DEC_PER];
      uint32_t slv[DEC_PER], fv[DEC_PER], szv[DEC_PER];
#pragma unroll
      for (int u = 0; u < DEC_PER; ++u) {
        const int v = v0 + 32 * u + lane;
        e[u] = v < a.HN ? gsk[v] : make_int2(0, sk_meta(SK_NONE, 0, 0));
      }
#pragma unroll
      for (int u = 0; u < DEC_PER; ++u) {
        const int v = v0 + 32 * u + lane;
        slv[u] = 0;
        fv[u] = 0;
        if (sk_state(e[u].y) != SK_NONE) {
          slv[u] = gsl[v];
          fv[u] = gf[v];
        }
      }
#pragma unroll
      for (int u = 0; u < DEC_PER; ++u) szv[u] = sk_state(e[u].y) != SK_NONE ? a.nodes[slv[u]].size : 0u;
#pragma unroll
      for (int u = 0; u < DEC_PER; ++u) {
        const int v = v0 + 32 * u + lane;
        if (v >= a.HN) continue;
        sk[v] = e[u];
        sl[v] = slv[u];
        f[v] = fv[u];
        osz[v] = szv[u];
      }
    }
  }
  under[lane] = 0;
  under[lane + 32] = 0;
  __syncwarp();
  if (lane == 0 && a.iflag[i]) under[0] = 2u;
  __syncwarp();
  for (int j = 0; j <= a.lam; ++j) {
    for (int v = (1 << j) + lane; v < (2 << j); v += 32) {
      const int m = sk[v].y;
      const int st = sk_state(m);
      if (st == SK_NONE) continue;
      const bool u = (under[v >> 5] >> (v & 31)) & 1u;
      if (st == SK_BUCKET) {
        if (!u) continue;
        const uint32_t L = a.link[(uint64_t)i * a.NB + sk_bucket(m)];
        if (L == LINK_NONE) continue;
        if (L & LINK_LEAF) a.groups[L & ~LINK_LEAF].flag = 1;
        else a.next_iflag[L] = 1;
        continue;
      }
      const int c0 = 2 * v;  // children c0 and c0 + 1 share a word of `under`
      if (u) {
        atomicOr(&under[c0 >> 5], 3u << (c0 & 31));
        continue;
      }
      const uint32_t c = f[v];
      if (c == 0) continue;  // nothing below changes
      const uint32_t slot = sl[v];
      const uint32_t old = osz[v], lold = osz[c0];
      const uint32_t N = a.insert ? old + c : old - c;
      const uint32_t L = a.insert ? lold + f[c0] : lold - f[c0];
      if (N > 0 && is_balanced(L, N, a.p.alpha_num, a.p.alpha_den)) {
        a.nsz[(uint64_t)i * a.HN + v] = N;  // written to the node once nothing can fail
        continue;
      }
      // rebuild this subtree; the batch points below it are contiguous
      int lv = v, rv = v;
      while (sk_state(sk[lv].y) == SK_INTERNAL) lv = 2 * lv;
      while (sk_state(sk[rv].y) == SK_INTERNAL) rv = 2 * rv + 1;
      const uint64_t kl = (uint64_t)i * a.NB + sk_bucket(sk[lv].y);
      const uint64_t kr = (uint64_t)i * a.NB + sk_bucket(sk[rv].y);
      const uint32_t depth = it.depth + (31 - __clz(v));
      push_rebuild(a, slot, depth, N, a.insert ? old : old - c, a.bstart[kl], a.bstart[kr] + a.blen[kr]);
      atomicOr(&under[c0 >> 5], 3u << (c0 & 31));
    }
    __syncwarp();
  }
}

// Reached leaves outside rebuilt subtrees: insert -> rebuild item
// Build(leaf + new); delete -> compacted in place (a leaf minus some of its
// points is a leaf again).
__global__ void k_leaf_items(UpdArgs a, LeafGroup* groups, const uint32_t* ngroups, uint32_t* compact,
                             uint32_t* ncompact) {
  if (pkd_failed_block(a.st)) return;  // uniform: before the block-wide reservation
  const uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t ng = *ngroups;
  bool push = false, comp = false;
  RebuildItem it{};
  if (gi < ng) {
    const LeafGroup G = groups[gi];
    if (!G.flag) {
      const uint32_t old = a.nodes[G.slot].size;
      if (a.insert) {
        push = true;
        it = RebuildItem{G.slot, G.depth, old + G.len, old, G.start, G.start + G.len, 0};
      } else if (G.found) {
        comp = true;
      }
    }
  }
  // one counter update per block
  const uint32_t c[2] = {push ? 1u : 0u, comp ? 1u : 0u};
  uint32_t* const ctrs[2] = {a.nitems_out, ncompact};
  uint32_t first[2];
  block_reserve<2>(c, ctrs, first);
  const unsigned long long tv[1] = {push ? (unsigned long long)it.size : 0ull};
  unsigned long long* const tc[1] = {a.items_total};
  block_add64<1>(tv, tc);
  const uint32_t bp = first[0], bc = first[1];
  if (push) {
    if (bp < a.items_cap) a.items_out[bp] = it;
    else set_error(a.st, DERR_CAPACITY, 811);
  }
  if (comp) compact[bc] = gi;
}

template <int D>
__global__ void __launch_bounds__(UPW_WARPS * 32) k_compact_leaves(const LeafGroup* groups, const uint32_t* list,
                                                                   const uint32_t* n, Node* nodes, Pts A,
                                                                   const uint8_t* dead) {
  const uint32_t nn = *n;
  const uint32_t k0 = (blockIdx.x * UPW_WARPS + warp_id()) * UPW;
  if (k0 >= nn) return;
  const int lane = lane_id();
  uint32_t slot = 0, a = 0, sz = 0;
  if (lane < UPW && k0 + lane < nn) {
    slot = groups[list[k0 + lane]].slot;
    const Node nd = nodes[slot];
    a = nd.a;
    sz = nd.size;
  }
  uint32_t qa[UPW], qsz[UPW], qslot[UPW];
  bool small = true;
#pragma unroll
  for (int q = 0; q < UPW; ++q) {
    qa[q] = __shfl_sync(FULL_MASK, a, q);
    qsz[q] = __shfl_sync(FULL_MASK, sz, q);
    qslot[q] = __shfl_sync(FULL_MASK, slot, q);
    small &= qsz[q] <= 32;
  }
  if (small) {
    // survivors move to the front, in order: all loads, then all stores
    int32_t x[UPW][D];
    uint32_t id[UPW];
    bool keep[UPW];
#pragma unroll
    for (int q = 0; q < UPW; ++q) {
      keep[q] = lane < qsz[q] && !dead[(uint64_t)qa[q] + lane];
      if (lane < qsz[q]) {
#pragma unroll
        for (int j = 0; j < D; ++j) x[q][j] = A.c[(uint64_t)j * A.stride + qa[q] + lane];
        id[q] = A.id[(uint64_t)qa[q] + lane];
      }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < UPW; ++q) {
      const unsigned m = __ballot_sync(FULL_MASK, keep[q]);
      if (keep[q]) {
        const uint64_t o = (uint64_t)qa[q] + __popc(m & lanemask_lt());
#pragma unroll
        for (int j = 0; j < D; ++j) A.c[(uint64_t)j * A.stride + o] = x[q][j];
        A.id[o] = id[q];
      }
      if (lane == 0 && k0 + q < nn) nodes[qslot[q]].size = (uint32_t)__popc(m);
    }
    return;
  }
#pragma unroll 1
  for (int q = 0; q < UPW; ++q) {
    if (k0 + q >= nn) break;
    uint32_t out = 0;
    for (uint32_t base = 0; base < qsz[q]; base += 32) {
      const uint32_t i = base + lane;
      const bool keep = i < qsz[q] && !dead[(uint64_t)qa[q] + i];
      int32_t x[D];
      uint32_t id = 0;
      if (keep) {
#pragma unroll
        for (int j = 0; j < D; ++j) x[j] = A.c[(uint64_t)j * A.stride + qa[q] + i];
        id = A.id[(uint64_t)qa[q] + i];
      }
      const unsigned m = __ballot_sync(FULL_MASK, keep);
      __syncwarp();
      if (keep) {
        const uint64_t o = (uint64_t)qa[q] + out + __popc(m & lanemask_lt());
#pragma unroll
        for (int j = 0; j < D; ++j) A.c[(uint64_t)j * A.stride + o] = x[j];
        A.id[o] = id;
      }
      out += __popc(m);
      __syncwarp();
    }
    if (lane == 0) nodes[qslot[q]].size = out;
  }
}

// Arena positions of the rebuild items (exclusive scan of their sizes).
__global__ void k_item_sizes(const RebuildItem* it, const uint32_t* n, uint32_t* sizes) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < *n) sizes[i] = it[i].size;
}

// An item of at most phi points is a leaf again (Build wraps it): its
// segment is skipped by the rebuild, which then only visits the items that
// split, and k_item_leaves writes its node once its points are in place.
__global__ void k_item_pos(RebuildItem* it, const uint32_t* n, const uint32_t* off, uint64_t top, Seg* segs,
                           uint32_t phi) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *n) return;
  const RebuildItem x = it[i];
  const uint64_t pos = top + off[i];
  it[i].pos = pos;
  segs[i] = Seg{pos, x.size <= phi ? SEG_SKIP : x.size, x.depth, x.slot, IN_A};
}

// The node of every item of at most phi points: a leaf over its new range.
// (Its depth is that of the old subtree's root, so the tree's depth bound
// needs no update.)
__global__ void k_item_leaves(const RebuildItem* it, const uint32_t* n, Node* nodes, uint8_t* ndim, uint32_t phi) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *n) return;
  const RebuildItem x = it[i];
  if (x.size > phi) return;
  nodes[x.slot] = Node{0, x.size, (uint32_t)x.pos, 0};
  ndim[x.slot] = PKD_LEAF;
}

// Breadth-first flatten of the old subtrees of the rebuild items: every
// frontier entry is (node, item, offset of its live points within the item).
struct Front {
  uint32_t slot;
  uint32_t item;
  uint64_t off;
};

// Leaves of more than BIG_LEAF points are copied one block each.
constexpr uint32_t BIG_LEAF = 1024;

constexpr int FRONT_BATCH = 8;  // frontier levels launched per host check

__global__ void k_front_init(const RebuildItem* it, const uint32_t* n, Front* f, uint32_t* nf) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool e = i < *n && it[i].old_live != 0;
  const uint32_t c[1] = {e ? 1u : 0u};
  uint32_t* const ctrs[1] = {nf};
  uint32_t first[1];
  block_reserve<1>(c, ctrs, first);
  if (e) f[first[0]] = Front{it[i].slot, i, 0};
}

// One level of the frontier: the grid strides over the device-side count
// *nf (block-uniform), so the host launches a batch of levels without
// reading any count in between; a level with an empty frontier does nothing.
// An entry past a list's capacity is not written: it sets *ovf, and the
// host redoes the flatten with larger lists.  The counts still include such
// entries, so a level reads at most `cap` entries of its frontier (the
// entries past it were never written; the attempt is redone anyway).
__global__ void k_front_expand(const Front* f, const uint32_t* nf, Front* g, uint32_t* ng, Front* leaves,
                               uint32_t* nleaves, Front* bigleaves, uint32_t* nbig, const Node* nodes,
                               const uint8_t* ndim, const uint32_t* aux, int use_aux, uint32_t cap, uint32_t bcap,
                               uint32_t* ovf) {
  const uint32_t n = min(*nf, cap);
  for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const bool have = i < n;
    Front e{};
    bool leaf = false, big = false;
    if (have) {
      e = f[i];
      leaf = ndim[e.slot] == PKD_LEAF;
      big = leaf && nodes[e.slot].size > BIG_LEAF;
    }
    const uint32_t c[3] = {have && leaf && !big ? 1u : 0u, have && !leaf ? 2u : 0u, big ? 1u : 0u};
    uint32_t* const ctrs[3] = {nleaves, ng, nbig};
    uint32_t first[3];
    block_reserve<3>(c, ctrs, first);
    if (!have) continue;
    if (leaf) {
      const uint32_t k = big ? first[2] : first[0];
      if (k < (big ? bcap : cap)) (big ? bigleaves : leaves)[k] = e;
      else atomicOr(ovf, 1u);
      continue;
    }
    const Node nd = nodes[e.slot];
    const uint32_t llive = nodes[nd.a].size - (use_aux ? aux[nd.a] : 0u);
    const uint32_t k = first[1];
    if (k + 2 > cap) {
      atomicOr(ovf, 1u);
      continue;
    }
    g[k] = Front{nd.a, e.item, e.off};
    g[k + 1] = Front{nd.b, e.item, e.off + llive};
  }
}

// Flattened leaves, UPW per warp: copy their live points to the item's range.
template <int D>
__global__ void __launch_bounds__(UPW_WARPS * 32) k_copy_leaves(const Front* lv, const uint32_t* n,
                                                                const RebuildItem* items, const Node* nodes, Pts A,
                                                                const uint8_t* dead, int use_dead) {
  const uint32_t nn = *n;
  const uint32_t k0 = (blockIdx.x * UPW_WARPS + warp_id()) * UPW;
  if (k0 >= nn) return;
  const int lane = lane_id();
  uint32_t a = 0, sz = 0;
  unsigned long long d0 = 0;
  if (lane < UPW && k0 + lane < nn) {
    const Front e = lv[k0 + lane];
    const Node nd = nodes[e.slot];
    a = nd.a;
    sz = nd.size;
    d0 = items[e.item].pos + e.off;
  }
  uint32_t qa[UPW], qsz[UPW];
  unsigned long long qd[UPW];
  bool small = true;
#pragma unroll
  for (int q = 0; q < UPW; ++q) {
    qa[q] = __shfl_sync(FULL_MASK, a, q);
    qsz[q] = __shfl_sync(FULL_MASK, sz, q);
    qd[q] = __shfl_sync(FULL_MASK, d0, q);
    small &= qsz[q] <= 32;
  }
  if (small) {
    int32_t x[UPW][D];
    uint32_t id[UPW];
    bool keep[UPW];
#pragma unroll
    for (int q = 0; q < UPW; ++q) {
      keep[q] = lane < qsz[q];
      if (keep[q]) {
        const uint64_t src = (uint64_t)qa[q] + lane;
        if (use_dead) keep[q] = !dead[src];
#pragma unroll
        for (int j = 0; j < D; ++j) x[q][j] = A.c[(uint64_t)j * A.stride + src];
        id[q] = A.id[src];
      }
    }
#pragma unroll
    for (int q = 0; q < UPW; ++q) {
      const unsigned m = __ballot_sync(FULL_MASK, keep[q]);
      if (keep[q]) {
        const uint64_t dst = qd[q] + __popc(m & lanemask_lt());
#pragma unroll
        for (int j = 0; j < D; ++j) A.c[(uint64_t)j * A.stride + dst] = x[q][j];
        A.id[dst] = id[q];
      }
    }
    return;
  }
#pragma unroll 1
  for (int q = 0; q < UPW; ++q) {
    uint32_t out = 0;
    for (uint32_t base = 0; base < qsz[q]; base += 32) {
      const uint32_t i = base + lane;
      const bool keep = i < qsz[q] && !(use_dead && dead[(uint64_t)qa[q] + i]);
      const unsigned m = __ballot_sync(FULL_MASK, keep);
      if (keep) {
        const uint64_t src = (uint64_t)qa[q] + i, dst = qd[q] + out + __popc(m & lanemask_lt());
#pragma unroll
        for (int j = 0; j < D; ++j) A.c[(uint64_t)j * A.stride + dst] = A.c[(uint64_t)j * A.stride + src];
        A.id[dst] = A.id[src];
      }
      out += __popc(m);
    }
  }
}

// Insert: append each item's new batch points after its old ones (UPW
// items per warp); items with more than NEW_BIG new points are left to
// k_copy_new_flat.
constexpr uint64_t NEW_BIG = 256;
template <int D>
__global__ void __launch_bounds__(UPW_WARPS * 32, (D <= 3 ? 8 : 1)) k_copy_new(const RebuildItem* items, const uint32_t* n, Pts F,
                                                             Pts A) {
  const uint32_t nn = *n;
  const uint32_t k0 = (blockIdx.x * UPW_WARPS + warp_id()) * UPW;
  if (k0 >= nn) return;
  const int lane = lane_id();
  unsigned long long ws = 0, cnt = 0, dst0 = 0;
  if (lane < UPW && k0 + lane < nn) {
    const RebuildItem it = items[k0 + lane];
    ws = it.ws;
    cnt = it.we - it.ws;
    dst0 = it.pos + it.old_live;
  }
  {
    // common case: at most 32 / UPW new points per item, one per lane
    constexpr int PER = 32 / UPW;
    const int mq = lane / PER, me = lane % PER;
    const unsigned long long mws = __shfl_sync(FULL_MASK, ws, mq), mcnt = __shfl_sync(FULL_MASK, cnt, mq);
    const unsigned long long md = __shfl_sync(FULL_MASK, dst0, mq);
    if (__all_sync(FULL_MASK, mcnt <= (unsigned long long)PER)) {
      if ((unsigned long long)me < mcnt) {
        const uint64_t src = mws + me, dst = md + me;
        int32_t x[D];
#pragma unroll
        for (int j = 0; j < D; ++j) x[j] = F.c[(uint64_t)j * F.stride + src];
        const uint32_t id = F.id[src];
#pragma unroll
        for (int j = 0; j < D; ++j) A.c[(uint64_t)j * A.stride + dst] = x[j];
        A.id[dst] = id;
      }
      return;
    }
  }
#pragma unroll 1
  for (int q = 0; q < UPW; ++q) {
    const unsigned long long qws = __shfl_sync(FULL_MASK, ws, q), qcnt = __shfl_sync(FULL_MASK, cnt, q);
    const unsigned long long qd = __shfl_sync(FULL_MASK, dst0, q);
    if (qcnt > NEW_BIG) continue;  // k_copy_new_flat copies these
    for (uint64_t i = lane; i < qcnt; i += 32) {
      const uint64_t src = qws + i, dst = qd + i;
#pragma unroll
      for (int j = 0; j < D; ++j) A.c[(uint64_t)j * A.stride + dst] = F.c[(uint64_t)j * F.stride + src];
      A.id[dst] = F.id[src];
    }
  }
}

// Insert: every new batch point of the rebuild items with more than NEW_BIG
// of them, one thread each: cnt[i] = those points of item i (0 for the
// others), off = their exclusive scan, so point j of
// the flat order belongs to the item whose range [off[i], off[i] + cnt[i])
// holds it (binary search).  A clustered batch can put millions of points
// into one item; this keeps all of them in flight instead of one warp's.
__global__ void k_item_newcounts(const RebuildItem* it, const uint32_t* n, uint32_t* cnt) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < *n) {
    const uint64_t c = it[i].we - it[i].ws;
    cnt[i] = c > NEW_BIG ? (uint32_t)c : 0u;  // the items k_copy_new leaves out
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_copy_new_flat(const RebuildItem* items, const uint32_t* n,
                                                       const uint32_t* off, const uint32_t* cnt, uint64_t m, Pts F,
                                                       Pts A) {
  const uint32_t ni = *n;
  if (ni == 0) return;
  const uint64_t total = (uint64_t)off[ni - 1] + cnt[ni - 1];
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < total && j < m;
       j += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = ni;  // the last item whose offset is <= j
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (off[mid] <= j) lo = mid;
      else hi = mid;
    }
    const RebuildItem it = items[lo];
    const uint64_t k = j - off[lo];
    const uint64_t src = it.ws + k, dst = it.pos + it.old_live + k;
#pragma unroll
    for (int q = 0; q < D; ++q) A.c[(uint64_t)q * A.stride + dst] = F.c[(uint64_t)q * F.stride + src];
    A.id[dst] = F.id[src];
  }
}

// Flattened leaves of more than BIG_LEAF points (heavy leaves, or leaves
// after skewed updates), one block each: live points keep their leaf's
// relative order, compacted by a block-wide ballot scan per 256 points.

template <int D>
__global__ void __launch_bounds__(256) k_copy_big_leaves(const Front* lv, const uint32_t* n,
                                                         const RebuildItem* items, const Node* nodes, Pts A,
                                                         const uint8_t* dead, int use_dead) {
  __shared__ int wsum[8];
  const uint32_t nn = *n;
  for (uint32_t k = blockIdx.x; k < nn; k += gridDim.x) {
    const Front e = lv[k];
    const Node nd = nodes[e.slot];
    const uint64_t d0 = items[e.item].pos + e.off;
    uint64_t out = 0;
    for (uint32_t base = 0; base < nd.size; base += 256) {
      const uint32_t i = base + threadIdx.x;
      const uint64_t src = (uint64_t)nd.a + i;
      const bool keep = i < nd.size && !(use_dead && dead[src]);
      int32_t x[D];
      uint32_t id = 0;
      if (keep) {
#pragma unroll
        for (int q = 0; q < D; ++q) x[q] = A.c[(uint64_t)q * A.stride + src];
        id = A.id[src];
      }
      const unsigned m = __ballot_sync(FULL_MASK, keep);
      if (lane_id() == 0) wsum[warp_id()] = __popc(m);
      __syncthreads();
      int before = 0, tot = 0;
      for (int w = 0; w < 8; ++w) {
        if (w < warp_id()) before += wsum[w];
        tot += wsum[w];
      }
      if (keep) {
        const uint64_t dst = d0 + out + before + __popc(m & lanemask_lt());
#pragma unroll
        for (int q = 0; q < D; ++q) A.c[(uint64_t)q * A.stride + dst] = x[q];
        A.id[dst] = id;
      }
      out += tot;
      __syncthreads();
    }
  }
}

template <int D>
static void launch_copy_new_flat(const RebuildItem* items, const uint32_t* n, const uint32_t* off,
                                 const uint32_t* cnt, uint64_t m, Pts F, Pts A, cudaStream_t s) {
  const unsigned g = (unsigned)std::min<uint64_t>((m + 255) / 256, 152ull * 32);
  PKD_LAUNCH(k_copy_new_flat<D><<<std::max(g, 1u), 256, 0, s>>>(items, n, off, cnt, m, F, A));
}
template <int D>
static void launch_copy_big_leaves(const Front* lv, const uint32_t* n, uint32_t nh, const RebuildItem* items,
                                   const Node* nodes, Pts A, const uint8_t* dead, int use_dead, cudaStream_t s) {
  const unsigned g = std::min<uint32_t>(nh, 152u * 8);
  PKD_LAUNCH(k_copy_big_leaves<D><<<std::max(g, 1u), 256, 0, s>>>(lv, n, items, nodes, A, dead, use_dead));
}

template <int D>
static void launch_match(LeafGroup* g, const uint32_t* ng, uint32_t n, const Node* nodes, Pts A, Pts F,
                         uint8_t* dead, uint32_t* aux, cudaStream_t s) {
  PKD_LAUNCH(k_match<D><<<upw_blocks(n), UPW_WARPS * 32, 0, s>>>(g, ng, nodes, A, F, dead, aux));
}
template <int D>
static void launch_compact(const LeafGroup* g, const uint32_t* list, const uint32_t* n, uint32_t nh, Node* nodes,
                           Pts A, const uint8_t* dead, cudaStream_t s) {
  PKD_LAUNCH(k_compact_leaves<D><<<upw_blocks(nh), UPW_WARPS * 32, 0, s>>>(g, list, n, nodes, A, dead));
}
template <int D>
static void launch_copy_leaves(const Front* lv, const uint32_t* n, uint32_t nh, const RebuildItem* items,
                               const Node* nodes, Pts A, const uint8_t* dead, int use_dead, cudaStream_t s) {
  PKD_LAUNCH(k_copy_leaves<D><<<upw_blocks(nh), UPW_WARPS * 32, 0, s>>>(lv, n, items, nodes, A, dead, use_dead));
}
template <int D>
static void launch_copy_new(const RebuildItem* items, const uint32_t* n, uint32_t nh, Pts F, Pts A, cudaStream_t s) {
  PKD_LAUNCH(k_copy_new<D><<<upw_blocks(nh), UPW_WARPS * 32, 0, s>>>(items, n, F, A));
}

// The deferred size updates of the nodes that stay (k_decide), applied once
// the update can no longer fail for lack of memory.
__global__ void k_apply_sizes(const uint32_t* slots, const uint32_t* nsz, uint64_t n, Node* nodes) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && nsz[i] != 0xFFFFFFFFu) nodes[slots[i]].size = nsz[i];
}

// Node records of the rebuild items' root slots, saved before the rebuild
// writes them and put back when it fails.
__global__ void k_save_roots(const RebuildItem* it, const uint32_t* n, const Node* nodes, const uint8_t* ndim,
                             Node* bn, uint8_t* bd) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < *n) {
    bn[i] = nodes[it[i].slot];
    bd[i] = ndim[it[i].slot];
  }
}
__global__ void k_restore_roots(const RebuildItem* it, const uint32_t* n, Node* nodes, uint8_t* ndim, const Node* bn,
                                const uint8_t* bd) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < *n) {
    nodes[it[i].slot] = bn[i];
    ndim[it[i].slot] = bd[i];
  }
}

__global__ void k_clear_aux(const uint32_t* slots, uint64_t n, uint32_t* aux) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const uint32_t s = slots[i];
    if (s != 0xFFFFFFFFu) aux[s] = 0;
  }
}

__global__ void k_stage(const int32_t* coords, const uint32_t* ids, uint64_t m, int d, Pts W) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  for (int j = 0; j < d; ++j) W.c[(uint64_t)j * W.stride + i] = coords[i * d + j];
  W.id[i] = ids[i];
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------

// Grow the arena (and the per-position node region) to hold `need` more
// points; node slots do not move, so the tree stays valid.
static int ensure_capacity(TreeMem& t, uint64_t need, cudaStream_t s) {
  if (t.top + need <= t.cap) return PKD_OK;
  uint64_t ncap = std::max<uint64_t>(t.cap + t.cap / 2, t.top + need + 4096);
  const uint64_t nnode = t.shared_cap + 2 * ncap;
  if (nnode >= 0xFFFFFFF0ull) return PKD_ENOMEM;
  Pts A2{};
  Node* n2 = nullptr;
  uint8_t* d2 = nullptr;
  cudaError_t e = big_alloc((void**)&A2.c, (size_t)t.p.d * ncap * 4, s);
  if (e == cudaSuccess) e = big_alloc((void**)&A2.id, (size_t)ncap * 4, s);
  if (e == cudaSuccess) e = big_alloc((void**)&n2, (size_t)nnode * sizeof(Node), s);
  if (e == cudaSuccess) e = big_alloc((void**)&d2, (size_t)nnode, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    for (void* q : {(void*)A2.c, (void*)A2.id, (void*)n2, (void*)d2}) big_free(q, s);
    return PKD_ENOMEM;
  }
  A2.stride = ncap;
  for (int j = 0; j < t.p.d; ++j)
    PKD_CUDA(cudaMemcpyAsync(A2.c + (uint64_t)j * ncap, t.A.c + (uint64_t)j * t.cap, t.top * 4,
                             cudaMemcpyDeviceToDevice, s));
  PKD_CUDA(cudaMemcpyAsync(A2.id, t.A.id, t.top * 4, cudaMemcpyDeviceToDevice, s));
  const uint64_t used = t.shared_cap + 2 * t.top;
  PKD_CUDA(cudaMemcpyAsync(n2, t.nodes, used * sizeof(Node), cudaMemcpyDeviceToDevice, s));
  PKD_CUDA(cudaMemcpyAsync(d2, t.ndim, used, cudaMemcpyDeviceToDevice, s));
  // delete scratch grows with the arena and keeps its marks
  uint8_t* dead2 = nullptr;
  uint32_t* aux2 = nullptr;
  if (t.dead) e = big_alloc((void**)&dead2, ncap, s);
  if (e == cudaSuccess && t.aux) e = big_alloc((void**)&aux2, nnode * 4, s);
  if (e != cudaSuccess) {  // nothing of the tree has changed
    cudaGetLastError();
    for (void* q : {(void*)A2.c, (void*)A2.id, (void*)n2, (void*)d2, (void*)dead2, (void*)aux2}) big_free(q, s);
    return PKD_ENOMEM;
  }
  if (dead2) {
    PKD_TRY(dev_fill(dead2, 0, ncap, s));
    PKD_CUDA(cudaMemcpyAsync(dead2, t.dead, t.cap, cudaMemcpyDeviceToDevice, s));
  }
  if (aux2) {
    PKD_TRY(dev_fill(aux2, 0, nnode * 4, s));
    PKD_CUDA(cudaMemcpyAsync(aux2, t.aux, t.node_cap * 4, cudaMemcpyDeviceToDevice, s));
  }
  for (void* q : {(void*)t.A.c, (void*)t.A.id, (void*)t.nodes, (void*)t.ndim, (void*)t.dead, (void*)t.aux})
    big_free(q, s);
  t.dead = dead2;
  t.aux = aux2;
  t.A = A2;
  t.nodes = n2;
  t.ndim = d2;
  t.cap = ncap;
  t.node_cap = nnode;
  return PKD_OK;
}

static int ensure_delete_scratch(TreeMem& t, cudaStream_t s) {
  bool zero = false;
  if (!t.dead) {
    PKD_CUDA(big_alloc_zeroed((void**)&t.dead, t.cap, s, &zero));
    if (!zero) PKD_TRY(dev_fill(t.dead, 0, t.cap, s));
  }
  if (!t.aux) {
    PKD_CUDA(big_alloc_zeroed((void**)&t.aux, t.node_cap * 4, s, &zero));
    if (!zero) PKD_TRY(dev_fill(t.aux, 0, t.node_cap * 4, s));
    else stat_items("scratch_zeroed", t.node_cap * 4);
  }
  return PKD_OK;
}

struct RouteRound {
  Seg* items;
  uint32_t n;
  int2* skel;
  uint32_t* slots;
  uint32_t* fnd;
  uint32_t* nsz;
  uint32_t* link;
  uint64_t* bstart;
  uint32_t* blen;
  uint32_t* iflag;
  uint32_t* d_n;  // device copy of n
};

// The batch comes either point-major from the caller (coords, ids) or
// already staged in structure-of-arrays form (`staged`, a buffer of at least
// m positions that the route may overwrite).
static int run_update(TreeMem& t, const int32_t* coords, const uint32_t* ids, const Pts* staged, uint64_t m,
                      bool insert, uint64_t* n_changed, cudaStream_t s) {
  const Params& p = t.p;
  const int d = p.d, lam = p.lambda, NB = 1 << lam, HN = 2 << lam;
  const int TILE = std::min(std::max(knobs().tile, 256), 4096);
  Scratch sc{s, {}};
  trace_mark(s, insert ? "insert: enter" : "delete: enter");
  if (!insert) PKD_TRY(ensure_delete_scratch(t, s));
  trace_mark(s, "upd: delete scratch");

  // batch buffers: W0/W1 ping-pong for the sieve, F final positions
  int32_t *wc[3] = {nullptr, nullptr, nullptr};
  uint32_t* wid[3] = {nullptr, nullptr, nullptr};
  for (int k = staged ? 1 : 0; k < 3; ++k) {
    PKD_TRY(sc.get(&wc[k], (size_t)d * m));
    PKD_TRY(sc.get(&wid[k], m));
  }
  Pts W[2] = {staged ? *staged : Pts{wc[0], wid[0], m}, Pts{wc[1], wid[1], m}};
  Pts F{wc[2], wid[2], m};
  if (!staged) PKD_LAUNCH(k_stage<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(coords, ids, m, d, W[0]));

  uint32_t* dctr;
  PKD_TRY(sc.get(&dctr, 32));
  PKD_TRY(dev_fill(dctr, 0, 32 * 4, s));
  PinnedBlock hblk(s);  // 128 bytes of host counters
  uint32_t* hctr = (uint32_t*)hblk.p;
  if (!hctr) return PKD_ENOMEM;
  uint32_t* d_ngroups = dctr + 4;
  uint32_t* d_nitems = dctr + 5;
  unsigned long long* d_total = (unsigned long long*)(dctr + 6);
  uint32_t* d_ncompact = dctr + 8;

  // every routed point ends in exactly one leaf group: at most m groups
  const uint32_t group_cap = (uint32_t)std::min<uint64_t>(m + 16, 0xFFFFFFF0ull);
  LeafGroup* groups;
  PKD_TRY(sc.get(&groups, group_cap));
  RebuildItem* items_out;
  const uint32_t items_cap = group_cap;  // at most one rebuild per routed point
  PKD_TRY(sc.get(&items_out, items_cap));

  UpdArgs ua{};
  ua.p = p;
  ua.lam = lam;
  ua.NB = NB;
  ua.HN = HN;
  ua.TILE = TILE;
  ua.insert = insert ? 1 : 0;
  ua.nodes = t.nodes;
  ua.ndim = t.ndim;
  ua.groups = groups;
  ua.ngroups = d_ngroups;
  ua.group_cap = group_cap;
  ua.items_out = items_out;
  ua.nitems_out = d_nitems;
  ua.items_total = d_total;
  ua.items_cap = items_cap;
  ua.aux = t.aux;
  ua.st = t.st;

  // ---- route ----
  std::vector<RouteRound> rounds;
  Seg root{0, (uint32_t)m, 0, t.root, IN_B};
  Seg* cur;
  Seg* cur_big;
  uint32_t *cur_bigmap, *cur_small;
  PKD_TRY(sc.get(&cur, 1));
  PKD_TRY(sc.get(&cur_big, 1));
  PKD_TRY(sc.get(&cur_bigmap, 1));
  PKD_TRY(sc.get(&cur_small, 1));
  uint32_t zero = 0;
  PKD_TRY(dev_store(cur, &root, sizeof(Seg), s));
  const bool root_big = m > SMALL_ITEM;
  if (root_big) {
    PKD_TRY(dev_store(cur_big, &root, sizeof(Seg), s));
    PKD_TRY(dev_store(cur_bigmap, &zero, 4, s));
  } else {
    PKD_TRY(dev_store(cur_small, &zero, 4, s));
  }
  uint32_t ncur = 1, tiles = root_big ? (uint32_t)((m + TILE - 1) / TILE) : 0;
  uint64_t big_pts = root_big ? m : 0;  // points the round's sieve kernels move
  uint32_t nbig = root_big ? 1 : 0, nsmall = root_big ? 0 : 1;
  int w = 0;
  uint32_t groups_before = 0;
  for (int r = 0; ncur > 0; ++r) {
    if (r > 200) return PKD_EINTERNAL;
    RouteRound R{};
    R.items = cur;
    R.n = ncur;
    PKD_TRY(sc.get(&R.skel, (size_t)ncur * HN));
    PKD_TRY(sc.get(&R.slots, (size_t)ncur * HN));
    PKD_TRY(sc.get(&R.fnd, (size_t)ncur * HN));
    PKD_TRY(sc.get(&R.nsz, (size_t)ncur * HN));
    PKD_TRY(dev_fill(R.nsz, 0xFF, (size_t)ncur * HN * 4, s));
    PKD_TRY(sc.get(&R.link, (size_t)ncur * NB));
    PKD_TRY(sc.get(&R.bstart, (size_t)ncur * NB));
    PKD_TRY(sc.get(&R.blen, (size_t)ncur * NB));
    PKD_TRY(sc.get(&R.iflag, ncur));
    PKD_TRY(sc.get(&R.d_n, 4));
    uint32_t hn[4] = {ncur, nbig, nsmall, 0};
    PKD_TRY(dev_fill(R.iflag, 0, (size_t)ncur * 4, s));
    PKD_TRY(dev_store(R.d_n, hn, 16, s));
    uint32_t* nbk;
    PKD_TRY(sc.get(&nbk, ncur));
    Seg *next, *next_big;
    uint32_t *next_bigmap, *next_small;
    PKD_TRY(sc.get(&next, (size_t)ncur * NB));
    PKD_TRY(sc.get(&next_big, (size_t)ncur * NB));
    PKD_TRY(sc.get(&next_bigmap, (size_t)ncur * NB));
    PKD_TRY(sc.get(&next_small, (size_t)ncur * NB));
    PKD_TRY(dev_fill(dctr, 0, 16, s));
    PKD_TRY(dev_fill(dctr + 16, 0, 4, s));

    ua.items = cur;
    ua.nitems = R.d_n;
    ua.skel = R.skel;
    ua.slots = R.slots;
    ua.nbk = nbk;
    ua.bstart = R.bstart;
    ua.blen = R.blen;
    ua.link = R.link;
    ua.fnd = R.fnd;
    ua.iflag = R.iflag;
    ua.next = next;
    ua.next_ctr = dctr;
    ua.next_big = next_big;
    ua.next_bigmap = next_bigmap;
    ua.next_small = next_small;
    const unsigned g1 = item_blocks(ncur);
    {
      const size_t smb = (size_t)ITEM_WARPS * HN * (sizeof(int2) + sizeof(uint32_t));
      static size_t set = 0;
      if (smb > 48 * 1024 && set < smb) {
        cudaFuncSetAttribute(k_fetch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
        set = smb;
      }
      PKD_LAUNCH(k_fetch<<<g1, ITEM_WARPS * 32, smb, s>>>(ua));
    }

    RoundArgs ra{};
    ra.wait_cycles = knobs().wait_cycles;
    ra.p = p;
    ra.lam = lam;
    ra.NB = NB;
    ra.HN = HN;
    ra.TILE = TILE;
    ra.src.soa = W[w];
    ra.src.is_aos = 0;
    ra.dst = W[w ^ 1];
    ra.skel = R.skel;
    ra.st = t.st;
    if (nbig) {
      // big items: tile histograms, bucket-major scan, scatter
      uint32_t *tile0, *hist, *hscan, *partial;
      uint64_t* excl;
      PKD_TRY(sc.get(&tile0, nbig));
      PKD_TRY(sc.get(&excl, nbig));
      PKD_TRY(sc.get(&hist, (size_t)tiles * NB));
      PKD_TRY(sc.get(&hscan, (size_t)tiles * NB));
      const uint64_t nh = (uint64_t)tiles * NB;
      PKD_TRY(sc.get(&partial, (nh + SCAN_TILE - 1) / SCAN_TILE + 1));
      ra.big = cur_big;
      ra.nbig = R.d_n + 1;
      ra.skel_map = cur_bigmap;
      ra.tile0 = tile0;
      ra.excl = excl;
      ra.hist = hist;
      ra.hscan = hscan;
      if (record_buckets(NB)) PKD_TRY(sc.get(&ra.bkt, (size_t)tiles * TILE));
      PKD_LAUNCH(k_big_prefix<<<1, 1024, 0, s>>>(cur_big, R.d_n + 1, (uint32_t)TILE, tile0, excl));
      PKD_DISPATCH_D(d, launch_count, ra, tiles, big_pts, "count_route", s);
      device_excl_scan(hist, hscan, nh, partial, s);
      PKD_LAUNCH(k_bucket_ranges<<<(unsigned)(((uint64_t)nbig * 32 + 127) / 128), 128, 0, s>>>(ra, R.bstart, R.blen,
                                                                                               nbk));
      PKD_DISPATCH_D(d, launch_scatter, ra, tiles, big_pts, "scatter_route", s);
      PKD_LAUNCH(k_copy_round<<<tiles, 256, 0, s>>>(ra, F));
    }
    if (nsmall) {
      PKD_DISPATCH_D(d, launch_route_small, ra, cur_small, R.d_n + 2, cur, nbk, R.bstart, R.blen, F, nsmall, s);
    }
    PKD_LAUNCH(k_route_emit<<<g1, ITEM_WARPS * 32, 0, s>>>(ua));
    PKD_CUDA(cudaMemcpyAsync(hctr, dctr, 68, cudaMemcpyDeviceToHost, s));
    PKD_CUDA(cudaStreamSynchronize(s));
    const uint32_t nnext = hctr[0], ntiles = hctr[1], ngroups = hctr[4];
    big_pts = hctr[16];
    groups_before = ngroups;
    rounds.push_back(R);
    cur = next;
    cur_big = next_big;
    cur_bigmap = next_bigmap;
    cur_small = next_small;
    ncur = nnext;
    tiles = ntiles;
    nbig = hctr[2];
    nsmall = hctr[3];
    w ^= 1;
  }
  const uint32_t ngroups = groups_before;
  trace_mark(s, "upd: route");

  // From here on, every exit clears the delete marks this batch sets (the
  // scratch must be zero for the next call).
  struct ClearMarks {
    TreeMem& t;
    const std::vector<RouteRound>& rounds;
    int HN;
    cudaStream_t s;
    bool on;
    ~ClearMarks() {
      if (!on) return;
      const bool ok = dev_fill(t.dead, 0, t.cap, s) == PKD_OK;
      for (const auto& R : rounds)
        PKD_LAUNCH(k_clear_aux<<<(unsigned)(((uint64_t)R.n * HN + 255) / 256), 256, 0, s>>>(R.slots, (uint64_t)R.n * HN,
                                                                                           t.aux));
      // (a leaf group's slot is a heap bucket of its round, cleared above)
      if (ok && cudaPeekAtLastError() == cudaSuccess) t.scratch_dirty = false;
    }
  } clear_marks{t, rounds, HN, s, !insert};
  if (!insert) t.scratch_dirty = true;

  // ---- match (delete) ----
  if (!insert && ngroups)
    PKD_DISPATCH_D(d, launch_match, groups, d_ngroups, ngroups, t.nodes, t.A, F, t.dead, t.aux, s);

  // ---- count, bottom-up ----
  for (int r = (int)rounds.size() - 1; r >= 0; --r) {
    RouteRound& R = rounds[r];
    ua.items = R.items;
    ua.nitems = R.d_n;
    ua.skel = R.skel;
    ua.slots = R.slots;
    ua.link = R.link;
    ua.fnd = R.fnd;
    ua.next_fnd = (r + 1 < (int)rounds.size()) ? rounds[r + 1].fnd : nullptr;
    ua.next_HN = HN;
    {
      const size_t smb = (size_t)ITEM_WARPS * HN * 2 * sizeof(uint32_t);
      static size_t set = 0;
      if (smb > 48 * 1024 && set < smb) {
        cudaFuncSetAttribute(k_aggregate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
        set = smb;
      }
      PKD_LAUNCH(k_aggregate<<<item_blocks(R.n), ITEM_WARPS * 32, smb, s>>>(ua));
    }
  }
  uint32_t total_changed = 0;
  PKD_CUDA(cudaMemcpyAsync(&total_changed, rounds[0].fnd + 1, 4, cudaMemcpyDeviceToHost, s));
  uint32_t* compact;
  PKD_TRY(sc.get(&compact, std::max<uint32_t>(ngroups, 1)));

  // ---- decide, top-down (sizes of the nodes that stay are only recorded) ----
  for (size_t r = 0; r < rounds.size(); ++r) {
    RouteRound& R = rounds[r];
    ua.items = R.items;
    ua.nitems = R.d_n;
    ua.skel = R.skel;
    ua.slots = R.slots;
    ua.link = R.link;
    ua.fnd = R.fnd;
    ua.nsz = R.nsz;
    ua.bstart = R.bstart;
    ua.blen = R.blen;
    ua.iflag = R.iflag;
    ua.next_iflag = (r + 1 < rounds.size()) ? rounds[r + 1].iflag : nullptr;
    {
      const size_t smb = (size_t)ITEM_WARPS * HN * (sizeof(int2) + 3 * sizeof(uint32_t));
      static size_t set = 0;
      if (smb > 48 * 1024 && set < smb) {
        cudaFuncSetAttribute(k_decide, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
        set = smb;
      }
      PKD_LAUNCH(k_decide<<<item_blocks(R.n), ITEM_WARPS * 32, smb, s>>>(ua));
    }
  }
  trace_mark(s, "upd: match+count+decide");
  if (ngroups) PKD_LAUNCH(k_leaf_items<<<(ngroups + 255) / 256, 256, 0, s>>>(ua, groups, d_ngroups, compact, d_ncompact));
  PKD_CUDA(cudaMemcpyAsync(hctr, dctr, 40, cudaMemcpyDeviceToHost, s));
  PKD_CUDA(cudaStreamSynchronize(s));
  const uint32_t nitems = hctr[5];
  const uint64_t total = *(unsigned long long*)(hctr + 6);
  const uint32_t ncompact = hctr[8];
  stat_items(insert ? "rebuilt_insert" : "rebuilt_delete", total);
  trace_mark(s, "upd: leaf items");

  // ---- rebuild ----
  // Nothing the tree shows has changed so far: the new sizes are recorded,
  // the leaves to compact are listed.  Every allocation of the rebuild comes
  // first; the new subtrees are built in fresh arena positions (past top);
  // the rebuild items' root records are saved and put back if the rebuild
  // fails, so PKD_ENOMEM leaves the tree as it was.
  if (nitems) {
    PKD_TRY(ensure_capacity(t, total, s));
    trace_mark(s, "upd: ensure capacity");
    uint32_t *isz, *ioff, *ipart, *saved_next;
    PKD_TRY(sc.get(&isz, nitems));
    PKD_TRY(sc.get(&ioff, nitems));
    PKD_TRY(sc.get(&ipart, ((uint64_t)nitems + SCAN_TILE - 1) / SCAN_TILE + 1));
    Seg* segs;
    PKD_TRY(sc.get(&segs, nitems));
    Node* saved_nodes;
    uint8_t* saved_dims;
    PKD_TRY(sc.get(&saved_nodes, nitems));
    PKD_TRY(sc.get(&saved_dims, nitems));
    PKD_TRY(sc.get(&saved_next, 1));
    // Capacity of the flatten's lists: every node of the old subtrees
    // appears once.  A subtree of P stored points has at most 2P - 1 nodes
    // unless deletes left empty leaves in it, so the first attempt is sized
    // by the stored points of the rebuilt subtrees (at most their new sizes
    // plus the points this batch deleted); when a level overflows it, the
    // flatten is redone with four entries per stored point of the tree.
    const uint64_t big_fcap = 4 * ((uint64_t)t.size + (uint64_t)nitems) + 1024;
    uint64_t fcap = 2 * (total + (insert ? 0ull : (uint64_t)total_changed) + (uint64_t)nitems) + 1024;
    if (knobs().front_cap > 0) fcap = (uint64_t)knobs().front_cap;
    fcap = std::max<uint64_t>(std::min(fcap, big_fcap), (uint64_t)nitems + 1024);  // the roots always fit
    Front *fa = nullptr, *fb = nullptr, *leaves = nullptr, *bigleaves = nullptr;
    uint32_t *ncnt = nullptr, *noff = nullptr, *npart = nullptr;
    if (insert) {
      PKD_TRY(sc.get(&ncnt, nitems));
      PKD_TRY(sc.get(&noff, nitems));
      PKD_TRY(sc.get(&npart, ((uint64_t)nitems + SCAN_TILE - 1) / SCAN_TILE + 1));
    }
    const unsigned gi = (nitems + 127) / 128;
    PKD_LAUNCH(k_item_sizes<<<gi, 128, 0, s>>>(items_out, d_nitems, isz));
    device_excl_scan(isz, ioff, nitems, ipart, s);
    PKD_LAUNCH(k_item_pos<<<gi, 128, 0, s>>>(items_out, d_nitems, ioff, t.top, segs, (uint32_t)p.phi));
    // flatten the old subtrees breadth first (capacity: every node of the
    // old subtrees appears once).  The levels run in batches whose counts
    // stay on the device; the host reads the frontier once per batch: one
    // level first (an insert's items are mostly leaves), then FRONT_BATCH
    // levels at a time (a rebuilt interior subtree is many levels deep).
    {
      uint32_t* fc = dctr + 12;  // [0] frontier, [1] overflow, [2] leaves, [3] big leaves
      uint32_t* lc;              // the frontier of every level of a batch
      PKD_TRY(sc.get(&lc, FRONT_BATCH + 1));
      const unsigned gexp = (unsigned)sm_count() * 8;
      for (int attempt = 0;; ++attempt) {
        const uint32_t fcap32 = (uint32_t)std::min<uint64_t>(fcap, 0xFFFFFFF0ull);
        const uint32_t bcap32 = (uint32_t)std::min<uint64_t>(fcap / BIG_LEAF + 16, 0xFFFFFFF0ull);
        PKD_TRY(sc.get(&fa, fcap32));
        PKD_TRY(sc.get(&fb, fcap32));
        PKD_TRY(sc.get(&leaves, fcap32));
        PKD_TRY(sc.get(&bigleaves, bcap32));
        PKD_TRY(dev_fill(fc, 0, 16, s));
        PKD_LAUNCH(k_front_init<<<gi, 128, 0, s>>>(items_out, d_nitems, fa, fc));
        int levels = 0;
        for (int batch = 1;; batch = FRONT_BATCH) {
          if (levels > 100000) return PKD_EINTERNAL;
          PKD_TRY(dev_fill(lc + 1, 0, (size_t)batch * 4, s));
          PKD_TRY(dev_copy_words(lc, fc, 1, s));
          for (int k = 0; k < batch; ++k) {
            PKD_LAUNCH(k_front_expand<<<gexp, 128, 0, s>>>(fa, lc + k, fb, lc + k + 1, leaves, fc + 2, bigleaves,
                                                            fc + 3, t.nodes, t.ndim, t.aux, insert ? 0 : 1, fcap32,
                                                            bcap32, fc + 1));
            std::swap(fa, fb);
          }
          levels += batch;
          PKD_TRY(dev_copy_words(fc, lc + batch, 1, s));
          PKD_CUDA(cudaMemcpyAsync(hctr + 12, fc, 16, cudaMemcpyDeviceToHost, s));
          PKD_CUDA(cudaStreamSynchronize(s));
          if (hctr[12] == 0 || hctr[13] != 0) break;
        }
        if (hctr[13] == 0) break;
        // a list overflowed: nothing the tree shows has changed yet
        if (fcap >= big_fcap) return PKD_EINTERNAL;
        stat_items("front_retries", 1);
        fcap = big_fcap;
      }
      const uint32_t nleaves = hctr[14], nbigleaves = hctr[15];
      if (nleaves)
        PKD_DISPATCH_D(d, launch_copy_leaves, leaves, fc + 2, nleaves, items_out, t.nodes, t.A, t.dead,
                       insert ? 0 : 1, s);
      if (nbigleaves)
        PKD_DISPATCH_D(d, launch_copy_big_leaves, bigleaves, fc + 3, nbigleaves, items_out, t.nodes, t.A, t.dead,
                       insert ? 0 : 1, s);
    }
    if (insert) {
      PKD_DISPATCH_D(d, launch_copy_new, items_out, d_nitems, nitems, F, t.A, s);
      PKD_LAUNCH(k_item_newcounts<<<gi, 128, 0, s>>>(items_out, d_nitems, ncnt));
      device_excl_scan(ncnt, noff, nitems, npart, s);
      PKD_DISPATCH_D(d, launch_copy_new_flat, items_out, d_nitems, noff, ncnt, m, F, t.A, s);
    }
    trace_mark(s, "upd: flatten + gather");
    PKD_LAUNCH(k_save_roots<<<gi, 128, 0, s>>>(items_out, d_nitems, t.nodes, t.ndim, saved_nodes, saved_dims));
    PKD_TRY(dev_copy_words(saved_next, t.shared_next, 1, s));
    BuildJob job;
    job.base = t.top;
    job.extent = std::max<uint64_t>(total, 1);
    job.dsegs = segs;
    job.dsegs_n = nitems;
    const int eb = run_build(t, job, s);
    if (eb != PKD_OK) {
      PKD_LAUNCH(k_restore_roots<<<gi, 128, 0, s>>>(items_out, d_nitems, t.nodes, t.ndim, saved_nodes, saved_dims));
      dev_copy_words(t.shared_next, saved_next, 1, s);
      return eb;
    }
    PKD_LAUNCH(k_item_leaves<<<gi, 128, 0, s>>>(items_out, d_nitems, t.nodes, t.ndim, (uint32_t)p.phi));
    trace_mark(s, "upd: rebuild");
  }

  // ---- the visible changes: nothing below allocates ----
  if (ncompact)  // delete: the reached leaves lose their deleted points
    PKD_DISPATCH_D(d, launch_compact, groups, compact, d_ncompact, ncompact, t.nodes, t.A, t.dead, s);
  for (const auto& R : rounds)
    PKD_LAUNCH(k_apply_sizes<<<(unsigned)(((uint64_t)R.n * HN + 255) / 256), 256, 0, s>>>(R.slots, R.nsz,
                                                                                         (uint64_t)R.n * HN, t.nodes));
  t.top += total;
  clear_marks.on = false;
  if (!insert) {
    PKD_TRY(dev_fill(t.dead, 0, t.cap, s));
    for (auto& R : rounds)
      PKD_LAUNCH(k_clear_aux<<<(unsigned)(((uint64_t)R.n * HN + 255) / 256), 256, 0, s>>>(R.slots, (uint64_t)R.n * HN, t.aux));
  }
  PKD_CUDA(cudaStreamSynchronize(s));
  if (!insert && cudaPeekAtLastError() == cudaSuccess) t.scratch_dirty = false;  // every mark is cleared
  trace_mark(s, "upd: cleanup");
  if (n_changed) *n_changed = total_changed;
  return PKD_OK;
}

}  // namespace pkd

using namespace pkd;

extern "C" {

int pkd_batch_insert(pkd_tree* tc, const int32_t* coords, const uint32_t* ids, uint64_t m, void* stream) {
  if (!tc) return PKD_EINVAL;
  if (m == 0) return PKD_OK;
  if (!coords || !ids) return PKD_EINVAL;
  TreeMem& t = tc->m;
  if (t.size + m >= (1ull << 31)) return PKD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  TreeTouch touch{&t, s};
  bool ok;
  PKD_TRY_(validate_coords(coords, m * (uint64_t)t.p.d, s, &ok));
  if (!ok) return PKD_EINVAL;
  PKD_TRY_(check_status(t, s));
  // the batch's ids take their slots first: a stored or repeated id rejects
  // the whole batch before the tree changes
  PKD_TRY_(ids_reserve(t, m, s));
  uint64_t* slots = nullptr;
  PKD_TRY_(dalloc(&slots, m, s));
  ids_claim(t, coords, ids, m, slots, s);
  t.ids.used += m;
  int fl = 0;
  int e = read_idflags(t, s, &fl);
  if (e == PKD_OK && fl) e = (fl & IDF_FULL) ? PKD_EINTERNAL : PKD_EINVAL;
  uint64_t changed = 0;
  if (e == PKD_OK) e = run_update(t, coords, ids, nullptr, m, true, &changed, s);
  if (e == PKD_OK) e = check_status(t, s);
  if (e == PKD_OK) {
    t.size += m;
    t.ids.live += m;
    if (t.bbox_on) e = boxes_compute(t, s);
  } else {
    ids_unclaim(t, slots, m, s);
  }
  dfree(slots, s);
  return e;
}

int pkd_batch_delete(pkd_tree* tc, const uint32_t* ids, uint64_t m, uint64_t* n_deleted, void* stream) {
  if (!tc) return PKD_EINVAL;
  if (n_deleted) *n_deleted = 0;
  if (m == 0) return PKD_OK;
  if (!ids) return PKD_EINVAL;
  TreeMem& t = tc->m;
  if (m >= (1ull << 31)) return PKD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  TreeTouch touch{&t, s};
  PKD_TRY_(check_status(t, s));
  // ids -> coordinates: every LIVE id of the batch is taken once (repeats and
  // unknown or deleted ids are skipped) and staged for the sieve
  Scratch sc{s, {}};
  const int d = t.p.d;
  int32_t* wc;
  uint32_t *wid, *cnt;
  uint64_t* wslots;
  PKD_TRY(sc.get(&wc, (size_t)d * m));
  PKD_TRY(sc.get(&wid, m));
  PKD_TRY(sc.get(&wslots, m));
  PKD_TRY(sc.get(&cnt, 1));
  PKD_TRY(dev_fill(cnt, 0, 4, s));
  Pts W{wc, wid, m};
  ids_take(t, ids, m, W, wslots, cnt, s);
  PinnedBlock hb(s);
  if (!hb.p) return PKD_ENOMEM;
  PKD_CUDA(cudaMemcpyAsync(hb.p, cnt, 4, cudaMemcpyDeviceToHost, s));
  int fl = 0;
  PKD_TRY(read_idflags(t, s, &fl));  // synchronises s
  const uint32_t taken = *(const uint32_t*)hb.p;
  if (fl) {
    ids_restore(t, wslots, taken, s);
    return PKD_EINTERNAL;
  }
  stat_items("delete_gather", taken);
  if (taken == 0) return PKD_OK;
  uint64_t removed = 0;
  int e = run_update(t, nullptr, nullptr, &W, taken, false, &removed, s);
  if (e == PKD_OK) e = check_status(t, s);
  if (e == PKD_OK && removed != taken) {
    fprintf(stderr, "pkd: delete removed %llu points for %u live ids\n", (unsigned long long)removed, taken);
    e = PKD_EINTERNAL;
  }
  if (e != PKD_OK) ids_restore(t, wslots, taken, s);
  if (e == PKD_OK) {
    t.size -= removed;
    t.ids.live -= removed;
    if (n_deleted) *n_deleted = removed;
    if (t.bbox_on) e = boxes_compute(t, s);
  }
  return e;
}

}  // extern "C"
