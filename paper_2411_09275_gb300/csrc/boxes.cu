// Stored bounding boxes (the paper's Pkd-bb variant, Sec. 6 "Study of the
// Impact of Bounding Boxes"): every node keeps the tight box of the points
// in its subtree, and the queries prune with it instead of the subspace the
// splitters above the node imply.  Query answers are the same; only the
// pruning differs (tighter, at the price of 8d bytes per node slot).
//
// Layout: box[slot * 2d + j] = lowest coordinate j in the subtree,
// box[slot * 2d + d + j] = highest; an empty subtree has lo = INT32_MAX and
// hi = INT32_MIN in every dimension (disjoint from every query box, and at
// infinite distance from every point).
//
// The boxes are computed bottom-up: a breadth-first walk from the root
// records the nodes level by level, every leaf takes the min / max of its
// points, and then each level, deepest first, takes the union of its
// children's boxes.
#include <algorithm>
#include <climits>
#include <cstdio>

#include "sieve.cuh"
#include "tree_impl.hpp"

namespace pkd {

namespace {

constexpr int BB_THREADS = 256;

// Level expansion: every interior node of level `f` appends its two children
// to level `g` (block-aggregated appends, one atomic per block).
__global__ void __launch_bounds__(BB_THREADS) k_bb_expand(const uint32_t* f, uint32_t nf, uint32_t* g,
                                                          uint32_t* ng, const Node* nodes, const uint8_t* ndim,
                                                          uint32_t cap, DevStatus* st) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool have = i < nf;
  uint32_t v = 0;
  bool inner = false;
  if (have) {
    v = f[i];
    inner = ndim[v] != PKD_LEAF;
  }
  const uint32_t c[1] = {inner ? 2u : 0u};
  uint32_t* const ctr[1] = {ng};
  uint32_t first[1];
  block_reserve<1>(c, ctr, first);
  if (!inner) return;
  if (first[0] + 2 > cap) {
    set_error(st, DERR_CAPACITY, 850);
    return;
  }
  const Node nd = nodes[v];
  g[first[0]] = nd.a;
  g[first[0] + 1] = nd.b;
}

// One level, deepest first: a leaf's box from its points (one warp per
// leaf, lanes striding over the points), an interior node's as the union of
// its children's boxes (computed on the previous launch).
template <int D>
__global__ void __launch_bounds__(BB_THREADS) k_bb_level(const uint32_t* lv, uint32_t n, const Node* nodes,
                                                         const uint8_t* ndim, Pts A, int32_t* box) {
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;  // warp-uniform
  const uint32_t v = lv[w];
  const Node nd = nodes[v];
  int32_t lo[D], hi[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    lo[j] = INT_MAX;
    hi[j] = INT_MIN;
  }
  if (ndim[v] == PKD_LEAF) {
    for (uint32_t i = lane; i < nd.size; i += 32) {
      const uint64_t g = (uint64_t)nd.a + i;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int32_t x = A.c[(uint64_t)j * A.stride + g];
        lo[j] = min(lo[j], x);
        hi[j] = max(hi[j], x);
      }
    }
  } else if (lane < 2) {
    const int32_t* cb = box + (uint64_t)(lane == 0 ? nd.a : nd.b) * 2 * D;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      lo[j] = cb[j];
      hi[j] = cb[D + j];
    }
  }
#pragma unroll
  for (int j = 0; j < D; ++j) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      lo[j] = min(lo[j], __shfl_xor_sync(FULL_MASK, lo[j], o));
      hi[j] = max(hi[j], __shfl_xor_sync(FULL_MASK, hi[j], o));
    }
  }
  if (lane == 0) {
    int32_t* b = box + (uint64_t)v * 2 * D;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      b[j] = lo[j];
      b[D + j] = hi[j];
    }
  }
}

template <int D>
void launch_bb_level(const uint32_t* lv, uint32_t n, const TreeMem& t, cudaStream_t s) {
  const unsigned blocks = (unsigned)(((uint64_t)n * 32 + BB_THREADS - 1) / BB_THREADS);
  PKD_LAUNCH(k_bb_level<D><<<blocks, BB_THREADS, 0, s>>>(lv, n, t.nodes, t.ndim, t.A, t.bbox));
}

}  // namespace

int boxes_compute(TreeMem& t, cudaStream_t s) {
  const int d = t.p.d;
  if (!t.bbox || t.bbox_cap < t.node_cap) {
    big_free(t.bbox, s);
    t.bbox = nullptr;
    t.bbox_cap = 0;
    cudaError_t e = big_alloc((void**)&t.bbox, (size_t)t.node_cap * 2 * d * 4, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? PKD_ENOMEM : PKD_ECUDA;
    }
    t.bbox_cap = t.node_cap;
  }
  // every node appears once across the levels, and every node has a slot of
  // its own among the used ones
  const uint64_t used = t.shared_cap + 2 * t.top;
  const uint64_t cap64 = used + 1;
  if (cap64 >= 0xFFFFFFF0ull) return PKD_EINVAL;
  const uint32_t cap = (uint32_t)cap64;
  Scratch sc{s, {}};
  uint32_t *all, *ctr;
  PKD_TRY(sc.get(&all, cap));
  PKD_TRY(sc.get(&ctr, 1));
  PinnedBlock hb(s);
  if (!hb.p) return PKD_ENOMEM;
  uint32_t* hn = (uint32_t*)hb.p;
  PKD_TRY_(dev_store(all, &t.root, 4, s));
  std::vector<uint64_t> level_start{0, 1};
  for (int lev = 0; lev < 100000; ++lev) {
    const uint64_t a = level_start[lev], b = level_start[lev + 1];
    const uint32_t nf = (uint32_t)(b - a);
    if (nf == 0) break;
    PKD_TRY(dev_fill(ctr, 0, 4, s));
    PKD_LAUNCH(k_bb_expand<<<(nf + BB_THREADS - 1) / BB_THREADS, BB_THREADS, 0, s>>>(
        all + a, nf, all + b, ctr, t.nodes, t.ndim, (uint32_t)(cap - b), t.st));
    PKD_CUDA(cudaMemcpyAsync(hn, ctr, 4, cudaMemcpyDeviceToHost, s));
    PKD_CUDA(cudaStreamSynchronize(s));
    const uint64_t ng = std::min<uint64_t>(hn[0], cap - b);
    level_start.push_back(b + ng);
  }
  for (int lev = (int)level_start.size() - 2; lev >= 0; --lev) {
    const uint64_t a = level_start[lev], b = level_start[lev + 1];
    if (b > a) PKD_DISPATCH_D(d, launch_bb_level, all + a, (uint32_t)(b - a), t, s);
  }
  PKD_CUDA(cudaGetLastError());
  return check_status(t, s);
}

void boxes_release(TreeMem& t, cudaStream_t s) {
  big_free(t.bbox, s);
  t.bbox = nullptr;
  t.bbox_cap = 0;
}

}  // namespace pkd

using namespace pkd;

extern "C" {

int pkd_set_bounding_boxes(pkd_tree* tc, int enable, void* stream) {
  if (!tc || (enable != 0 && enable != 1)) return PKD_EINVAL;
  TreeMem& t = tc->m;
  cudaStream_t s = (cudaStream_t)stream;
  TreeTouch touch{&t, s};
  PKD_TRY_(check_status(t, s));
  if (!enable) {
    t.bbox_on = false;
    boxes_release(t, s);
    return PKD_OK;
  }
  const int e = boxes_compute(t, s);
  t.bbox_on = e == PKD_OK;
  if (e != PKD_OK) boxes_release(t, s);
  return e;
}

int pkd_export_boxes(const pkd_tree* tc, int32_t* lo, int32_t* hi, uint64_t n_nodes) {
  if (!tc || !lo || !hi) return PKD_EINVAL;
  const TreeMem& t = tc->m;
  if (!t.bbox_on) return PKD_EINVAL;
  HostTree h;
  PKD_TRY_(download_tree(t, h, false));
  const int d = t.p.d;
  const uint64_t used = t.shared_cap + 2 * t.top;
  std::vector<int32_t> box((size_t)used * 2 * d);
  PKD_CUDA(cudaMemcpy(box.data(), t.bbox, box.size() * 4, cudaMemcpyDeviceToHost));
  // pre-order, as pkd_export
  std::vector<uint32_t> stack{t.root};
  uint64_t k = 0;
  while (!stack.empty()) {
    const uint32_t v = stack.back();
    stack.pop_back();
    if (v >= used || k >= n_nodes) return PKD_EINVAL;
    for (int j = 0; j < d; ++j) {
      lo[k * d + j] = box[(size_t)v * 2 * d + j];
      hi[k * d + j] = box[(size_t)v * 2 * d + d + j];
    }
    ++k;
    if (h.ndim[v] != PKD_LEAF) {
      stack.push_back(h.nodes[v].b);
      stack.push_back(h.nodes[v].a);
    }
  }
  return k == n_nodes ? PKD_OK : PKD_EINVAL;
}

}  // extern "C"
