// Batched build of many independent trees in one pass.
//
// Every tree of the batch is a root segment of one BuildJob: the sieve
// rounds process the large trees' segments side by side (one grid per round
// for all of them) and the base-case kernels finish every small tree and
// every bucket of every tree in the same launches, so a batch of T trees
// costs the launches and host synchronisations of one build instead of T.
// Each tree is exactly the tree pkd_build would give for its own points
// (Alg. 1 per tree: its own root at depth 0, its own samples).
//
// The trees share one arena and one node array: tree i's points occupy
// arena positions [offsets[i], offsets[i+1]) and its root is node slot i.
#include <vector>

#include "engine.hpp"
#include "tree_impl.hpp"

struct pkd_forest {
  pkd::TreeMem m;
  std::vector<uint64_t> offsets;  // T + 1
};

using namespace pkd;

extern "C" {

int pkd_build_forest(const int32_t* coords, const uint32_t* ids, const uint64_t* offsets, uint32_t n_trees,
                     const pkd_params* params, void* stream, pkd_forest** out) {
  if (!out || !offsets || n_trees == 0 || n_trees >= (1u << 24)) return PKD_EINVAL;
  *out = nullptr;
  int e = check_params(params);
  if (e) return e;
  if (offsets[0] != 0) return PKD_EINVAL;
  for (uint32_t i = 0; i < n_trees; ++i)
    if (offsets[i + 1] < offsets[i]) return PKD_EINVAL;
  const uint64_t n = offsets[n_trees];
  if (n >= (1ull << 31)) return PKD_EINVAL;
  if (n > 0 && !coords) return PKD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Params p{params->d, params->phi, params->lambda, params->sigma_log2, params->sigma_os,
           params->count_mode, params->alpha_num, params->alpha_den, params->seed};
  bool ok;
  e = validate_coords(coords, n * (uint64_t)p.d, s, &ok);
  if (e) return e;
  if (!ok) return PKD_EINVAL;
  pkd_forest* f = new pkd_forest();
  f->offsets.assign(offsets, offsets + n_trees + 1);
  const uint64_t cap = n + n / 4 + 4096;
  // node slots 0..T-1 are the roots; the shared region also holds the
  // skeleton nodes of every tree's sieve rounds
  e = tree_alloc(f->m, p, cap, shared_region_for(p, cap) + 2 * (uint64_t)n_trees, s);
  if (e) {
    delete f;
    return e;
  }
  const uint32_t first_free = n_trees;
  dev_store(f->m.shared_next, &first_free, 4, s);
  BuildJob job;
  job.input_coords = coords;
  job.input_ids = ids;
  job.base = 0;
  job.extent = std::max<uint64_t>(n, 1);
  job.segs.reserve(n_trees);
  for (uint32_t i = 0; i < n_trees; ++i)
    job.segs.push_back(Seg{offsets[i], (uint32_t)(offsets[i + 1] - offsets[i]), 0, i, IN_INPUT});
  e = run_build(f->m, job, s);
  if (e == PKD_OK) e = check_status(f->m, s);
  if (e) {
    tree_release(f->m);
    delete f;
    return e;
  }
  f->m.size = n;
  f->m.top = n;
  tree_touch(f->m, s);
  *out = f;
  return PKD_OK;
}

uint32_t pkd_forest_trees(const pkd_forest* f) { return f ? (uint32_t)(f->offsets.size() - 1) : 0u; }

uint64_t pkd_forest_size(const pkd_forest* f, uint32_t tree) {
  if (!f || tree + 1 >= f->offsets.size()) return 0;
  return f->offsets[tree + 1] - f->offsets[tree];
}

int pkd_forest_export(const pkd_forest* f, uint32_t tree, uint8_t* dims, int32_t* splits, uint64_t* sizes,
                      uint64_t* n_nodes, uint32_t* leaf_ids, uint64_t* leaf_offsets, uint64_t* n_leaves) {
  if (!f || tree + 1 >= f->offsets.size()) return PKD_EINVAL;
  HostTree h;
  int e = download_tree(f->m, h);
  if (e) return e;
  return export_from(h, tree, f->m.top, pkd_forest_size(f, tree), dims, splits, sizes, n_nodes, leaf_ids,
                     leaf_offsets, n_leaves);
}

int pkd_forest_knn(const pkd_forest* f, uint32_t tree, const int32_t* queries, uint64_t q, int k,
                   uint32_t* out_ids, int64_t* out_d2, void* stream) {
  if (!f || tree + 1 >= f->offsets.size()) return PKD_EINVAL;
  return knn_on(const_cast<TreeMem&>(f->m), tree, queries, q, k, out_ids, out_d2, (cudaStream_t)stream);
}

void pkd_forest_free(pkd_forest* f) {
  if (!f) return;
  tree_wait_uses(f->m);  // the frees below are ordered after every call's work
  tree_release(f->m);
  delete f;
}

}  // extern "C"
