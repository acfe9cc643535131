// Internal declarations shared by the C-ABI translation units.
#pragma once

#include <vector>

#include "engine.hpp"

struct pkd_tree {
  pkd::TreeMem m;
};

namespace pkd {

#define PKD_TRY_(x)              \
  do {                           \
    int _r = (x);                \
    if (_r != PKD_OK) return _r; \
  } while (0)

int check_params(const pkd_params* p);
int validate_coords(const int32_t* c, uint64_t cnt, cudaStream_t s, bool* ok);
int tree_alloc(TreeMem& t, const Params& p, uint64_t cap, uint64_t shared_cap, cudaStream_t s);
void tree_release(TreeMem& t);
uint64_t shared_region_for(const Params& p, uint64_t n);

// Host copy of the node arrays (and, optionally, the arena ids) for export.
struct HostTree {
  std::vector<Node> nodes;
  std::vector<uint8_t> ndim;
  std::vector<uint32_t> ids;
};
int download_tree(const TreeMem& t, HostTree& h, bool with_ids = true);

// Canonical form (see pkd_export) of the tree rooted at node slot `root`
// holding `size` points of an arena whose positions [0, top) are in use.
int export_from(const HostTree& h, uint32_t root, uint64_t top, uint64_t size, uint8_t* dims, int32_t* splits,
                uint64_t* sizes, uint64_t* n_nodes, uint32_t* leaf_ids, uint64_t* leaf_offsets, uint64_t* n_leaves);

// k-NN (see pkd_knn) on the tree rooted at node slot `root`.
int knn_on(TreeMem& t, uint32_t root, const int32_t* queries, uint64_t q, int k, uint32_t* out_ids,
           int64_t* out_d2, cudaStream_t s);

}  // namespace pkd
