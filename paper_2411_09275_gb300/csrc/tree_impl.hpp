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

}  // namespace pkd
