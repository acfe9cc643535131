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
// A non-blocking stream of the library's own on the current device, for work
// that overlaps the caller's stream within one call.
cudaStream_t side_stream();

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

// Id table (ids.cu; layout in ids.cuh).
//  ids_create   an empty table for n ids with room to grow
//  ids_reserve  room for `extra` more claims (rehashes into a larger table)
//  ids_claim    launch: points take their ids' slots (LIVE); slots[i] gets
//               the claimed slot or ID_NO_SLOT (slots may be NULL); a bad id
//               raises IDF_BAD_ID in the status word; ids NULL (0..m-1) only
//               into a new, empty table
//  ids_unclaim  launch: claimed slots go back to DEAD (a rejected batch)
//  ids_take     launch: LIVE ids become DEAD and their (coords, id) are
//               appended to W (count is the device append counter), the slot
//               of each appended point to wslots
//  ids_restore  launch: taken slots become LIVE again (a failed delete)
//  read_idflags synchronises `s`, returns and clears the flags
int ids_create(TreeMem& t, uint64_t n, cudaStream_t s);
int ids_reserve(TreeMem& t, uint64_t extra, cudaStream_t s);
void ids_release(IdTable& T, cudaStream_t s);
void ids_claim(TreeMem& t, const int32_t* coords, const uint32_t* ids, uint64_t m, uint64_t* slots, cudaStream_t s);
void ids_unclaim(TreeMem& t, const uint64_t* slots, uint64_t m, cudaStream_t s);
void ids_take(TreeMem& t, const uint32_t* ids, uint64_t m, Pts W, uint64_t* wslots, uint32_t* count,
              cudaStream_t s);
void ids_restore(TreeMem& t, const uint64_t* wslots, uint64_t n, cudaStream_t s);
int read_idflags(TreeMem& t, cudaStream_t s, int* flags);

// Stored bounding boxes (boxes.cu): compute every node's tight box into
// t.bbox (allocated or grown to node_cap), or free them.
int boxes_compute(TreeMem& t, cudaStream_t s);
void boxes_release(TreeMem& t, cudaStream_t s);

// k-NN (see pkd_knn) on the tree rooted at node slot `root`.
int knn_on(TreeMem& t, uint32_t root, const int32_t* queries, uint64_t q, int k, uint32_t* out_ids,
           int64_t* out_d2, cudaStream_t s);

}  // namespace pkd
