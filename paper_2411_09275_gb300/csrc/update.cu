// Batch updates (Alg. 2 and Sec. 4.2).
#include "engine.hpp"
#include "tree_impl.hpp"

using namespace pkd;

extern "C" {

int pkd_batch_insert(pkd_tree* t, const int32_t* coords, const uint32_t* ids, uint64_t m,
                     void* stream) {
  (void)t;
  (void)coords;
  (void)ids;
  (void)m;
  (void)stream;
  return PKD_EINVAL;
}

int pkd_batch_delete(pkd_tree* t, const int32_t* coords, const uint32_t* ids, uint64_t m,
                     uint64_t* n_deleted, void* stream) {
  (void)t;
  (void)coords;
  (void)ids;
  (void)m;
  (void)n_deleted;
  (void)stream;
  return PKD_EINVAL;
}

}  // extern "C"
