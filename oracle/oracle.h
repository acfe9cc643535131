/*
 * Pkd-tree CPU oracle: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded C restatement of the Pkd-tree of
 * "Parallel kd-tree with Batch Updates" (Men, Shen, Gu, Sun, SIGMOD 2025):
 * construction (Alg. 1, Sec. 3.1), batch insertion (Alg. 2, Sec. 4.1), batch
 * deletion (Sec. 4.2), k-NN and range count (Sec. 5 "Queries").  It is used
 * by the tests, by the package's smoke check and by the CPU-baseline leg of
 * the benchmark, and by nothing else.  It shares no code with the CUDA path.
 *
 * Points carry int32 coordinates in [0, 2^30) and a uint32 id.  The tree is a
 * deterministic function of (point multiset, ids, parameters, seed): samples
 * are chosen by a hash of (seed, depth, id), medians are exact on the sample,
 * and splitting ties go right.
 */
#ifndef PKD_ORACLE_H
#define PKD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_DMAX 8

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2 };

typedef struct {
  int d;            /* dimensions, 1..8 */
  int phi;          /* leaf wrap: a node of at most phi points is a leaf */
  int lambda;       /* skeleton levels built per sieve round, 1..10 */
  int sigma_log2;   /* rate mode: sample rate 2^-sigma_log2 (0 = every point) */
  int sigma_os;     /* oversampling: a skeleton node splits only with >= 2*sigma_os samples */
  int count_mode;   /* 1: sample about 2^lambda*sigma_os points per node (Alg. 1) */
  int alpha_num;    /* balance parameter alpha = alpha_num / alpha_den, 0 <= alpha <= 1/2 */
  int alpha_den;
  uint64_t seed;
} orc_params;

typedef struct orc_tree orc_tree;

/* Alg. 1: build over coords[n][d] with ids (NULL -> 0..n-1).  NULL on error
 * (ORC_EINVAL also when two points share an id or an id is 0xFFFFFFFF, the
 * k-NN padding value: ids name the points, so they are unique). */
orc_tree* orc_build(const int32_t* coords, const uint32_t* ids, uint64_t n,
                    const orc_params* p, int* err);
/* The same build for a subtree whose root sits at tree depth `depth` (the
 * depth salts the sample hash); the rebuilds of Alg. 2 use it. */
orc_tree* orc_build_at_depth(const int32_t* coords, const uint32_t* ids, uint64_t n,
                             const orc_params* p, uint32_t depth, int* err);
/* Alg. 2: insert m points.  Returns ORC_OK, or ORC_EINVAL with the tree
 * unchanged when a coordinate is out of range, an id is 0xFFFFFFFF, an id
 * names a point already in the tree, or two batch points share an id. */
int orc_insert(orc_tree* t, const int32_t* coords, const uint32_t* ids, uint64_t m);
/* Sec. 4.2: delete the points named by ids.  Each id is looked up among the
 * stored points to find its coordinates; ids that name no stored point and
 * repeats of an id are skipped.  *n_deleted = points removed. */
int orc_delete(orc_tree* t, const uint32_t* ids, uint64_t m, uint64_t* n_deleted);
void orc_free(orc_tree* t);

uint64_t orc_size(const orc_tree* t);
int orc_height(const orc_tree* t); /* edges on the longest root-to-leaf path */

/* Canonical form: nodes in pre-order (interior: dim, split, size; leaf:
 * dim 0xFF, split 0, size = point count), leaves in in-order with their ids
 * sorted ascending; leaf_offsets has n_leaves + 1 entries.  Any NULL buffer
 * is skipped, so a first call with NULL buffers returns the two counts. */
int orc_export(const orc_tree* t, uint8_t* dims, int32_t* splits, uint64_t* sizes,
               uint64_t* n_nodes, uint32_t* leaf_ids, uint64_t* leaf_offsets,
               uint64_t* n_leaves);
/* Leaf contents with coordinates, in in-order: ids[n], coords[n][d]. */
int orc_points(const orc_tree* t, uint32_t* ids, int32_t* coords);

/* k-NN: for every query the k smallest (squared distance, id) pairs in
 * lexicographic order; slots past the tree size hold id 0xFFFFFFFF and
 * distance INT64_MAX.  _brute scans every point (the definition), _tree runs
 * the depth-first search of Sec. 5. */
void orc_knn_brute(const orc_tree* t, const int32_t* q, uint64_t nq, int k,
                   uint32_t* out_ids, int64_t* out_d2);
void orc_knn_tree(const orc_tree* t, const int32_t* q, uint64_t nq, int k,
                  uint32_t* out_ids, int64_t* out_d2);
/* Range count over closed boxes lo[i][j] <= x_j <= hi[i][j]. */
void orc_range_count_brute(const orc_tree* t, const int32_t* lo, const int32_t* hi,
                           uint64_t nq, uint64_t* out);
void orc_range_count_tree(const orc_tree* t, const int32_t* lo, const int32_t* hi,
                          uint64_t nq, uint64_t* out);

/* Building blocks, exported so tests can pin them one by one. */
uint64_t orc_mix64(uint64_t z);
uint64_t orc_sample_hash(uint64_t seed, uint32_t depth, uint32_t id);
int orc_sample_shift(const orc_params* p, uint64_t n);
int orc_is_sampled(uint64_t seed, uint32_t depth, uint32_t id, int shift);
/* Splitter rule R on pts[n][d]: returns 0 and (dim, x), or -1 when the
 * points are all identical (no split exists). */
int orc_split_rule(const int32_t* pts, uint64_t n, int d, int* dim, int32_t* x);
int orc_balanced(uint64_t left, uint64_t total, int alpha_num, int alpha_den);

#ifdef __cplusplus
}
#endif
#endif
