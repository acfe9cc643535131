/*
 * Pkd-tree CPU oracle: TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Plain single-threaded C, written from the paper's definitions:
 *   - kd-tree, splitters, weight balance ......... Sec. 2 ("The kd-Tree")
 *   - construction: sample, skeleton, sieve ...... Alg. 1, Sec. 3.1
 *   - leaf wrap, heavy (duplicate) leaves ........ Sec. 2, Sec. 5, App. C
 *   - batch insertion ............................ Alg. 2, Sec. 4.1
 *   - batch deletion (two rounds) ................ Sec. 4.2
 *   - k-NN and range count ....................... Sec. 5 ("Queries")
 *
 * Readings of the paper (where it is silent or leaves a choice open):
 *   R1 sampling: a point is in the sample of a subproblem at tree depth t iff
 *      H(seed, t, id) >> (64 - s) == 0, H = SplitMix64's finaliser of
 *      seed ^ t*K_DEPTH ^ id*K_ID.  s is fixed (rate mode, rate 2^-s) or
 *      s = max(0, floor(log2(|P| / (2^lambda * sigma_os)))) (count mode, about
 *      2^lambda*sigma_os samples as in Alg. 1).  Without replacement.
 *   R2 skeleton: a skeleton node is a bucket when it sits lambda levels down,
 *      holds fewer than 2*sigma_os samples, or holds identical samples
 *      (Lemma 3.1 relies on every split seeing >= 2*sigma_os samples).
 *      When the skeleton root itself is a bucket the subproblem takes one
 *      level of the plain construction instead (the base case of Alg. 1).
 *   R3 splitter rule: widest stretch of the set (ties: lowest dimension),
 *      coordinate = element of rank floor(|X|/2) on that dimension; when no
 *      element lies strictly below it, the next larger distinct value.
 *      Left = strictly smaller (Sec. 2), so equal coordinates go right.
 *   R4 leaves: |P| <= phi -> leaf; all points identical -> one (heavy) leaf
 *      of any size holding every id (App. C keeps coordinate + count).
 *   R5 balance: 0.5 - alpha <= L/N <= 0.5 + alpha, inclusive, in integers.
 *      The test is applied to the nodes an update reaches: Sec. 4.1 rebuilds
 *      a node that the insertion makes unbalanced, so a node whose
 *      subtree receives no updated point is left as it is, even when it was
 *      already unbalanced (sampled splits can leave it so; rebuilding it at
 *      its own depth would draw a new sample and could change it).
 *      A node whose size drops to 0 becomes an empty leaf.
 *   R6 deletion key: the id.  Sec. 4.2 deletes points; ids name them.  An
 *      id is looked up among the stored points for its coordinates, which
 *      are then sieved as Sec. 4.2 sieves a point; ids that name no stored
 *      point (never inserted, or deleted already) and repeats are skipped,
 *      as round 1 discards points that are not in the tree.
 *   R9 ids name points: every id in a tree is unique and not 0xFFFFFFFF (the
 *      k-NN padding value).  A build with a repeated id, or an insert whose
 *      batch repeats an id or names a stored point, is rejected whole.
 */
#include "oracle.h"

#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_K_DEPTH 0x9E3779B97F4A7C15ull
#define ORC_K_ID 0xC2B2AE3D27D4EB4Full
#define ORC_COORD_LIMIT ((int64_t)1 << 30)

typedef struct {
  uint32_t id;
  int32_t x[ORC_DMAX];
} opt;

typedef struct onode {
  int leaf;
  int dim;
  int32_t split;
  uint64_t size;
  struct onode* lc;
  struct onode* rc;
  opt* pts;            /* leaf payload, size entries */
  unsigned char* dead; /* deletion marks during orc_delete */
  uint64_t ndead;      /* deleted records in the subtree during orc_delete */
} onode;

struct orc_tree {
  orc_params p;
  onode* root;
};

static void* xmalloc(size_t n) {
  void* r = malloc(n ? n : 1);
  if (!r) {
    fprintf(stderr, "pkd oracle: out of memory\n");
    abort();
  }
  return r;
}

/* A growable array of points. */
typedef struct {
  opt* a;
  uint64_t n, cap;
} ovec;

static void ovec_push(ovec* v, const opt* p) {
  if (v->n == v->cap) {
    v->cap = v->cap ? 2 * v->cap : 16;
    opt* b = (opt*)xmalloc(v->cap * sizeof(opt));
    if (v->n) memcpy(b, v->a, v->n * sizeof(opt));
    free(v->a);
    v->a = b;
  }
  v->a[v->n++] = *p;
}

/* ------------------------------------------------------------------ */
/* Sampling (Alg. 1 "Uniformly sample"; reading R1)                     */
/* ------------------------------------------------------------------ */

uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t orc_sample_hash(uint64_t seed, uint32_t depth, uint32_t id) {
  return orc_mix64(seed ^ ((uint64_t)depth * ORC_K_DEPTH) ^ ((uint64_t)id * ORC_K_ID));
}

int orc_sample_shift(const orc_params* p, uint64_t n) {
  if (!p->count_mode) return p->sigma_log2;
  uint64_t target = ((uint64_t)1 << p->lambda) * (uint64_t)p->sigma_os;
  int s = 0;
  while (s < 40 && (target << (s + 1)) <= n) ++s;
  return s;
}

int orc_is_sampled(uint64_t seed, uint32_t depth, uint32_t id, int shift) {
  if (shift == 0) return 1;
  return (orc_sample_hash(seed, depth, id) >> (64 - shift)) == 0;
}

/* ------------------------------------------------------------------ */
/* Splitter rule (Sec. 2: widest dimension, median; reading R3)         */
/* ------------------------------------------------------------------ */

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

static int all_identical(const opt* X, uint64_t n, int d) {
  for (uint64_t i = 1; i < n; ++i)
    for (int j = 0; j < d; ++j)
      if (X[i].x[j] != X[0].x[j]) return 0;
  return 1;
}

static int rule_R(const opt* X, uint64_t n, int d, int* dim_out, int32_t* x_out) {
  if (n == 0) return -1;
  int best = -1;
  int64_t best_ext = 0;
  for (int j = 0; j < d; ++j) {
    int32_t mn = X[0].x[j], mx = X[0].x[j];
    for (uint64_t i = 1; i < n; ++i) {
      if (X[i].x[j] < mn) mn = X[i].x[j];
      if (X[i].x[j] > mx) mx = X[i].x[j];
    }
    if ((int64_t)mx - mn > best_ext) {
      best_ext = (int64_t)mx - mn;
      best = j;
    }
  }
  if (best < 0) return -1; /* every point identical: no splitter */
  int32_t* v = (int32_t*)xmalloc(n * sizeof(int32_t));
  for (uint64_t i = 0; i < n; ++i) v[i] = X[i].x[best];
  qsort(v, n, sizeof(int32_t), cmp_i32);
  int32_t x = v[n / 2];
  if (v[0] == x) { /* nothing strictly left of x: take the next distinct value */
    uint64_t i = 0;
    while (v[i] == v[0]) ++i;
    x = v[i];
  }
  free(v);
  *dim_out = best;
  *x_out = x;
  return 0;
}

int orc_split_rule(const int32_t* pts, uint64_t n, int d, int* dim, int32_t* x) {
  if (d < 1 || d > ORC_DMAX) return -1;
  opt* X = (opt*)xmalloc(n * sizeof(opt));
  for (uint64_t i = 0; i < n; ++i) {
    X[i].id = (uint32_t)i;
    for (int j = 0; j < d; ++j) X[i].x[j] = pts[i * d + j];
  }
  int r = rule_R(X, n, d, dim, x);
  free(X);
  return r;
}

int orc_balanced(uint64_t left, uint64_t total, int alpha_num, int alpha_den) {
  /* 0.5 - a <= L/N <= 0.5 + a  <=>  (den - 2num) N <= 2 den L <= (den + 2num) N */
  uint64_t den = (uint64_t)alpha_den, num = (uint64_t)alpha_num;
  uint64_t lhs = 2 * den * left;
  return lhs >= (den - 2 * num) * total && lhs <= (den + 2 * num) * total;
}

/* ------------------------------------------------------------------ */
/* Tree nodes                                                            */
/* ------------------------------------------------------------------ */

static onode* make_leaf(const opt* P, uint64_t n) {
  onode* v = (onode*)calloc(1, sizeof(onode));
  if (!v) abort();
  v->leaf = 1;
  v->dim = -1;
  v->size = n;
  v->pts = (opt*)xmalloc(n * sizeof(opt));
  if (n) memcpy(v->pts, P, n * sizeof(opt));
  return v;
}

static onode* make_interior(int dim, int32_t split) {
  onode* v = (onode*)calloc(1, sizeof(onode));
  if (!v) abort();
  v->dim = dim;
  v->split = split;
  return v;
}

static void free_subtree(onode* v) {
  if (!v) return;
  free_subtree(v->lc);
  free_subtree(v->rc);
  free(v->pts);
  free(v->dead);
  free(v);
}

/* All points of a subtree, in in-order (the "flatten" of Sec. 4.1). */
static void collect(const onode* v, ovec* out) {
  if (v->leaf) {
    for (uint64_t i = 0; i < v->size; ++i) ovec_push(out, &v->pts[i]);
    return;
  }
  collect(v->lc, out);
  collect(v->rc, out);
}

/* ------------------------------------------------------------------ */
/* Construction: Alg. 1                                                  */
/* ------------------------------------------------------------------ */

/* Skeleton node: the first lambda levels of a kd-tree on the sample S. */
typedef struct skel {
  int bucket;
  int dim;
  int32_t split;
  struct skel* l;
  struct skel* r;
  ovec pts; /* points sieved into this bucket */
} skel;

static skel* skeleton(const orc_params* p, const opt* S, uint64_t m, int j) {
  skel* k = (skel*)calloc(1, sizeof(skel));
  if (!k) abort();
  int dim;
  int32_t x;
  if (j == p->lambda || m < 2 * (uint64_t)p->sigma_os || rule_R(S, m, p->d, &dim, &x) != 0) {
    k->bucket = 1;
    return k;
  }
  k->dim = dim;
  k->split = x;
  opt* SL = (opt*)xmalloc(m * sizeof(opt));
  opt* SR = (opt*)xmalloc(m * sizeof(opt));
  uint64_t nl = 0, nr = 0;
  for (uint64_t i = 0; i < m; ++i) {
    if (S[i].x[dim] < x)
      SL[nl++] = S[i];
    else
      SR[nr++] = S[i];
  }
  k->l = skeleton(p, SL, nl, j + 1);
  k->r = skeleton(p, SR, nr, j + 1);
  free(SL);
  free(SR);
  return k;
}

static void free_skel(skel* k) {
  if (!k) return;
  free_skel(k->l);
  free_skel(k->r);
  free(k->pts.a);
  free(k);
}

static onode* build(const orc_params* p, const opt* P, uint64_t n, uint32_t t);

/* Replace every bucket by the tree built on its points (Alg. 1, the
 * parallel-foreach over external nodes). */
static onode* materialize(const orc_params* p, skel* k, uint32_t t) {
  if (k->bucket) return build(p, k->pts.a, k->pts.n, t);
  onode* v = make_interior(k->dim, k->split);
  v->lc = materialize(p, k->l, t + 1);
  v->rc = materialize(p, k->r, t + 1);
  v->size = v->lc->size + v->rc->size;
  return v;
}

/* Build(P) at tree depth t. */
static onode* build(const orc_params* p, const opt* P, uint64_t n, uint32_t t) {
  if (n == 0) return make_leaf(P, 0);
  if (n <= (uint64_t)p->phi) return make_leaf(P, n);      /* leaf wrap */
  if (all_identical(P, n, p->d)) return make_leaf(P, n);  /* heavy leaf */

  /* Sample. */
  int s = orc_sample_shift(p, n);
  opt* S = (opt*)xmalloc(n * sizeof(opt));
  uint64_t m = 0;
  for (uint64_t i = 0; i < n; ++i)
    if (orc_is_sampled(p->seed, t, P[i].id, s)) S[m++] = P[i];

  /* Skeleton on the sample. */
  skel* K = skeleton(p, S, m, 0);
  free(S);

  if (K->bucket) {
    /* Too few samples for a skeleton: one level of the plain construction. */
    free_skel(K);
    int dim;
    int32_t x;
    rule_R(P, n, p->d, &dim, &x); /* succeeds: P is not all identical */
    opt* PL = (opt*)xmalloc(n * sizeof(opt));
    opt* PR = (opt*)xmalloc(n * sizeof(opt));
    uint64_t nl = 0, nr = 0;
    for (uint64_t i = 0; i < n; ++i) {
      if (P[i].x[dim] < x)
        PL[nl++] = P[i];
      else
        PR[nr++] = P[i];
    }
    onode* v = make_interior(dim, x);
    v->lc = build(p, PL, nl, t + 1);
    v->rc = build(p, PR, nr, t + 1);
    v->size = n;
    free(PL);
    free(PR);
    return v;
  }

  /* Sieve: every point walks the skeleton to its bucket. */
  for (uint64_t i = 0; i < n; ++i) {
    skel* k = K;
    while (!k->bucket) k = (P[i].x[k->dim] < k->split) ? k->l : k->r;
    ovec_push(&k->pts, &P[i]);
  }
  onode* v = materialize(p, K, t);
  free_skel(K);
  return v;
}

static int check_params(const orc_params* p) {
  if (!p) return ORC_EINVAL;
  if (p->d < 1 || p->d > ORC_DMAX) return ORC_EINVAL;
  if (p->phi < 1) return ORC_EINVAL;
  if (p->lambda < 1 || p->lambda > 10) return ORC_EINVAL;
  if (p->sigma_log2 < 0 || p->sigma_log2 > 30) return ORC_EINVAL;
  if (p->sigma_os < 1 || p->sigma_os > (1 << 16)) return ORC_EINVAL;
  if (p->count_mode != 0 && p->count_mode != 1) return ORC_EINVAL;
  if (p->alpha_den < 1 || p->alpha_den > (1 << 20)) return ORC_EINVAL;
  if (p->alpha_num < 0 || 2 * p->alpha_num > p->alpha_den) return ORC_EINVAL;
  return ORC_OK;
}

static opt* load_points(const int32_t* coords, const uint32_t* ids, uint64_t n, int d,
                        uint32_t id_base, int* err) {
  opt* P = (opt*)xmalloc(n * sizeof(opt));
  for (uint64_t i = 0; i < n; ++i) {
    P[i].id = ids ? ids[i] : (uint32_t)(id_base + i);
    memset(P[i].x, 0, sizeof(P[i].x));
    for (int j = 0; j < d; ++j) {
      int32_t c = coords[i * d + j];
      if (c < 0 || (int64_t)c >= ORC_COORD_LIMIT) {
        free(P);
        *err = ORC_EINVAL;
        return NULL;
      }
      P[i].x[j] = c;
    }
  }
  *err = ORC_OK;
  return P;
}

/* Ids name points (reading R9).  Sorting a copy is the plain way to see a
 * repeat: equal ids end up next to each other. */
static int cmp_u32_asc(const void* a, const void* b) {
  uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
  return (x > y) - (x < y);
}

static uint32_t* sorted_ids(const opt* P, uint64_t n) {
  uint32_t* v = (uint32_t*)xmalloc(n * sizeof(uint32_t));
  for (uint64_t i = 0; i < n; ++i) v[i] = P[i].id;
  qsort(v, n, sizeof(uint32_t), cmp_u32_asc);
  return v;
}

/* 1 when some id repeats or is 0xFFFFFFFF. */
static int ids_bad(const opt* P, uint64_t n) {
  if (n == 0) return 0;
  uint32_t* v = sorted_ids(P, n);
  int bad = v[n - 1] == 0xFFFFFFFFu;
  for (uint64_t i = 1; i < n && !bad; ++i) bad = v[i] == v[i - 1];
  free(v);
  return bad;
}

/* 1 when x is in the ascending array v[0..n). */
static int id_in(const uint32_t* v, uint64_t n, uint32_t x) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (v[mid] < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo < n && v[lo] == x;
}

orc_tree* orc_build(const int32_t* coords, const uint32_t* ids, uint64_t n, const orc_params* p,
                    int* err) {
  return orc_build_at_depth(coords, ids, n, p, 0, err);
}

orc_tree* orc_build_at_depth(const int32_t* coords, const uint32_t* ids, uint64_t n,
                             const orc_params* p, uint32_t depth, int* err) {
  int e = check_params(p);
  if (e == ORC_OK && n >= 0xFFFFFFFFull) e = ORC_EINVAL;
  if (e != ORC_OK) {
    if (err) *err = e;
    return NULL;
  }
  opt* P = load_points(coords, ids, n, p->d, 0, &e);
  if (e == ORC_OK && ids_bad(P, n)) {
    free(P);
    e = ORC_EINVAL;
  }
  if (e != ORC_OK) {
    if (err) *err = e;
    return NULL;
  }
  orc_tree* t = (orc_tree*)calloc(1, sizeof(orc_tree));
  if (!t) abort();
  t->p = *p;
  t->root = build(p, P, n, depth);
  free(P);
  if (err) *err = ORC_OK;
  return t;
}

void orc_free(orc_tree* t) {
  if (!t) return;
  free_subtree(t->root);
  free(t);
}

uint64_t orc_size(const orc_tree* t) { return t->root->size; }

static int height_of(const onode* v) {
  if (v->leaf) return 0;
  int a = height_of(v->lc), b = height_of(v->rc);
  return 1 + (a > b ? a : b);
}

int orc_height(const orc_tree* t) { return height_of(t->root); }

/* ------------------------------------------------------------------ */
/* Batch insertion: Alg. 2                                               */
/* ------------------------------------------------------------------ */

/* Mirror of the skeleton at a tree node: its first lambda levels, cut at
 * leaves (Alg. 2, "the skeleton at T"). */
typedef struct sknode {
  onode* tn;
  int ext;
  struct sknode* l;
  struct sknode* r;
  ovec pts;     /* batch points sieved to this external node */
  uint64_t cnt; /* batch points below this skeleton node */
} sknode;

static sknode* fetch_skeleton(onode* u, int j, int lambda) {
  sknode* s = (sknode*)calloc(1, sizeof(sknode));
  if (!s) abort();
  s->tn = u;
  if (j == lambda || u->leaf) {
    s->ext = 1;
    return s;
  }
  s->l = fetch_skeleton(u->lc, j + 1, lambda);
  s->r = fetch_skeleton(u->rc, j + 1, lambda);
  return s;
}

static uint64_t skel_counts(sknode* s) {
  s->cnt = s->ext ? s->pts.n : skel_counts(s->l) + skel_counts(s->r);
  return s->cnt;
}

static void skel_gather(const sknode* s, ovec* out) {
  if (s->ext) {
    for (uint64_t i = 0; i < s->pts.n; ++i) ovec_push(out, &s->pts.a[i]);
    return;
  }
  skel_gather(s->l, out);
  skel_gather(s->r, out);
}

static void free_sk(sknode* s) {
  if (!s) return;
  free_sk(s->l);
  free_sk(s->r);
  free(s->pts.a);
  free(s);
}

static onode* batch_insert(const orc_params* p, onode* T, const opt* P, uint64_t m, uint32_t t);

static onode* insert_to_skeleton(const orc_params* p, sknode* s, uint32_t t) {
  if (s->ext) return batch_insert(p, s->tn, s->pts.a, s->pts.n, t);
  onode* u = s->tn;
  if (s->cnt == 0) return u; /* reading R5: nothing inserted below u */
  uint64_t N = u->size + s->cnt;
  uint64_t L = u->lc->size + s->l->cnt;
  if (orc_balanced(L, N, p->alpha_num, p->alpha_den)) {
    u->lc = insert_to_skeleton(p, s->l, t + 1);
    u->rc = insert_to_skeleton(p, s->r, t + 1);
    u->size = N;
    return u;
  }
  /* Unbalanced after insertion: rebuild t with its new points. */
  ovec all = {0};
  collect(u, &all);
  skel_gather(s, &all);
  onode* v = build(p, all.a, all.n, t);
  free(all.a);
  free_subtree(u);
  return v;
}

static onode* batch_insert(const orc_params* p, onode* T, const opt* P, uint64_t m, uint32_t t) {
  if (m == 0) return T;
  if (T->leaf) {
    ovec all = {0};
    collect(T, &all);
    for (uint64_t i = 0; i < m; ++i) ovec_push(&all, &P[i]);
    onode* v = build(p, all.a, all.n, t);
    free(all.a);
    free_subtree(T);
    return v;
  }
  sknode* K = fetch_skeleton(T, 0, p->lambda);
  for (uint64_t i = 0; i < m; ++i) { /* Sieve(P, skeleton) */
    sknode* s = K;
    while (!s->ext) s = (P[i].x[s->tn->dim] < s->tn->split) ? s->l : s->r;
    ovec_push(&s->pts, &P[i]);
  }
  skel_counts(K);
  onode* v = insert_to_skeleton(p, K, t);
  free_sk(K);
  return v;
}

int orc_insert(orc_tree* t, const int32_t* coords, const uint32_t* ids, uint64_t m) {
  if (!t || (m && (!coords || !ids))) return ORC_EINVAL;
  if (t->root->size + m >= 0xFFFFFFFFull) return ORC_EINVAL;
  int e;
  opt* P = load_points(coords, ids, m, t->p.d, 0, &e);
  if (e != ORC_OK) return e;
  /* reading R9: the batch is rejected whole, before any change */
  int bad = ids_bad(P, m);
  if (!bad && m) {
    ovec all = {0};
    collect(t->root, &all);
    uint32_t* live = sorted_ids(all.a, all.n);
    for (uint64_t i = 0; i < m && !bad; ++i) bad = id_in(live, all.n, P[i].id);
    free(live);
    free(all.a);
  }
  if (bad) {
    free(P);
    return ORC_EINVAL;
  }
  t->root = batch_insert(&t->p, t->root, P, m, 0);
  free(P);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Batch deletion: Sec. 4.2 (two rounds)                                 */
/* ------------------------------------------------------------------ */

static int same_point(const opt* a, const opt* b, int d) {
  if (a->id != b->id) return 0;
  for (int j = 0; j < d; ++j)
    if (a->x[j] != b->x[j]) return 0;
  return 1;
}

/* Round 1: sieve one batch point down to its leaf and mark every stored
 * copy of it; points not in the tree find nothing and are discarded. */
static void mark_point(onode* v, const opt* q, int d) {
  while (!v->leaf) v = (q->x[v->dim] < v->split) ? v->lc : v->rc;
  if (!v->dead && v->size) {
    v->dead = (unsigned char*)calloc(v->size, 1);
    if (!v->dead) abort();
  }
  for (uint64_t i = 0; i < v->size; ++i)
    if (same_point(&v->pts[i], q, d)) v->dead[i] = 1;
}

/* Exact number of deleted records in every subtree. */
static uint64_t count_dead(onode* v) {
  if (v->leaf) {
    v->ndead = 0;
    if (v->dead)
      for (uint64_t i = 0; i < v->size; ++i) v->ndead += v->dead[i];
    return v->ndead;
  }
  v->ndead = count_dead(v->lc) + count_dead(v->rc);
  return v->ndead;
}

static void collect_live(const onode* v, ovec* out) {
  if (v->leaf) {
    for (uint64_t i = 0; i < v->size; ++i)
      if (!v->dead || !v->dead[i]) ovec_push(out, &v->pts[i]);
    return;
  }
  collect_live(v->lc, out);
  collect_live(v->rc, out);
}

/* Round 2: top-down with the post-deletion sizes. */
static onode* delete_rec(const orc_params* p, onode* u, uint32_t t) {
  if (u->ndead == 0) return u; /* reading R5 */
  uint64_t N = u->size - u->ndead;
  if (N == 0) {
    free_subtree(u);
    return make_leaf(NULL, 0);
  }
  if (u->leaf) {
    ovec live = {0};
    collect_live(u, &live);
    onode* v = build(p, live.a, live.n, t); /* <= phi or identical: a leaf */
    free(live.a);
    free_subtree(u);
    return v;
  }
  uint64_t L = u->lc->size - u->lc->ndead;
  if (orc_balanced(L, N, p->alpha_num, p->alpha_den)) {
    u->lc = delete_rec(p, u->lc, t + 1);
    u->rc = delete_rec(p, u->rc, t + 1);
    u->size = N;
    u->ndead = 0;
    return u;
  }
  ovec live = {0};
  collect_live(u, &live);
  onode* v = build(p, live.a, live.n, t);
  free(live.a);
  free_subtree(u);
  return v;
}

static int cmp_opt_id(const void* a, const void* b) {
  uint32_t x = ((const opt*)a)->id, y = ((const opt*)b)->id;
  return (x > y) - (x < y);
}

int orc_delete(orc_tree* t, const uint32_t* ids, uint64_t m, uint64_t* n_deleted) {
  if (!t || (m && !ids)) return ORC_EINVAL;
  int d = t->p.d;
  /* reading R6: the stored points sorted by id give each id's coordinates */
  ovec all = {0};
  collect(t->root, &all);
  if (all.n) qsort(all.a, all.n, sizeof(opt), cmp_opt_id);
  /* distinct batch ids */
  uint32_t* q = (uint32_t*)xmalloc((m ? m : 1) * sizeof(uint32_t));
  if (m) memcpy(q, ids, m * sizeof(uint32_t));
  qsort(q, m, sizeof(uint32_t), cmp_u32_asc);
  for (uint64_t i = 0; i < m; ++i) {
    if (i > 0 && q[i] == q[i - 1]) continue; /* a repeat */
    uint64_t lo = 0, hi = all.n;
    while (lo < hi) {
      uint64_t mid = lo + (hi - lo) / 2;
      if (all.a[mid].id < q[i])
        lo = mid + 1;
      else
        hi = mid;
    }
    if (lo < all.n && all.a[lo].id == q[i]) mark_point(t->root, &all.a[lo], d); /* round 1 */
  }
  free(q);
  free(all.a);
  uint64_t k = count_dead(t->root);
  if (n_deleted) *n_deleted = k;
  t->root = delete_rec(&t->p, t->root, 0); /* round 2 */
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Export                                                               */
/* ------------------------------------------------------------------ */

static int cmp_u32(const void* a, const void* b) {
  uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
  return (x > y) - (x < y);
}

typedef struct {
  uint8_t* dims;
  int32_t* splits;
  uint64_t* sizes;
  uint32_t* leaf_ids;
  uint64_t* leaf_offsets;
  uint64_t nn, nl, nid;
} exporter;

static void export_rec(const onode* v, exporter* e) {
  uint64_t i = e->nn++;
  if (v->leaf) {
    if (e->dims) e->dims[i] = 0xFF;
    if (e->splits) e->splits[i] = 0;
    if (e->sizes) e->sizes[i] = v->size;
    if (e->leaf_offsets) e->leaf_offsets[e->nl] = e->nid;
    if (e->leaf_ids) {
      for (uint64_t k = 0; k < v->size; ++k) e->leaf_ids[e->nid + k] = v->pts[k].id;
      qsort(e->leaf_ids + e->nid, v->size, sizeof(uint32_t), cmp_u32);
    }
    e->nid += v->size;
    e->nl++;
    return;
  }
  if (e->dims) e->dims[i] = (uint8_t)v->dim;
  if (e->splits) e->splits[i] = v->split;
  if (e->sizes) e->sizes[i] = v->size;
  export_rec(v->lc, e);
  export_rec(v->rc, e);
}

int orc_export(const orc_tree* t, uint8_t* dims, int32_t* splits, uint64_t* sizes,
               uint64_t* n_nodes, uint32_t* leaf_ids, uint64_t* leaf_offsets,
               uint64_t* n_leaves) {
  exporter e = {dims, splits, sizes, leaf_ids, leaf_offsets, 0, 0, 0};
  export_rec(t->root, &e);
  if (leaf_offsets) leaf_offsets[e.nl] = e.nid;
  if (n_nodes) *n_nodes = e.nn;
  if (n_leaves) *n_leaves = e.nl;
  return ORC_OK;
}

static void points_rec(const onode* v, int d, uint32_t* ids, int32_t* coords, uint64_t* k) {
  if (v->leaf) {
    for (uint64_t i = 0; i < v->size; ++i, ++*k) {
      if (ids) ids[*k] = v->pts[i].id;
      if (coords)
        for (int j = 0; j < d; ++j) coords[*k * d + j] = v->pts[i].x[j];
    }
    return;
  }
  points_rec(v->lc, d, ids, coords, k);
  points_rec(v->rc, d, ids, coords, k);
}

int orc_points(const orc_tree* t, uint32_t* ids, int32_t* coords) {
  uint64_t k = 0;
  points_rec(t->root, t->p.d, ids, coords, &k);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Queries: Sec. 5                                                       */
/* ------------------------------------------------------------------ */

static int64_t sqdist(const int32_t* a, const int32_t* b, int d) {
  int64_t s = 0;
  for (int j = 0; j < d; ++j) {
    int64_t t = (int64_t)a[j] - b[j];
    s += t * t;
  }
  return s;
}

/* Keep the k smallest (d2, id) pairs, sorted ascending. */
static void topk_offer(int64_t* bd, uint32_t* bi, int k, int64_t d2, uint32_t id) {
  if (d2 > bd[k - 1] || (d2 == bd[k - 1] && id >= bi[k - 1])) return;
  int i = k - 1;
  while (i > 0 && (bd[i - 1] > d2 || (bd[i - 1] == d2 && bi[i - 1] > id))) {
    bd[i] = bd[i - 1];
    bi[i] = bi[i - 1];
    --i;
  }
  bd[i] = d2;
  bi[i] = id;
}

static void knn_brute_rec(const onode* v, const int32_t* q, int d, int64_t* bd, uint32_t* bi,
                          int k) {
  if (v->leaf) {
    for (uint64_t i = 0; i < v->size; ++i)
      topk_offer(bd, bi, k, sqdist(v->pts[i].x, q, d), v->pts[i].id);
    return;
  }
  knn_brute_rec(v->lc, q, d, bd, bi, k);
  knn_brute_rec(v->rc, q, d, bd, bi, k);
}

void orc_knn_brute(const orc_tree* t, const int32_t* q, uint64_t nq, int k, uint32_t* out_ids,
                   int64_t* out_d2) {
  int d = t->p.d;
  for (uint64_t i = 0; i < nq; ++i) {
    int64_t* bd = out_d2 + i * k;
    uint32_t* bi = out_ids + i * k;
    for (int j = 0; j < k; ++j) {
      bd[j] = INT64_MAX;
      bi[j] = 0xFFFFFFFFu;
    }
    knn_brute_rec(t->root, q + i * d, d, bd, bi, k);
  }
}

/* Squared distance from q to the box lo <= x <= hi (the node's subspace,
 * computed on the fly from the splitters, Sec. 5). */
static int64_t box_dist(const int32_t* q, const int64_t* lo, const int64_t* hi, int d) {
  int64_t s = 0;
  for (int j = 0; j < d; ++j) {
    int64_t t = 0;
    if (q[j] < lo[j]) t = lo[j] - q[j];
    if (q[j] > hi[j]) t = q[j] - hi[j];
    s += t * t;
  }
  return s;
}

static void knn_dfs(const onode* v, const int32_t* q, int d, int64_t* lo, int64_t* hi,
                    int64_t* bd, uint32_t* bi, int k) {
  /* Prune only when strictly farther than the k-th candidate: an equally
   * distant point may still win on its id. */
  if (box_dist(q, lo, hi, d) > bd[k - 1]) return;
  if (v->leaf) {
    for (uint64_t i = 0; i < v->size; ++i)
      topk_offer(bd, bi, k, sqdist(v->pts[i].x, q, d), v->pts[i].id);
    return;
  }
  int j = v->dim;
  int64_t x = v->split;
  int64_t save_lo = lo[j], save_hi = hi[j];
  int near_left = q[j] < x;
  for (int pass = 0; pass < 2; ++pass) {
    int go_left = (pass == 0) ? near_left : !near_left;
    if (go_left) {
      hi[j] = x - 1 < save_hi ? x - 1 : save_hi;
      knn_dfs(v->lc, q, d, lo, hi, bd, bi, k);
      hi[j] = save_hi;
    } else {
      lo[j] = x > save_lo ? x : save_lo;
      knn_dfs(v->rc, q, d, lo, hi, bd, bi, k);
      lo[j] = save_lo;
    }
  }
}

void orc_knn_tree(const orc_tree* t, const int32_t* q, uint64_t nq, int k, uint32_t* out_ids,
                  int64_t* out_d2) {
  int d = t->p.d;
  for (uint64_t i = 0; i < nq; ++i) {
    int64_t* bd = out_d2 + i * k;
    uint32_t* bi = out_ids + i * k;
    for (int j = 0; j < k; ++j) {
      bd[j] = INT64_MAX;
      bi[j] = 0xFFFFFFFFu;
    }
    int64_t lo[ORC_DMAX], hi[ORC_DMAX];
    for (int j = 0; j < d; ++j) {
      lo[j] = 0;
      hi[j] = ORC_COORD_LIMIT - 1;
    }
    knn_dfs(t->root, q + i * d, d, lo, hi, bd, bi, k);
  }
}

static int inside(const int32_t* x, const int32_t* lo, const int32_t* hi, int d) {
  for (int j = 0; j < d; ++j)
    if (x[j] < lo[j] || x[j] > hi[j]) return 0;
  return 1;
}

static uint64_t rc_brute(const onode* v, const int32_t* lo, const int32_t* hi, int d) {
  if (v->leaf) {
    uint64_t c = 0;
    for (uint64_t i = 0; i < v->size; ++i) c += inside(v->pts[i].x, lo, hi, d);
    return c;
  }
  return rc_brute(v->lc, lo, hi, d) + rc_brute(v->rc, lo, hi, d);
}

void orc_range_count_brute(const orc_tree* t, const int32_t* lo, const int32_t* hi, uint64_t nq,
                           uint64_t* out) {
  int d = t->p.d;
  for (uint64_t i = 0; i < nq; ++i) out[i] = rc_brute(t->root, lo + i * d, hi + i * d, d);
}

static uint64_t rc_dfs(const onode* v, const int32_t* qlo, const int32_t* qhi, int d, int64_t* lo,
                       int64_t* hi) {
  int contained = 1;
  for (int j = 0; j < d; ++j) {
    if (hi[j] < qlo[j] || lo[j] > qhi[j]) return 0; /* disjoint */
    if (lo[j] < qlo[j] || hi[j] > qhi[j]) contained = 0;
  }
  if (contained) return v->size; /* whole subspace inside: its stored size */
  if (v->leaf) {
    uint64_t c = 0;
    for (uint64_t i = 0; i < v->size; ++i) c += inside(v->pts[i].x, qlo, qhi, d);
    return c;
  }
  int j = v->dim;
  int64_t x = v->split, save_lo = lo[j], save_hi = hi[j];
  uint64_t c = 0;
  hi[j] = x - 1 < save_hi ? x - 1 : save_hi;
  if (hi[j] >= lo[j]) c += rc_dfs(v->lc, qlo, qhi, d, lo, hi);
  hi[j] = save_hi;
  lo[j] = x > save_lo ? x : save_lo;
  if (hi[j] >= lo[j]) c += rc_dfs(v->rc, qlo, qhi, d, lo, hi);
  lo[j] = save_lo;
  return c;
}

void orc_range_count_tree(const orc_tree* t, const int32_t* lo, const int32_t* hi, uint64_t nq,
                          uint64_t* out) {
  int d = t->p.d;
  for (uint64_t i = 0; i < nq; ++i) {
    int64_t blo[ORC_DMAX], bhi[ORC_DMAX];
    for (int j = 0; j < d; ++j) {
      blo[j] = 0;
      bhi[j] = ORC_COORD_LIMIT - 1;
    }
    out[i] = rc_dfs(t->root, lo + i * d, hi + i * d, d, blo, bhi);
  }
}
