// Persistent sieve kernels (count and scatter of Alg. 1's sieve) that stream
// their tiles through shared memory with bulk asynchronous copies.
//
// Each CTA owns a contiguous run of tiles and is split into one producer
// warp and STM_CONSUMERS consumer threads.  The producer keeps STM_STAGES
// tiles in flight: for every array of a tile (the d coordinate arrays and
// the ids, or one point-major array) it issues one cp.async.bulk of the
// 16-byte aligned body into a stage buffer, completing on the stage's "full"
// mbarrier, and loads the at most three elements before and after the body
// itself; the consumers walk the tile from shared memory only and release
// the stage on its "empty" mbarrier.  Every wait is bounded: on expiry the
// kernel records DERR_TIMEOUT and its threads leave together.
//
// The skeleton of the tile's segment is expanded into a complete heap of
// lambda levels (a node below a bucket always goes left) plus a table from
// the 2^lambda level-lambda positions to bucket numbers, so a walk is lambda
// branch-free steps.  The count walks every point once and, with at most
// 256 buckets, records its bucket in one byte; the scatter's producer then
// copies those bytes with the tile, so the scatter does not walk again.
#pragma once

#include "sieve.cuh"

namespace pkd {

constexpr long long STM_WAIT_CYCLES = 4000000000ll;  // about 2 s at 2 GHz: the default limit, and the
                                                     // fixed limit of the drain before a CTA exits

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// Bulk copy of `bytes` (a multiple of 16) from global `src` (16-byte
// aligned) to shared `dst` (16-byte aligned), completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of `bar`; false when `limit` clock cycles
// went by first (limit 0: one non-blocking test).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  if (mbar_test_wait(bar, parity)) return true;
  if (limit <= 0) return false;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

// One array of a tile: m 4-byte elements from global P.  Elements [h, h+L)
// arrive by bulk copy into buf[sh + h, sh + h + L) (sh + h is a multiple of
// 4, so the shared address is 16-byte aligned); the producer loads the rest.
struct StmArr {
  const uint32_t* P;
  int m, h, L, sh;
};

__device__ __forceinline__ StmArr stm_arr(const void* P, int m) {
  StmArr a;
  a.P = (const uint32_t*)P;
  a.m = m;
  const int mis = (int)(((uintptr_t)P >> 2) & 3);
  a.h = min(m, (4 - mis) & 3);
  a.L = ((m - a.h) >> 2) << 2;
  a.sh = (4 - a.h) & 3;
  return a;
}

// The tile geometry of the sieve: tile `tile` of segment s.
struct StmTile {
  uint32_t s;   // big segment
  uint32_t t0;  // first tile of the segment
  uint32_t tl;  // tile index within the segment
  uint32_t nt;  // tiles of the segment
  uint64_t g0;  // first point (absolute arena position)
  int cnt;      // points
};

__device__ __forceinline__ StmTile stm_tile(const RoundArgs& r, uint32_t s, uint32_t tile) {
  StmTile t;
  const Seg seg = r.big[s];
  t.s = s;
  t.t0 = r.tile0[s];
  t.tl = tile - t.t0;
  t.nt = (seg.len + r.TILE - 1) / r.TILE;
  t.g0 = seg.start + (uint64_t)t.tl * r.TILE;
  const uint64_t first = (uint64_t)t.tl * r.TILE;
  t.cnt = first >= seg.len ? 0 : (int)min((uint64_t)r.TILE, (uint64_t)seg.len - first);
  return t;
}

// Per-stage record, written by the producer before it arrives on "full".
template <int D>
struct StmStage {
  StmTile t;
  int sh[D + 1];     // element i of array a is at buf[a * stride + sh[a] + i]
  int ids_implicit;  // point-major input without ids: id = position
};

constexpr int STM_STAGES = 2;
constexpr int STM_CONSUMERS = 512;                // consumer threads (16 warps)
constexpr int STM_THREADS = STM_CONSUMERS + 32;   // plus one producer warp
constexpr int STM_PER = 4;                        // points per consumer: TILE <= 2048
constexpr int STM_BAR_CONSUMERS = 1;              // named barrier of the consumers

__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync %0, %1;" ::"r"(STM_BAR_CONSUMERS), "r"(STM_CONSUMERS) : "memory");
}

__device__ __forceinline__ size_t stm_stride(int tile) { return (size_t)((tile + 4 + 3) & ~3); }

// Words of one stage buffer: D coordinate arrays (or one point-major array
// of D * tile words, which fits in the same space) and optionally the ids.
template <int D>
__host__ __device__ inline size_t stm_stage_words(int tile, bool ids) {
  return (size_t)(D + (ids ? 1 : 0)) * (size_t)((tile + 4 + 3) & ~3);
}

// Producer warp: fill stage `buf` with tile `tile` of segment s and arrive on
// `full` with the bytes the bulk copies will deliver.
template <int D>
__device__ void stm_produce(const RoundArgs& r, const Src& src, uint32_t s, uint32_t tile, bool ids, uint32_t* buf,
                            StmStage<D>* rec, uint64_t* full, uint32_t* gbs, uint8_t* sbk) {
  const int lane = lane_id();
  const StmTile t = stm_tile(r, s, tile);
  if (gbs) {
    const uint64_t hb = (uint64_t)t.t0 * r.NB;
    const uint32_t g0 = r.hscan[hb];
    for (int b = lane; b < r.NB; b += 32) gbs[b] = r.hscan[hb + (uint64_t)b * t.nt + t.tl] - g0;
  }
  const size_t stride = stm_stride(r.TILE);
  StmArr arr[D + 1];
  int implicit = 0;
  if (!src.is_aos) {
#pragma unroll
    for (int j = 0; j < D; ++j) arr[j] = stm_arr(src.soa.c + (uint64_t)j * src.soa.stride + t.g0, t.cnt);
    arr[D] = stm_arr(src.soa.id + t.g0, ids ? t.cnt : 0);
  } else {
    arr[0] = stm_arr(src.aos + t.g0 * D, t.cnt * D);
#pragma unroll
    for (int j = 1; j < D; ++j) arr[j] = stm_arr(nullptr, 0);
    arr[D] = stm_arr(nullptr, 0);
    if (ids) {
      if (src.aos_ids) arr[D] = stm_arr(src.aos_ids + t.g0, t.cnt);
      else implicit = 1;
    }
  }
  // the ragged ends: element e < 3 of the head, e >= 3 of the tail
  for (int q = lane; q < (D + 1) * 6; q += 32) {
    const int a = q / 6, e = q % 6;
    const StmArr& A = arr[a];
    const int i = e < 3 ? e : A.h + A.L + (e - 3);
    const bool take = e < 3 ? i < A.h : i < A.m;
    if (take) buf[(size_t)a * stride + A.sh + i] = A.P[i];
  }
  __syncwarp();
  if (lane == 0) {
    uint32_t bytes = 0;
#pragma unroll
    for (int a = 0; a <= D; ++a) bytes += (uint32_t)arr[a].L * 4u;
    // the tile's bucket bytes (tile-aligned rows of TILE bytes, so the copy
    // starts 16-byte aligned; it may read past cnt within the row)
    const uint32_t kb = sbk ? ((uint32_t)t.cnt + 15u) & ~15u : 0u;
    bytes += kb;
    StmStage<D> st;
    st.t = t;
#pragma unroll
    for (int a = 0; a <= D; ++a) st.sh[a] = arr[a].sh;
    st.ids_implicit = implicit;
    *rec = st;
    mbar_arrive_expect_tx(full, bytes);
#pragma unroll
    for (int a = 0; a <= D; ++a)
      if (arr[a].L) bulk_g2s(buf + (size_t)a * stride + arr[a].sh + arr[a].h, arr[a].P + arr[a].h,
                             (uint32_t)arr[a].L * 4u, full);
    if (kb) bulk_g2s(sbk, r.bkt + (uint64_t)tile * r.TILE, kb, full);
  }
}

// Coordinate j / id of point i of a stage.
template <int D>
__device__ __forceinline__ int32_t stm_x(const StmStage<D>& st, const uint32_t* buf, size_t stride, bool aos, int j,
                                         int i) {
  return aos ? (int32_t)buf[st.sh[0] + i * D + j] : (int32_t)buf[(size_t)j * stride + st.sh[j] + i];
}
template <int D>
__device__ __forceinline__ uint32_t stm_id(const StmStage<D>& st, const uint32_t* buf, size_t stride, int i) {
  return st.ids_implicit ? (uint32_t)(st.t.g0 + (uint64_t)i) : buf[(size_t)D * stride + st.sh[D] + i];
}

// The run of tiles of this CTA.
__device__ __forceinline__ void stm_range(uint32_t ntiles, uint32_t& t_begin, uint32_t& t_end) {
  const uint32_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  t_begin = min(ntiles, blockIdx.x * per);
  t_end = min(ntiles, t_begin + per);
}

__device__ __forceinline__ uint32_t stm_advance(const RoundArgs& r, uint32_t s, uint32_t nb, uint32_t tile) {
  while (s + 1 < nb && r.tile0[s + 1] <= tile) ++s;
  return s;
}

// Before the producer warp leaves (at the end of its tiles, or after a wait
// ran out), every bulk copy it issued has landed: it waits, with the fixed
// limit STM_WAIT_CYCLES, for the last phase of each stage's "full" barrier.
// The CTA, and so its shared memory, lives as long as this warp does, so no
// copy can land in shared memory that another CTA has been given.
__device__ __forceinline__ void stm_drain(uint64_t* full, uint32_t issued, DevStatus* st) {
  if (lane_id() != 0) return;
  for (uint32_t k = issued > (uint32_t)STM_STAGES ? issued - STM_STAGES : 0; k < issued; ++k)
    if (!mbar_wait(&full[k % STM_STAGES], (k / STM_STAGES) & 1, STM_WAIT_CYCLES)) set_error(st, DERR_TIMEOUT, 704);
}

// Producer warp main loop over the CTA's tiles.
template <int D>
__device__ void stm_producer(const RoundArgs& r, const Src& src, uint32_t tb, uint32_t te, bool ids, uint32_t* bufs, size_t swords,
                             StmStage<D>* recs, uint64_t* full, uint64_t* empty, uint32_t* gbs,
                             uint8_t* sbk) {
  const uint32_t nb = *r.nbig;
  uint32_t s = seg_of_tile(r.tile0, nb, tb);
  uint32_t k = 0;
  for (; tb + k < te; ++k) {
    const int stg = (int)(k % STM_STAGES);
    if (k >= (uint32_t)STM_STAGES) {
      bool ok = true;
      if (lane_id() == 0) ok = mbar_wait(&empty[stg], ((k / STM_STAGES) - 1) & 1, r.wait_cycles);
      if (!__shfl_sync(FULL_MASK, (int)ok, 0)) {
        if (lane_id() == 0) set_error(r.st, DERR_TIMEOUT, 702);
        break;
      }
      fence_proxy_async_smem();
    }
    s = stm_advance(r, s, nb, tb + k);
    stm_produce<D>(r, src, s, tb + k, ids, bufs + stg * swords, &recs[stg], &full[stg], gbs ? gbs + stg * r.NB : nullptr,
                   sbk ? sbk + (size_t)stg * r.TILE : nullptr);
  }
  stm_drain(full, k, r.st);
}

// Consumers: wait for stage `stg` of tile k (thread 0 waits, the others
// follow through the consumer barrier); false on time-out, for all of them.
__device__ __forceinline__ bool stm_consume_wait(uint64_t* full, int stg, uint32_t k, int* flag, DevStatus* st,
                                                 long long limit) {
  if (threadIdx.x == 0) {
    const bool ok = mbar_wait(&full[stg], (k / STM_STAGES) & 1, limit);
    *flag = ok ? 1 : 0;
    if (!ok) set_error(st, DERR_TIMEOUT, 703);
  }
  consumers_sync();
  return *(volatile int*)flag != 0;
}

// Expand the skeleton of big segment s into the walk tables: wt[h] =
// (split, dim) for h in [1, 2^lam) (a node that is not an interior skeleton
// node gets split INT_MAX: its points go left), wb[p] = bucket of level-lam
// position p.  Returns whether the segment is a heavy leaf.
__device__ __forceinline__ bool stm_tables(const RoundArgs& r, uint32_t s, int2* wt, uint16_t* wb, int tid) {
  const int2* gsk = r.skel + (uint64_t)(r.skel_map ? r.skel_map[s] : s) * r.HN;
  const int L = 1 << r.lam;
  for (int v = 1 + tid; v < 2 * L; v += STM_CONSUMERS) {
    const int2 e = gsk[v];
    const int st = sk_state(e.y);
    if (v < L) wt[v] = st == SK_INTERNAL ? make_int2(e.x, sk_dim(e.y)) : make_int2(INT32_MAX, 0);
    if (st == SK_BUCKET || st == SK_HEAVY) {
      const int j = 31 - __clz(v);
      wb[(v << (r.lam - j)) - L] = (uint16_t)sk_bucket(e.y);
    }
  }
  return sk_state(gsk[1].y) == SK_HEAVY;
}

// The walks of a thread's STM_PER points advance level by level together,
// so their shared-memory lookups overlap; bk[u] = bucket, or -1 when point u
// is not in the tile.
template <int D>
__device__ __forceinline__ void stm_walk4(const int2* wt, const uint16_t* wb, const int32_t (&x)[STM_PER][D],
                                          const bool (&in)[STM_PER], int lam, int (&bk)[STM_PER]) {
  int h[STM_PER];
#pragma unroll
  for (int u = 0; u < STM_PER; ++u) h[u] = 1;
  for (int l = 0; l < lam; ++l) {
#pragma unroll
    for (int u = 0; u < STM_PER; ++u) {
      const int2 e = wt[h[u]];
      int xs = x[u][0];
#pragma unroll
      for (int j = 1; j < D; ++j)
        if (e.y == j) xs = x[u][j];
      h[u] = 2 * h[u] + (xs >= e.x);
    }
  }
#pragma unroll
  for (int u = 0; u < STM_PER; ++u) bk[u] = in[u] ? (int)wb[h[u] - (1 << lam)] : -1;
}

// ---------------------------------------------------------------------------
// Count: per tile, the number of points that reach each bucket.
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(STM_THREADS) k_count_stream(RoundArgs r, uint32_t ntiles) {
  extern __shared__ __align__(16) uint8_t sm[];
  const size_t stride = stm_stride(r.TILE);
  const size_t swords = stm_stage_words<D>(r.TILE, false);
  const int L = 1 << r.lam;
  uint32_t* bufs = (uint32_t*)sm;
  uint64_t* full = (uint64_t*)(bufs + STM_STAGES * swords);
  uint64_t* empty = full + STM_STAGES;
  StmStage<D>* recs = (StmStage<D>*)(empty + STM_STAGES);
  int2* wt = (int2*)(recs + STM_STAGES);
  unsigned* lh = (unsigned*)(wt + L);
  uint16_t* wb = (uint16_t*)(lh + r.NB);
  int* flag = (int*)(wb + L + 2);
  const int tid = threadIdx.x;
  const bool aos = (r.dyn ? r.dyn[*r.sel].src.is_aos : r.src.is_aos) != 0;
  uint32_t tb, te;
  stm_range(round_tiles(r, ntiles), tb, te);
  if (tb >= te) return;
  if (tid == 0) {
    for (int k = 0; k < STM_STAGES; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 1);
    }
    fence_mbar_init();
  }
  for (int b = tid; b < r.NB; b += blockDim.x) lh[b] = 0;
  __syncthreads();
  if (tid >= STM_CONSUMERS) {
    stm_producer<D>(r, round_src(r), tb, te, false, bufs, swords, recs, full, empty, nullptr, nullptr);
    return;
  }
  uint32_t cur_seg = 0xFFFFFFFFu;
  bool heavy = false;
  for (uint32_t k = 0; tb + k < te; ++k) {
    const int stg = (int)(k % STM_STAGES);
    if (!stm_consume_wait(full, stg, k, flag, r.st, r.wait_cycles)) return;
    const StmStage<D> st = recs[stg];
    const uint32_t* buf = bufs + stg * swords;
    if (st.t.s != cur_seg) {  // uniform: every consumer reads the same record
      cur_seg = st.t.s;
      heavy = stm_tables(r, cur_seg, wt, wb, tid);
      consumers_sync();
    }
    if (!heavy) {
      int32_t x[STM_PER][D];
      bool in[STM_PER];
      int bk[STM_PER];
#pragma unroll
      for (int u = 0; u < STM_PER; ++u) {
        const int i = u * STM_CONSUMERS + tid;
        in[u] = i < st.t.cnt;
#pragma unroll
        for (int j = 0; j < D; ++j) x[u][j] = in[u] ? stm_x<D>(st, buf, stride, aos, j, i) : 0;
      }
      stm_walk4<D>(wt, wb, x, in, r.lam, bk);
#pragma unroll
      for (int u = 0; u < STM_PER; ++u)
        if (bk[u] >= 0) atomicAdd(&lh[bk[u]], 1u);
      if (r.bkt) {
        uint8_t* row = r.bkt + (uint64_t)(tb + k) * r.TILE;
#pragma unroll
        for (int u = 0; u < STM_PER; ++u)
          if (bk[u] >= 0) row[u * STM_CONSUMERS + tid] = (uint8_t)bk[u];
      }
    }
    consumers_sync();
    // the stage is no longer read: let the producer refill it
    if (tid == 0) mbar_arrive(&empty[stg]);
    // the tile's counts, bucket-major as the device scan expects (the next
    // tile's counting starts after the barrier of its stage wait)
    const uint64_t hb = (uint64_t)st.t.t0 * r.NB;
    for (int b = tid; b < r.NB; b += STM_CONSUMERS) {
      r.hist[hb + (uint64_t)b * st.t.nt + st.t.tl] = heavy ? 0u : lh[b];
      lh[b] = 0;
    }
  }
}

template <int D>
static size_t count_stream_smem(const RoundArgs& r) {
  const int L = 1 << r.lam;
  return STM_STAGES * stm_stage_words<D>(r.TILE, false) * 4 + STM_STAGES * 16 + STM_STAGES * sizeof(StmStage<D>) +
         (size_t)L * 8 + (size_t)r.NB * 4 + (size_t)(L + 2) * 2 + 16 + 16;
}

// ---------------------------------------------------------------------------
// Scatter: per tile, rank the points within their buckets, stage them in
// shared memory bucket by bucket and write every bucket's run contiguously.
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(STM_THREADS) k_scatter_stream(RoundArgs r, uint32_t ntiles) {
  if (pkd_failed_block(r.st)) return;
  extern __shared__ __align__(16) uint8_t sm[];
  const int tilecap = r.TILE;
  const size_t stride = stm_stride(tilecap);
  const size_t swords = stm_stage_words<D>(tilecap, true);
  const int L = 1 << r.lam;
  uint32_t* bufs = (uint32_t*)sm;
  uint64_t* full = (uint64_t*)(bufs + STM_STAGES * swords);
  uint64_t* empty = full + STM_STAGES;
  StmStage<D>* recs = (StmStage<D>*)(empty + STM_STAGES);
  int2* wt = (int2*)(recs + STM_STAGES);
  unsigned* cur = (unsigned*)(wt + L);      // [NB] per-bucket counters
  unsigned* lstart = cur + r.NB;            // [NB]
  uint32_t* gbase = lstart + r.NB;          // [NB]
  int32_t* stx = (int32_t*)(gbase + r.NB);  // [D][TILE]
  uint32_t* sid = (uint32_t*)(stx + (size_t)D * tilecap);
  uint16_t* sb = (uint16_t*)(sid + tilecap);
  uint16_t* wb = sb + tilecap;              // [L]
  int* flag = (int*)(wb + L + 2);
  uint32_t* gbs = (uint32_t*)(flag + 4);    // [STM_STAGES][NB]
  uint8_t* sbk = r.bkt ? (uint8_t*)(((uintptr_t)(gbs + STM_STAGES * r.NB) + 15) & ~(uintptr_t)15)
                       : nullptr;  // [STM_STAGES][TILE], 16-byte aligned for the bulk copies
  const int tid = threadIdx.x;
  const bool aos = (r.dyn ? r.dyn[*r.sel].src.is_aos : r.src.is_aos) != 0;
  uint32_t tb, te;
  stm_range(round_tiles(r, ntiles), tb, te);
  if (tb >= te) return;
  if (tid == 0) {
    for (int k = 0; k < STM_STAGES; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 1);
    }
    fence_mbar_init();
  }
  __shared__ Pts sdst[1];
  if (tid == 0) sdst[0] = round_dst(r);
  for (int b = tid; b < r.NB; b += blockDim.x) cur[b] = 0;
  __syncthreads();
  if (tid >= STM_CONSUMERS) {
    stm_producer<D>(r, round_src(r), tb, te, true, bufs, swords, recs, full, empty, gbs, sbk);
    return;
  }
  uint32_t cur_seg = 0xFFFFFFFFu;
  bool heavy = false;
  for (uint32_t k = 0; tb + k < te; ++k) {
    const int stg = (int)(k % STM_STAGES);
    if (!stm_consume_wait(full, stg, k, flag, r.st, r.wait_cycles)) return;
    const StmStage<D> st = recs[stg];
    const uint32_t* buf = bufs + stg * swords;
    if (st.t.s != cur_seg) {
      cur_seg = st.t.s;
      heavy = stm_tables(r, cur_seg, wt, wb, tid);
      consumers_sync();
    }
    if (heavy) {  // a heavy segment's points are copied elsewhere
      consumers_sync();
      if (tid == 0) mbar_arrive(&empty[stg]);
      continue;
    }
    const uint64_t hb = (uint64_t)st.t.t0 * r.NB;
    const uint64_t seg_start = st.t.g0 - (uint64_t)st.t.tl * r.TILE;
    const int cnt = st.t.cnt;
    // this tile's global bucket bases, up to two per thread (NB <= 1024);
    // the loads are issued here and used after the ranking
    for (int b = tid; b < r.NB; b += STM_CONSUMERS) gbase[b] = gbs[stg * r.NB + b];
    int32_t x[STM_PER][D];
    uint32_t id[STM_PER];
    bool in[STM_PER];
    int bk[STM_PER], rk[STM_PER];
#pragma unroll
    for (int u = 0; u < STM_PER; ++u) {
      const int i = u * STM_CONSUMERS + tid;
      in[u] = i < cnt;
#pragma unroll
      for (int j = 0; j < D; ++j) x[u][j] = in[u] ? stm_x<D>(st, buf, stride, aos, j, i) : 0;
      id[u] = in[u] ? stm_id<D>(st, buf, stride, i) : 0u;
    }
    if (sbk) {  // buckets recorded by the count
      const uint8_t* tb8 = sbk + (size_t)stg * r.TILE;
#pragma unroll
      for (int u = 0; u < STM_PER; ++u) bk[u] = in[u] ? (int)tb8[u * STM_CONSUMERS + tid] : -1;
    } else {
      stm_walk4<D>(wt, wb, x, in, r.lam, bk);
    }
    consumers_sync();
    // the stage is no longer read: let the producer refill it
    if (tid == 0) mbar_arrive(&empty[stg]);
    // rank within the tile's buckets: one shared atomic per point (the order
    // inside a bucket is immaterial: later steps see only sets)
#pragma unroll
    for (int u = 0; u < STM_PER; ++u) rk[u] = bk[u] >= 0 ? (int)atomicAdd(&cur[bk[u]], 1u) : 0;
    consumers_sync();
    // the tile's bucket starts (one warp; it also clears the counters for
    // the next tile, whose ranking comes after two more barriers)
    if (tid < 32) {
      const int per = (r.NB + 31) >> 5, b0 = lane_id() * per;
      unsigned sum = 0;
      for (int k2 = 0; k2 < per; ++k2)
        if (b0 + k2 < r.NB) sum += cur[b0 + k2];
      unsigned run = (unsigned)warp_incl_scan((int)sum) - sum;
      for (int k2 = 0; k2 < per; ++k2)
        if (b0 + k2 < r.NB) {
          const unsigned c = cur[b0 + k2];
          lstart[b0 + k2] = run;
          run += c;
          cur[b0 + k2] = 0;
        }
    }
    consumers_sync();
#pragma unroll
    for (int u = 0; u < STM_PER; ++u) {
      if (bk[u] >= 0) {
        const int pos = (int)lstart[bk[u]] + rk[u];
#pragma unroll
        for (int j = 0; j < D; ++j) stx[j * tilecap + pos] = x[u][j];
        sid[pos] = id[u];
        sb[pos] = (uint16_t)bk[u];
      }
    }
    consumers_sync();
    // every bucket's run leaves the tile as one contiguous range; the next
    // tile overwrites the staging arrays only after three more barriers
    {
      const Pts dst = *sdst;  // re-read after the barriers: not held in registers
      int32_t* oc[D];
#pragma unroll
      for (int j = 0; j < D; ++j) oc[j] = dst.c + (uint64_t)j * dst.stride + seg_start;
      uint32_t* oid = dst.id + seg_start;
#pragma unroll
      for (int u = 0; u < STM_PER; ++u) {
        const int pos = u * STM_CONSUMERS + tid;
        if (pos < cnt) {
          const int b = sb[pos];
          const uint32_t g = gbase[b] + (uint32_t)(pos - (int)lstart[b]);  // within the segment (< 2^31)
#pragma unroll
          for (int j = 0; j < D; ++j) oc[j][g] = stx[j * tilecap + pos];
          oid[g] = sid[pos];
        }
      }
    }
  }
}

template <int D>
static size_t scatter_stream_smem(const RoundArgs& r) {
  const int L = 1 << r.lam;
  return STM_STAGES * stm_stage_words<D>(r.TILE, true) * 4 + STM_STAGES * 16 + STM_STAGES * sizeof(StmStage<D>) +
         (size_t)L * 8 + (size_t)r.NB * 12 + (size_t)D * r.TILE * 4 + (size_t)r.TILE * 4 + (size_t)r.TILE * 2 +
         (size_t)(L + 2) * 2 + 16 + 16 + (size_t)STM_STAGES * r.NB * 4 + (r.bkt ? (size_t)STM_STAGES * r.TILE + 16 : 0);
}

// ---------------------------------------------------------------------------
// Launch: the streaming kernels by default; the one-tile-per-CTA kernels of
// sieve.cuh with the "sieve_kernel" option set to 1, or when the stages of
// a tile do not fit in shared memory (large d).
// ---------------------------------------------------------------------------
static int stream_sm_count() {
  static int v = -1;
  if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) v = 1;
  }
  return v;
}

static size_t stream_smem_limit() {
  static int v = -1;
  if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (v <= 0) v = 48 * 1024;
  }
  return (size_t)v;
}

// Whether the count records every point's bucket for the scatter (one byte
// a point; the streaming kernels only).
static inline bool record_buckets(int NB) { return NB <= 256 && knobs().sieve_kernel == 0; }

// `fam` names the kernel timer family, `pts` the points of the launch.
template <int D>
static void launch_count(const RoundArgs& r, uint32_t tiles, uint64_t pts, const char* fam, cudaStream_t s) {
  const size_t smb = count_stream_smem<D>(r);
  if (knobs().sieve_kernel == 1 || smb > stream_smem_limit() || r.TILE > STM_CONSUMERS * STM_PER) {
    launch_count_tiles<D>(r, tiles, pts, fam, s);
    return;
  }
  static size_t set = 0;
  if (set < smb) {
    cudaFuncSetAttribute(k_count_stream<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    set = smb;
  }
  const uint32_t grid = std::min<uint32_t>(tiles, (uint32_t)stream_sm_count() * 2);
  KTimer kt;
  ktimer_begin(kt, fam, pts, s);
  PKD_LAUNCH(k_count_stream<D><<<grid, STM_THREADS, smb, s>>>(r, tiles));
  ktimer_end(kt);
}

template <int D>
static void launch_scatter(const RoundArgs& r, uint32_t tiles, uint64_t pts, const char* fam, cudaStream_t s) {
  const size_t smb = scatter_stream_smem<D>(r);
  if (knobs().sieve_kernel == 1 || smb > stream_smem_limit() || r.TILE > STM_CONSUMERS * STM_PER) {
    launch_scatter_tiles<D>(r, tiles, pts, fam, s);
    return;
  }
  static size_t set = 0;
  if (set < smb) {
    cudaFuncSetAttribute(k_scatter_stream<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    set = smb;
  }
  const uint32_t grid = std::min<uint32_t>(tiles, (uint32_t)stream_sm_count() * 2);
  KTimer kt;
  ktimer_begin(kt, fam, pts, s);
  PKD_LAUNCH(k_scatter_stream<D><<<grid, STM_THREADS, smb, s>>>(r, tiles));
  ktimer_end(kt);
}

}  // namespace pkd
