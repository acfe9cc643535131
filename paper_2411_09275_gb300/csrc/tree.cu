// C ABI of the Pkd-tree library: tree lifetime, build, export, status,
// tuning knobs and per-kernel timing.  Every step of the work runs in the
// library's CUDA kernels; this file sequences them and owns the memory.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "engine.hpp"
#include "tree_impl.hpp"

namespace pkd {

Knobs& knobs() {
  static Knobs k;
  return k;
}

cudaMemPool_t mem_pool() {
  static cudaMemPool_t pools[64] = {};
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&pools[dev], &props) != cudaSuccess) {
      cudaGetLastError();
      cudaDeviceGetDefaultMemPool(&pools[dev], dev);
    }
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
  }
  return pools[dev];
}

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return PKD_OK;
  if (e == cudaErrorMemoryAllocation) return PKD_ENOMEM;
  return PKD_ECUDA;
}

// ----------------------------------------------------------------------------
// kernel timers
// ----------------------------------------------------------------------------

namespace {
struct TimerStat {
  uint64_t launches = 0;
  double ms = 0;
  uint64_t items = 0;
};
struct Pending {
  std::string name;
  cudaEvent_t a, b;
  uint64_t items;
};
std::mutex g_tmu;
bool g_timing = false;
std::map<std::string, TimerStat> g_stats;
std::vector<Pending> g_pending;

void resolve_pending() {
  for (auto& p : g_pending) {
    float ms = 0;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      auto& s = g_stats[p.name];
      s.launches++;
      s.ms += ms;
      s.items += p.items;
    }
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  g_pending.clear();
}
}  // namespace

bool ktiming_enabled() { return g_timing; }

void trace_mark(cudaStream_t s, const char* what) {
  static const bool on = getenv("PKD_TRACE") && getenv("PKD_TRACE")[0] == '1';
  if (!on) return;
  static auto last = std::chrono::steady_clock::now();
  cudaStreamSynchronize(s);
  auto now = std::chrono::steady_clock::now();
  fprintf(stderr, "[pkd] %-28s %9.3f ms\n", what, std::chrono::duration<double, std::milli>(now - last).count());
  last = now;
}

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void ktimer_begin(KTimer& k, const char* name, uint64_t items, cudaStream_t s) {
  k.on = g_timing && !flow_capturing();
  if (!k.on) return;
  k.name = name;
  k.items = items;
  k.s = s;
  cudaEventCreate(&k.a);
  cudaEventCreate(&k.b);
  cudaEventRecord(k.a, s);
}

void stat_items(const char* name, uint64_t items) {
  if (!g_timing) return;
  std::lock_guard<std::mutex> g(g_tmu);
  auto& st = g_stats[name];
  st.launches++;
  st.items += items;
}

void stat_host_ms(const char* name, double ms, uint64_t items) {
  if (!g_timing) return;
  std::lock_guard<std::mutex> g(g_tmu);
  auto& st = g_stats[name];
  st.launches++;
  st.ms += ms;
  st.items += items;
}

void ktimer_end(KTimer& k) {
  if (!k.on) return;
  cudaEventRecord(k.b, k.s);
  std::lock_guard<std::mutex> g(g_tmu);
  g_pending.push_back(Pending{k.name, k.a, k.b, k.items});
}

// ----------------------------------------------------------------------------
// status
// ----------------------------------------------------------------------------

int check_status(TreeMem& t, cudaStream_t s) {
  PKD_CUDA(cudaMemcpyAsync(t.st_host, t.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  PKD_CUDA(cudaStreamSynchronize(s));
  const int e = t.st_host->err;
  if (e == DERR_NONE) return PKD_OK;
  fprintf(stderr, "pkd: device status %d (detail %d)\n", e, t.st_host->detail);
  if (e == DERR_TIMEOUT) return PKD_ETIMEOUT;
  return PKD_EINTERNAL;
}

// ----------------------------------------------------------------------------
// validation
// ----------------------------------------------------------------------------

int check_params(const pkd_params* p) {
  if (!p) return PKD_EINVAL;
  if (p->d < 1 || p->d > PKD_DMAX) return PKD_EINVAL;
  if (p->phi < 1) return PKD_EINVAL;
  if (p->lambda < 1 || p->lambda > 10) return PKD_EINVAL;
  if (p->sigma_log2 < 0 || p->sigma_log2 > 30) return PKD_EINVAL;
  if (p->sigma_os < 1 || p->sigma_os > (1 << 16)) return PKD_EINVAL;
  if (p->count_mode != 0 && p->count_mode != 1) return PKD_EINVAL;
  if (p->alpha_den < 1 || p->alpha_den > (1 << 20)) return PKD_EINVAL;
  if (p->alpha_num < 0 || 2 * p->alpha_num > p->alpha_den) return PKD_EINVAL;
  return PKD_OK;
}

// Every coordinate in [0, 2^30): a value is out of range exactly when one of
// its two top bits is set.  A scalar head up to the first 16-byte boundary,
// then 16-byte loads, four in flight per thread, then a scalar tail.
static_assert(PKD_COORD_LIMIT == (1 << 30), "range test by the top two bits");
__global__ void k_validate(const int32_t* c, uint64_t cnt, int* bad) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t head = min(cnt, (uint64_t)(((16u - ((uintptr_t)c & 15u)) & 15u) >> 2));
  unsigned b = 0;
  if (tid < head) b |= (unsigned)c[tid];
  const int4* v4 = reinterpret_cast<const int4*>(c + head);
  const uint64_t n4 = (cnt - head) >> 2;
  uint64_t i = tid;
  for (; i + 3 * nth < n4; i += 4 * nth) {
    const int4 a0 = v4[i], a1 = v4[i + nth], a2 = v4[i + 2 * nth], a3 = v4[i + 3 * nth];
    b |= (unsigned)(a0.x | a0.y | a0.z | a0.w | a1.x | a1.y | a1.z | a1.w);
    b |= (unsigned)(a2.x | a2.y | a2.z | a2.w | a3.x | a3.y | a3.z | a3.w);
  }
  for (; i < n4; i += nth) {
    const int4 a = v4[i];
    b |= (unsigned)(a.x | a.y | a.z | a.w);
  }
  const uint64_t t0 = head + 4 * n4;
  if (tid < cnt - t0) b |= (unsigned)c[t0 + tid];
  if (__any_sync(0xffffffffu, (b >> 30) != 0) && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
}

int validate_coords(const int32_t* c, uint64_t cnt, cudaStream_t s, bool* ok) {
  *ok = true;
  if (cnt == 0) return PKD_OK;
  int* d = nullptr;
  PKD_TRY_(dalloc(&d, 1, s));
  int h = 0;
  dev_fill(d, 0, 4, s);
  KTimer kt;
  ktimer_begin(kt, "validate", cnt, s);
  PKD_LAUNCH(k_validate<<<152 * 8, 256, 0, s>>>(c, cnt, d));
  ktimer_end(kt);
  cudaMemcpyAsync(&h, d, 4, cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  dfree(d, s);
  if (e != cudaSuccess) return cuda_err(e);
  *ok = (h == 0);
  return PKD_OK;
}

// ----------------------------------------------------------------------------
// tree memory
// ----------------------------------------------------------------------------

uint64_t shared_region_for(const Params& p, uint64_t n) {
  const uint64_t per = (uint64_t)2 << p.lambda;
  const uint64_t cap = (uint64_t)std::max(base_cap_for(p.d), 64);
  return per * (8 * (n / cap) + 2048);
}

struct CachedBlock {
  void* p;
  size_t bytes;
  int dev;
  cudaEvent_t ev;  // recorded on the stream that freed the block
  size_t zeroed;   // its first `zeroed` bytes are known to be zero
};
static std::mutex g_big_mu;
static std::vector<CachedBlock> g_big_cache;
static std::map<void*, std::pair<size_t, int>> g_big_live;  // block -> (bytes, device)
static size_t g_big_cached = 0;
constexpr size_t BIG_CACHE_MAX = (size_t)128 << 30;

static void big_flush_locked() {
  for (CachedBlock& b : g_big_cache) {
    cudaEventSynchronize(b.ev);
    cudaEventDestroy(b.ev);
    cudaFree(b.p);
  }
  g_big_cache.clear();
  g_big_cached = 0;
}

static std::atomic<unsigned long long> g_allocs{0};
static std::atomic<long long> g_fail_budget{-1};

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  long long b = g_fail_budget.load();
  while (b >= 0) {  // fault injection armed
    if (b == 0) return cudaErrorMemoryAllocation;
    if (g_fail_budget.compare_exchange_weak(b, b - 1)) break;
  }
  g_allocs.fetch_add(1, std::memory_order_relaxed);
  return cudaMallocFromPoolAsync(p, bytes, mem_pool(), s);
}

// A cached block is taken when it fits and wastes at most half of itself.
// Plain requests prefer blocks not known to be zero, so that the zeroed
// ones (a released tree's delete scratch, cleared after every delete) stay
// for big_alloc_zeroed, which prefers them and reports whether it got one.
static cudaError_t big_alloc_impl(void** p, size_t bytes, cudaStream_t s, bool want_zero, bool* zero) {
  *p = nullptr;
  if (zero) *zero = false;
  if (bytes < BIG_BLOCK_MIN) return pool_alloc(p, bytes, s);
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(g_big_mu);
  int best = -1;
  auto rank = [&](const CachedBlock& b) {  // lower is better
    const bool z = b.zeroed >= bytes;
    return (want_zero ? (z ? 0 : 1) : (b.zeroed == 0 ? 0 : 1));
  };
  for (size_t k = 0; k < g_big_cache.size(); ++k) {
    const CachedBlock& b = g_big_cache[k];
    if (b.dev != dev || b.bytes < bytes || b.bytes > 2 * bytes) continue;
    if (best < 0 || rank(b) < rank(g_big_cache[best]) ||
        (rank(b) == rank(g_big_cache[best]) && b.bytes < g_big_cache[best].bytes))
      best = (int)k;
  }
  if (best >= 0) {
    CachedBlock b = g_big_cache[best];
    g_big_cache.erase(g_big_cache.begin() + best);
    g_big_cached -= b.bytes;
    cudaStreamWaitEvent(s, b.ev, 0);
    cudaEventDestroy(b.ev);
    g_big_live[b.p] = {b.bytes, dev};
    *p = b.p;
    if (zero) *zero = b.zeroed >= bytes;
    return cudaSuccess;
  }
  cudaError_t e = pool_alloc(p, bytes, s);
  if (e == cudaErrorMemoryAllocation && !g_big_cache.empty() && g_fail_budget.load() < 0) {
    cudaGetLastError();
    big_flush_locked();
    e = pool_alloc(p, bytes, s);
  }
  if (e == cudaSuccess) g_big_live[*p] = {bytes, dev};
  return e;
}

cudaError_t big_alloc(void** p, size_t bytes, cudaStream_t s) { return big_alloc_impl(p, bytes, s, false, nullptr); }

cudaError_t big_alloc_zeroed(void** p, size_t bytes, cudaStream_t s, bool* zero) {
  return big_alloc_impl(p, bytes, s, true, zero);
}

void big_free_zeroed(void* p, size_t zeroed, cudaStream_t s) {
  if (!p) return;
  std::lock_guard<std::mutex> g(g_big_mu);
  auto it = g_big_live.find(p);
  if (it == g_big_live.end()) {  // a small block from the pool
    cudaFreeAsync(p, s);
    return;
  }
  const size_t bytes = it->second.first;
  const int dev = it->second.second;
  g_big_live.erase(it);
  cudaEvent_t ev = nullptr;
  if (g_big_cached + bytes <= BIG_CACHE_MAX && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess &&
      cudaEventRecord(ev, s) == cudaSuccess) {
    g_big_cache.push_back(CachedBlock{p, bytes, dev, ev, std::min(zeroed, bytes)});
    g_big_cached += bytes;
    return;
  }
  cudaGetLastError();
  if (ev) cudaEventDestroy(ev);
  cudaFreeAsync(p, s);
}

void big_free(void* p, cudaStream_t s) { big_free_zeroed(p, 0, s); }

static std::mutex g_pin_mu;
static std::vector<void*> g_pin_free;

void* pinned_get() {
  std::lock_guard<std::mutex> g(g_pin_mu);
  if (g_pin_free.empty()) {
    constexpr size_t CHUNK = 256;  // blocks per chunk
    char* c = nullptr;
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    if (cudaMallocHost((void**)&c, CHUNK * PINNED_BLOCK) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (size_t k = 0; k < CHUNK; ++k) g_pin_free.push_back(c + k * PINNED_BLOCK);
  }
  void* p = g_pin_free.back();
  g_pin_free.pop_back();
  return p;
}

void pinned_put(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> g(g_pin_mu);
  g_pin_free.push_back(p);
}

static void CUDART_CB pinned_put_cb(void* p) { pinned_put(p); }

void pinned_put_after(cudaStream_t s, void* p) {
  if (!p) return;
  if (cudaLaunchHostFunc(s, pinned_put_cb, p) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(s);
    pinned_put(p);
  }
}

void tree_release(TreeMem& t) {
  cudaStream_t s = 0;
  for (void* p : {(void*)t.A.c, (void*)t.A.id, (void*)t.nodes, (void*)t.ndim, (void*)t.shared_next, (void*)t.st})
    big_free(p, s);
  // the delete scratch is all zero again after every delete: the next tree's
  // first delete can take it without a fill
  const bool clean = !t.scratch_dirty;
  big_free_zeroed(t.dead, clean ? t.cap : 0, s);
  big_free_zeroed(t.aux, clean ? t.node_cap * 4 : 0, s);
  ids_release(t.ids, s);
  big_free(t.bbox, s);
  pinned_put_after(s, t.st_host);
  t = TreeMem{};
}

namespace {
constexpr int STORE_WORDS = 64;  // 256 bytes of kernel arguments a launch
struct StoreBlock {
  uint32_t w[STORE_WORDS];
};
__global__ void k_store_words(uint32_t* dst, StoreBlock v, uint32_t n) {
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = v.w[i];
}
__global__ void k_copy_words(uint32_t* dst, const uint32_t* src, uint32_t n) {
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}
__global__ void k_fill_bytes(uint8_t* p, uint8_t v, uint32_t n) {
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) p[i] = v;
}
__global__ void k_fill16(uint4* p, uint4 v, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = v;
}
}  // namespace

int dev_fill(void* dst, int value, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return PKD_OK;
  uint8_t* p = (uint8_t*)dst;
  const uint8_t v = (uint8_t)(value & 0xFF);
  size_t head = (16 - ((uintptr_t)p & 15)) & 15;
  if (head > bytes) head = bytes;
  const size_t body = (bytes - head) / 16 * 16, tail = bytes - head - body;
  if (head) PKD_LAUNCH(k_fill_bytes<<<1, 32, 0, s>>>(p, v, (uint32_t)head));
  if (body) {
    static int sms = 0;
    if (!sms) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (sms <= 0) sms = 1;
    }
    const uint32_t w = 0x01010101u * v;
    const uint64_t n16 = body / 16;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n16 + 255) / 256, (uint64_t)sms * 8));
    PKD_LAUNCH(k_fill16<<<grid, 256, 0, s>>>((uint4*)(p + head), make_uint4(w, w, w, w), n16));
  }
  if (tail) PKD_LAUNCH(k_fill_bytes<<<1, 32, 0, s>>>(p + head + body, v, (uint32_t)tail));
  PKD_CUDA(cudaGetLastError());
  return PKD_OK;
}

int dev_store(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes % 4 || ((uintptr_t)dst & 3)) return PKD_EINVAL;
  if (bytes > 4096) {
    PKD_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
    return PKD_OK;
  }
  const uint32_t nw = (uint32_t)(bytes / 4);
  for (uint32_t o = 0; o < nw; o += STORE_WORDS) {
    StoreBlock v{};
    const uint32_t n = std::min<uint32_t>(STORE_WORDS, nw - o);
    memcpy(v.w, (const uint32_t*)src + o, (size_t)n * 4);
    PKD_LAUNCH(k_store_words<<<1, 64, 0, s>>>((uint32_t*)dst + o, v, n));
  }
  PKD_CUDA(cudaGetLastError());
  return PKD_OK;
}

int dev_copy_words(uint32_t* dst, const uint32_t* src, uint32_t n, cudaStream_t s) {
  if (n == 0) return PKD_OK;
  PKD_LAUNCH(k_copy_words<<<1, 256, 0, s>>>(dst, src, n));
  PKD_CUDA(cudaGetLastError());
  return PKD_OK;
}

static std::mutex g_use_mu;

void tree_touch(TreeMem& t, cudaStream_t s, bool noalloc) {
  std::lock_guard<std::mutex> g(g_use_mu);
  for (auto& u : t.uses)
    if (u.first == s) {
      if (cudaEventRecord(u.second, s) != cudaSuccess) {
        cudaGetLastError();
        t.untracked = true;
      }
      return;
    }
  cudaEvent_t ev = nullptr;
  if (noalloc || cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(ev, s) != cudaSuccess) {
    cudaGetLastError();
    if (ev) cudaEventDestroy(ev);
    t.untracked = true;
    return;
  }
  t.uses.emplace_back(s, ev);
}

void tree_wait_uses(TreeMem& t) {
  std::lock_guard<std::mutex> g(g_use_mu);
  if (t.untracked) cudaDeviceSynchronize();
  for (auto& u : t.uses) {
    if (!t.untracked) cudaStreamWaitEvent(0, u.second, 0);
    cudaEventDestroy(u.second);
  }
  t.uses.clear();
  t.untracked = false;
}

cudaStream_t side_stream() {
  static cudaStream_t streams[64] = {};
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    streams[dev] = nullptr;
  }
  return streams[dev];
}

int export_from(const HostTree& h, uint32_t root, uint64_t top, uint64_t size, uint8_t* dims, int32_t* splits,
                uint64_t* sizes, uint64_t* n_nodes, uint32_t* leaf_ids, uint64_t* leaf_offsets, uint64_t* n_leaves) {
  uint64_t nn = 0, nl = 0, nid = 0;
  std::vector<uint32_t> stack;
  stack.push_back(root);
  while (!stack.empty()) {
    const uint32_t v = stack.back();
    stack.pop_back();
    if (v >= h.nodes.size() || nn > h.nodes.size()) return PKD_EINTERNAL;
    const Node& nd = h.nodes[v];
    const uint8_t dm = h.ndim[v];
    if (dm == PKD_LEAF) {
      if ((uint64_t)nd.a + nd.size > top || nid + nd.size > size) return PKD_EINTERNAL;
      if (dims) dims[nn] = PKD_LEAF;
      if (splits) splits[nn] = 0;
      if (sizes) sizes[nn] = nd.size;
      if (leaf_offsets) leaf_offsets[nl] = nid;
      if (leaf_ids) {
        for (uint32_t k = 0; k < nd.size; ++k) leaf_ids[nid + k] = h.ids[(uint64_t)nd.a + k];
        std::sort(leaf_ids + nid, leaf_ids + nid + nd.size);
      }
      nid += nd.size;
      ++nl;
    } else {
      if (dims) dims[nn] = dm;
      if (splits) splits[nn] = nd.split;
      if (sizes) sizes[nn] = nd.size;
      stack.push_back(nd.b);
      stack.push_back(nd.a);
    }
    ++nn;
  }
  if (leaf_offsets) leaf_offsets[nl] = nid;
  if (n_nodes) *n_nodes = nn;
  if (n_leaves) *n_leaves = nl;
  return PKD_OK;
}

int download_tree(const TreeMem& t, HostTree& h, bool with_ids) {
  const uint64_t used = t.shared_cap + 2 * t.top;
  h.nodes.resize(used);
  h.ndim.resize(used);
  PKD_CUDA(cudaDeviceSynchronize());
  PKD_CUDA(cudaMemcpy(h.nodes.data(), t.nodes, used * sizeof(Node), cudaMemcpyDeviceToHost));
  PKD_CUDA(cudaMemcpy(h.ndim.data(), t.ndim, used, cudaMemcpyDeviceToHost));
  if (with_ids) {
    h.ids.resize(std::max<uint64_t>(t.top, 1));
    if (t.top) PKD_CUDA(cudaMemcpy(h.ids.data(), t.A.id, t.top * 4, cudaMemcpyDeviceToHost));
  }
  return PKD_OK;
}

int tree_alloc(TreeMem& t, const Params& p, uint64_t cap, uint64_t shared_cap, cudaStream_t s) {
  t.p = p;
  cudaGetDevice(&t.device);
  t.cap = std::max<uint64_t>(cap, 1);
  t.shared_cap = shared_cap;
  t.node_cap = shared_cap + 2 * t.cap;
  if (t.node_cap >= 0xFFFFFFF0ull) return PKD_EINVAL;
  cudaError_t e;
  e = big_alloc((void**)&t.A.c, (size_t)p.d * t.cap * 4, s);
  if (e == cudaSuccess) e = big_alloc((void**)&t.A.id, (size_t)t.cap * 4, s);
  if (e == cudaSuccess) e = big_alloc((void**)&t.nodes, (size_t)t.node_cap * sizeof(Node), s);
  if (e == cudaSuccess) e = big_alloc((void**)&t.ndim, (size_t)t.node_cap, s);
  if (e == cudaSuccess) e = pool_alloc((void**)&t.shared_next, 16, s);
  if (e == cudaSuccess) e = pool_alloc((void**)&t.st, sizeof(DevStatus), s);
  static_assert(sizeof(DevStatus) <= PINNED_BLOCK, "status block");
  if (e == cudaSuccess) {
    t.st_host = (DevStatus*)pinned_get();
    if (!t.st_host) e = cudaErrorMemoryAllocation;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    tree_release(t);
    return e == cudaErrorMemoryAllocation ? PKD_ENOMEM : PKD_ECUDA;
  }
  t.A.stride = t.cap;
  dev_fill(t.st, 0, sizeof(DevStatus), s);
  dev_fill(t.shared_next, 0, 16, s);
  return PKD_OK;
}

}  // namespace pkd

using namespace pkd;

extern "C" {

const char* pkd_strerror(int code) {
  switch (code) {
    case PKD_OK: return "ok";
    case PKD_EINVAL: return "invalid argument";
    case PKD_ENOMEM: return "out of device memory";
    case PKD_ECUDA: return "CUDA runtime error";
    case PKD_ETIMEOUT: return "device-side wait ran out";
    case PKD_EINTERNAL: return "device-side consistency check failed";
    default: return "unknown error";
  }
}

int pkd_build(const int32_t* coords, const uint32_t* ids, uint64_t n, const pkd_params* params,
              void* stream, pkd_tree** out) {
  if (!out) return PKD_EINVAL;
  *out = nullptr;
  int e = check_params(params);
  if (e) return e;
  if (n >= (1ull << 31)) return PKD_EINVAL;
  if (n > 0 && !coords) return PKD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Params p{params->d, params->phi, params->lambda, params->sigma_log2, params->sigma_os,
           params->count_mode, params->alpha_num, params->alpha_den, params->seed};
  bool ok;
  trace_mark(s, "build: enter");
  e = validate_coords(coords, n * (uint64_t)p.d, s, &ok);
  if (e) return e;
  if (!ok) return PKD_EINVAL;
  trace_mark(s, "build: validate");
  pkd_tree* t = new pkd_tree();
  // Rebuilt subtrees take fresh arena ranges, so a batch insert that
  // touches most leaves needs about n + (its points + the leaves' points)
  // positions: leave room for that before the first growth (a copy).
  // Node slots are 32-bit (2 per arena position), so very large trees
  // start closer to their size.
  uint64_t cap = 2 * n + n / 4 + 4096;
  if (shared_region_for(p, cap) + 2 * cap >= 0xF0000000ull) cap = n + n / 4 + 4096;
  e = tree_alloc(t->m, p, cap, shared_region_for(p, cap), s);
  if (e) {
    delete t;
    return e;
  }
  t->m.root = 0;
  uint32_t one = 1;
  dev_store(t->m.shared_next, &one, 4, s);
  // The id table (id -> coordinates, and the check that ids are unique) is
  // filled on a second stream while the shared-memory base cases run: they
  // are bound by instruction issue, the table fill by memory traffic.
  cudaStream_t s2 = side_stream();
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (!s2 || cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    for (cudaEvent_t x : ev)
      if (x) cudaEventDestroy(x);
    tree_release(t->m);
    delete t;
    return PKD_ECUDA;
  }
  int eid = PKD_OK;
  bool queued = false;
  pkd_tree* tt = t;
  auto fill_ids = [&](cudaEvent_t start) {
    queued = true;
    if (!start) {
      cudaEventRecord(ev[0], s);
      start = ev[0];
    }
    cudaStreamWaitEvent(s2, start, 0);
    eid = ids_create(tt->m, n, s2);
    if (eid == PKD_OK) ids_claim(tt->m, coords, ids, n, nullptr, s2);
    cudaEventRecord(ev[1], s2);
  };
  BuildJob job;
  job.before_base = fill_ids;
  job.input_coords = coords;
  job.input_ids = ids;
  job.base = 0;
  job.extent = std::max<uint64_t>(n, 1);
  job.segs.push_back(Seg{0, (uint32_t)n, 0, 0, IN_INPUT});
  trace_mark(s, "build: alloc tree");
  e = run_build(t->m, job, s);
  trace_mark(s, "build: run_build");
  if (e == PKD_OK && !queued) fill_ids(nullptr);  // run_build returned before its base cases
  cudaStreamWaitEvent(s, ev[1], 0);
  if (e == PKD_OK) e = eid;
  if (e == PKD_OK) e = check_status(t->m, s);
  if (e == PKD_OK && t->m.st_host->idflags) e = (t->m.st_host->idflags & IDF_FULL) ? PKD_EINTERNAL : PKD_EINVAL;
  cudaStreamSynchronize(s2);
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (e) {
    tree_release(t->m);
    delete t;
    return e;
  }
  t->m.size = n;
  t->m.top = n;
  t->m.ids.live = n;
  t->m.ids.used = n;
  tree_touch(t->m, s);
  *out = t;
  return PKD_OK;
}

void pkd_free(pkd_tree* t) {
  if (!t) return;
  trace_mark(0, "free: enter");
  tree_wait_uses(t->m);  // the frees below are ordered after every call's work
  tree_release(t->m);
  delete t;
  trace_mark(0, "free: release");
}

uint64_t pkd_size(const pkd_tree* t) { return t ? t->m.size : 0; }

int pkd_export(const pkd_tree* tc, uint8_t* dims, int32_t* splits, uint64_t* sizes, uint64_t* n_nodes,
               uint32_t* leaf_ids, uint64_t* leaf_offsets, uint64_t* n_leaves) {
  if (!tc) return PKD_EINVAL;
  HostTree h;
  int e = download_tree(tc->m, h);
  if (e) return e;
  return export_from(h, tc->m.root, tc->m.top, tc->m.size, dims, splits, sizes, n_nodes, leaf_ids, leaf_offsets,
                     n_leaves);
}

int pkd_height(const pkd_tree* tc, int* height) {
  if (!tc || !height) return PKD_EINVAL;
  HostTree h;
  int e = download_tree(tc->m, h, false);
  if (e) return e;
  int best = 0;
  std::vector<std::pair<uint32_t, int>> stack{{tc->m.root, 0}};
  while (!stack.empty()) {
    auto [v, dep] = stack.back();
    stack.pop_back();
    if (v >= h.nodes.size() || dep > 100000) return PKD_EINTERNAL;
    if (h.ndim[v] == PKD_LEAF) {
      best = std::max(best, dep);
    } else {
      stack.push_back({h.nodes[v].a, dep + 1});
      stack.push_back({h.nodes[v].b, dep + 1});
    }
  }
  *height = best;
  return PKD_OK;
}

int pkd_set_option(const char* name, int64_t value) {
  if (!name) return PKD_EINVAL;
  std::string n(name);
  if (n == "base_cap") {
    if (value != 0 && (value < 64 || value > 16384)) return PKD_EINVAL;
    knobs().base_cap = (int)value;
  } else if (n == "skel_cap") {
    if (value != 0 && (value < 64 || value > 16384)) return PKD_EINVAL;
    knobs().skel_cap = (int)value;
  } else if (n == "front_cap") {
    if (value < 0) return PKD_EINVAL;
    knobs().front_cap = value;
  } else if (n == "sieve_kernel") {
    if (value < 0 || value > 2) return PKD_EINVAL;
    knobs().sieve_kernel = (int)value;
  } else if (n == "base_kernel") {
    if (value != 0 && value != 1) return PKD_EINVAL;
    knobs().base_kernel = (int)value;
  } else if (n == "fail_alloc_after") {
    if (value < -1) return PKD_EINVAL;
    knobs().fail_alloc_after = value;
    g_fail_budget.store(value);
  } else if (n == "wait_cycles") {
    if (value < 0 || value > 4000000000000ll) return PKD_EINVAL;
    knobs().wait_cycles = value;
  } else if (n == "graph_rounds") {
    if (value != 0 && value != 1) return PKD_EINVAL;
    knobs().graph_rounds = (int)value;
  } else if (n == "tile") {
    if (value < 256 || value > 4096 || (value & (value - 1))) return PKD_EINVAL;
    knobs().tile = (int)value;
  } else {
    return PKD_EINVAL;
  }
  return PKD_OK;
}

int pkd_mem_info(uint64_t* device_free, uint64_t* pool_reserved, uint64_t* pool_used, uint64_t* cached,
                 uint64_t* available) {
  size_t fr = 0, tot = 0;
  PKD_CUDA(cudaMemGetInfo(&fr, &tot));
  cudaMemPool_t pool = mem_pool();
  uint64_t res = 0, used = 0;
  cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &res);
  cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
  int dev = 0;
  cudaGetDevice(&dev);
  uint64_t cache = 0;
  {
    std::lock_guard<std::mutex> g(g_big_mu);
    for (const CachedBlock& b : g_big_cache)
      if (b.dev == dev) cache += b.bytes;
  }
  // blocks in the large-block cache are counted as used by the pool
  const uint64_t pool_free = res > used ? res - used : 0;
  if (device_free) *device_free = fr;
  if (pool_reserved) *pool_reserved = res;
  if (pool_used) *pool_used = used;
  if (cached) *cached = cache;
  if (available) *available = (uint64_t)fr + pool_free + cache;
  return PKD_OK;
}

int pkd_kernel_timing(int enable) {
  std::lock_guard<std::mutex> g(g_tmu);
  resolve_pending();
  g_stats.clear();
  g_launches.store(0);
  g_timing = enable != 0;
  return PKD_OK;
}

int pkd_kernel_stats(const char* name, uint64_t* launches, double* total_ms, uint64_t* items) {
  if (!name) return PKD_EINVAL;
  std::lock_guard<std::mutex> g(g_tmu);
  if (std::string(name) == "launches") {
    if (launches) *launches = g_launches.load();
    if (total_ms) *total_ms = 0;
    if (items) *items = 0;
    return PKD_OK;
  }
  if (std::string(name) == "graph_builds") {  // since the library was loaded
    if (launches) *launches = (uint64_t)graph_builds();
    if (total_ms) *total_ms = 0;
    if (items) *items = (uint64_t)graph_reuses();
    return PKD_OK;
  }
  if (std::string(name) == "allocations") {  // since the library was loaded
    if (launches) *launches = g_allocs.load();
    if (total_ms) *total_ms = 0;
    if (items) *items = 0;
    return PKD_OK;
  }
  resolve_pending();
  auto it = g_stats.find(name);
  TimerStat s = it == g_stats.end() ? TimerStat{} : it->second;
  if (launches) *launches = s.launches;
  if (total_ms) *total_ms = s.ms;
  if (items) *items = s.items;
  return PKD_OK;
}

}  // extern "C"
