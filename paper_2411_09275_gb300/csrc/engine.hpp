// Host-side engine state of a Pkd-tree (device memory it owns, streams,
// tuning knobs, kernel timers).
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <string>
#include <vector>

#include "common.cuh"
#include "ids.cuh"

namespace pkd {

// Tunables; none of them changes any result.
struct Knobs {
  long long fail_alloc_after = -1;  // >= 0: allocations fail after this many more (fault injection)
  long long wait_cycles = 4000000000ll;  // limit of the streaming sieve's waits (clock cycles, ~2 s)
  int base_cap = 0;   // 0: derived from d and the shared memory per block
  int skel_cap = 0;   // 0: derived
  int tile = 2048;    // points per tile in the sieve kernels
  int base_kernel = 0;  // base case: 0 presorted lists, 1 radix select per node
  int sieve_kernel = 0;  // sieve: 0 persistent with bulk copies and recorded
                         // buckets, 2 persistent re-walking, 1 one tile per CTA
  int graph_rounds = 1;  // build rounds: 1 decided on the device (one CUDA graph
                         // with conditional nodes), 0 sequenced by the host
  long long front_cap = 0;  // > 0: first capacity of an update's flatten lists (testing)
};
Knobs& knobs();

// Device memory of one tree.
//
// Node slots: [0, shared_cap) is a shared region handed out by an atomic
// counter (skeleton nodes of sieve rounds, tree roots); slot
// shared_cap + 2*pos + k (k < 2) belongs to arena position pos, so the
// nodes of a subproblem finished in shared memory over positions
// [s, s + L) live in [shared_cap + 2s, shared_cap + 2s + 2L) without any
// global coordination (a binary tree over L >= 1 points has <= 2L - 1 nodes).
struct TreeMem {
  Params p{};
  int device = 0;
  Pts A{};                 // point arena (SoA), capacity `cap`
  uint64_t cap = 0;
  uint64_t top = 0;        // arena positions [0, top) are in use or garbage
  Node* nodes = nullptr;
  uint8_t* ndim = nullptr;
  uint64_t shared_cap = 0;
  uint64_t node_cap = 0;   // shared_cap + 2*cap
  uint32_t* shared_next = nullptr;  // device: next free slot of the shared region
  uint32_t root = 0;
  uint64_t size = 0;
  uint8_t* dead = nullptr;          // delete scratch: per arena position (kept zero)
  uint32_t* aux = nullptr;          // delete scratch: per node slot (kept zero)
  bool scratch_dirty = false;       // a delete has set marks it has not cleared yet
  DevStatus* st = nullptr;          // device status word
  DevStatus* st_host = nullptr;     // pinned mirror
  IdTable ids;                      // id -> coordinates of the stored points
  int32_t* bbox = nullptr;          // stored bounding boxes (boxes.cu), node_cap * 2d
  uint64_t bbox_cap = 0;            // node slots bbox covers
  bool bbox_on = false;             // kept current after every update; queries prune with them
  // the last use of the tree on every stream a call queued work on (an event
  // recorded after that work), so that freeing the tree waits for exactly
  // that work; untracked: a use that could not record one (a call that may
  // not allocate), after which freeing waits for the whole device
  std::vector<std::pair<cudaStream_t, cudaEvent_t>> uses;
  bool untracked = false;
};

// Small host values into device memory, in stream order, by a kernel that
// takes them as arguments (bytes: a multiple of 4, dst 4-byte aligned).  A
// host-to-device copy would queue behind whatever large copy the caller has
// on the same copy engine (the next step's input, say) and hold the stream
// back for its whole duration; a kernel does not.  Up to 4 KiB; larger
// values go through cudaMemcpyAsync.
int dev_store(void* dst, const void* src, size_t bytes, cudaStream_t s);
// n words from device to device the same way (a small copy).
int dev_copy_words(uint32_t* dst, const uint32_t* src, uint32_t n, cudaStream_t s);
// bytes of dst set to `value` by a kernel (for the same reason: a fill that
// the runtime may hand to a copy engine would wait for the caller's copies).
int dev_fill(void* dst, int value, size_t bytes, cudaStream_t s);

// Records the use of tree t by the work queued so far on stream s.
void tree_touch(TreeMem& t, cudaStream_t s, bool noalloc = false);
// Orders the legacy default stream after every recorded use (or, after an
// untracked one, waits for the device) and forgets the uses.
void tree_wait_uses(TreeMem& t);

// Records the tree's use by the calling entry point when it returns (every
// return path, after its last enqueue).
struct TreeTouch {
  TreeMem* t;
  cudaStream_t s;
  bool noalloc = false;
  ~TreeTouch() {
    if (t) tree_touch(*t, s, noalloc);
  }
};

// Every kernel launch of the library goes through PKD_LAUNCH, which counts
// it (pkd_kernel_stats("launches", ...) reports the count).
void count_launch();
#define PKD_LAUNCH(...)        \
  do {                         \
    ::pkd::count_launch();     \
    __VA_ARGS__;               \
  } while (0)

// Host-side tracing: with PKD_TRACE=1 in the environment, trace_mark()
// synchronises the stream and prints the wall time since the previous mark.
void trace_mark(cudaStream_t s, const char* what);

// Error helpers.
int cuda_err(cudaError_t e);
#define PKD_CUDA(x)                          \
  do {                                       \
    cudaError_t _e = (x);                    \
    if (_e != cudaSuccess) return cuda_err(_e); \
  } while (0)

// The library's stream-ordered memory pool on the current device.  Its
// release threshold is unlimited: memory freed by one build stays mapped for
// the next instead of being returned to the driver at every synchronisation.
cudaMemPool_t mem_pool();

// Large blocks (tree arenas and node arrays) go through a small cache in
// front of the pool: a freed block is kept with an event recorded on the
// freeing stream and handed to the next request it fits (the requesting
// stream waits on that event), so building, updating and freeing trees in a
// loop does not map and unmap gigabytes each time.  Blocks below
// BIG_BLOCK_MIN go straight to the pool.  On exhaustion the cache is
// emptied and the request retried once.
constexpr size_t BIG_BLOCK_MIN = (size_t)64 << 20;
cudaError_t big_alloc(void** p, size_t bytes, cudaStream_t s);
void big_free(void* p, cudaStream_t s);
// The same for a block that must start zeroed: *zero says whether the block
// handed out is known to be zero over `bytes` (a cached block released with
// big_free_zeroed); otherwise the caller clears it.
cudaError_t big_alloc_zeroed(void** p, size_t bytes, cudaStream_t s, bool* zero);
void big_free_zeroed(void* p, size_t zeroed, cudaStream_t s);

// Every device allocation of the library goes through pool_alloc: a
// stream-ordered allocation from the pool above that is counted (reported by
// pkd_kernel_stats("allocations")) and that fails with
// cudaErrorMemoryAllocation, without allocating, once the option
// "fail_alloc_after" is set to k >= 0 and k allocations have succeeded since
// (host-side fault injection for the out-of-memory paths).
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s);

// Stream-ordered allocation from that pool.
template <class T>
int dalloc(T** p, size_t n, cudaStream_t s) {
  *p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = pool_alloc((void**)p, n * sizeof(T), s);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return PKD_ENOMEM;
  }
  return e == cudaSuccess ? PKD_OK : cuda_err(e);
}
template <class T>
void dfree(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
}

// Pinned host blocks of PINNED_BLOCK bytes from a library-owned pool that
// grows by whole chunks and is never returned (pinning and unpinning memory
// are slow, synchronising driver calls).  nullptr when pinning fails.
constexpr size_t PINNED_BLOCK = 256;
void* pinned_get();
void pinned_put(void* p);
// Return a block once the work queued on `s` so far has completed (a copy
// into it may still be in flight).
void pinned_put_after(cudaStream_t s, void* p);

// A pinned block of PINNED_BLOCK bytes owned by one scope.
struct PinnedBlock {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  explicit PinnedBlock(cudaStream_t st) : p(pinned_get()), s(st) {}
  ~PinnedBlock() { pinned_put_after(s, p); }
  PinnedBlock(const PinnedBlock&) = delete;
  PinnedBlock& operator=(const PinnedBlock&) = delete;
};

// Reads the device status word; PKD_OK or the mapped error.
int check_status(TreeMem& t, cudaStream_t s);

// Kernel timing (CUDA events on the launching stream).
struct KTimer {
  bool on = false;
  cudaEvent_t a = nullptr, b = nullptr;
  std::string name;
  uint64_t items = 0;
  cudaStream_t s = nullptr;
};
void ktimer_begin(KTimer& k, const char* name, uint64_t items, cudaStream_t s);
void ktimer_end(KTimer& k);
bool ktiming_enabled();
// While timing is on, add `items` to the counter family `name` (a count
// with no kernel time, e.g. the points a batch update rebuilt).
void stat_items(const char* name, uint64_t items);
// A host-side duration (ms) under a timer family (e.g. recording a graph).
void stat_host_ms(const char* name, double ms, uint64_t items);

// A build of independent subproblems ("segments"): every segment's points
// sit at arena positions [start, start+len) of A (or of the caller's input
// when `input_coords` is set), its root goes to node slot `root`, its depth
// salts the samples.  On return each segment's points are in A in leaf order
// and its subtree is written to the node arrays.
struct BuildJob {
  const int32_t* input_coords = nullptr;  // point-major input (segments IN_INPUT)
  const uint32_t* input_ids = nullptr;
  uint64_t base = 0;       // lowest arena position of any segment
  uint64_t extent = 0;     // highest position + 1 - base
  std::vector<Seg> segs;   // host list of root segments, or:
  const Seg* dsegs = nullptr;  // device list of root segments (dsegs_n of them)
  uint64_t dsegs_n = 0;
  // Called once on the host when the shared-memory base cases have been
  // queued or recorded (work that should overlap them, which are bound by
  // instruction issue rather than memory traffic, is queued from here).  The
  // argument is an event that completes when they may start (null: the work
  // queued so far on the stream).
  std::function<void(cudaEvent_t)> before_base;
};
int run_build(TreeMem& t, const BuildJob& job, cudaStream_t s);

// Builds whose rounds ran from one graph launch (since the library was loaded).
int graph_builds();
// ... of them, the builds that launched a graph recorded by an earlier build.
int graph_reuses();

// True while this host thread records a CUDA graph (kernel timers are off).
bool& flow_capturing();

// Derived shared-memory capacities.
int base_cap_for(int d);
int skel_cap_for(int d);

}  // namespace pkd
