// sort.cu -- prefix scans, visibility compaction and the stable LSD radix sort that build the
// front-to-back ordered covering lists (Section 3.1: per pixel, the covering Gaussians near to
// far). All scans are reduce-then-scan (three kernels, no inter-block waiting), so no kernel
// here ever spins on another block, except the single-pass scan, whose waits are bounded and
// only ever on blocks that have already started. Sorts that fit in the shared memory of one
// thread-block cluster run as a single launch whose blocks meet only at the hardware cluster
// barrier (the blocks of a cluster are co-scheduled by construction).
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "rgs_internal.cuh"

namespace cg = cooperative_groups;

namespace rgs {
namespace {

__device__ __forceinline__ uint32_t read_count(const uint32_t* n_dev, int64_t n_cap) {
  if (!n_dev) return (uint32_t)n_cap;
  const uint32_t n = *n_dev;
  return n < (uint64_t)n_cap ? n : (uint32_t)n_cap;
}

// Block-wide exclusive scan of one value per thread; returns the block total in *total.
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sums[THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < THREADS / 32 ? warp_sums[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < THREADS / 32) warp_sums[lane] = w;  // inclusive warp prefix
  }
  __syncthreads();
  const uint32_t warp_prefix = warp > 0 ? warp_sums[warp - 1] : 0u;
  if (total) *total = warp_sums[THREADS / 32 - 1];
  const uint32_t r = warp_prefix + x - v;
  __syncthreads();  // warp_sums may be reused by the caller's next scan
  return r;
}

// Lanes of the warp whose valid keys carry the same digit as this lane's (0 for an invalid
// lane): one ballot per digit bit, each keeping the lanes that agree on that bit.
__device__ __forceinline__ uint32_t warp_digit_peers(uint32_t digit, bool valid, int nbits) {
  uint32_t peers = __ballot_sync(0xffffffffu, valid);
  for (int b = 0; b < nbits; ++b) {
    const uint32_t bit = (digit >> b) & 1u;
    const uint32_t ones = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? ones : ~ones;
  }
  return valid ? peers : 0u;
}

// Loaders: value of element k.
struct PlainLoad {
  const uint32_t* in;
  __device__ uint32_t operator()(uint32_t k) const { return in[k]; }
};
struct GatherLoad {
  const uint32_t* in;
  const uint32_t* order;
  __device__ uint32_t operator()(uint32_t k) const { return in[order[k]]; }
};

// Pass 1: per-block sums.
template <typename Load>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(Load load, int64_t n_cap,
                                                                   const uint32_t* n_dev,
                                                                   uint32_t* block_sums) {
  chain_wait();
  const uint32_t n = read_count(n_dev, n_cap);
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t s = 0;
  if (base < n) {
#pragma unroll 4
    for (int k = 0; k < kScanItems; ++k) {
      const int64_t idx = base + (int64_t)k * kScanThreads + threadIdx.x;
      if (idx < n) s += load((uint32_t)idx);
    }
  }
  uint32_t total;
  block_exclusive_scan<kScanThreads>(s, &total);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// Pass 2: one block scans the block sums in place (exclusive) and writes the grand total.
__global__ void __launch_bounds__(1024) scan_block_sums_kernel(uint32_t* block_sums,
                                                               int64_t n_blocks,
                                                               uint32_t* total) {
  chain_wait();
  uint32_t carry = 0;
  for (int64_t base = 0; base < n_blocks; base += 1024 * 4) {
    uint32_t v[4];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t idx = base + (int64_t)threadIdx.x * 4 + k;
      v[k] = idx < n_blocks ? block_sums[idx] : 0u;
      s += v[k];
    }
    uint32_t chunk_total;
    uint32_t pre = block_exclusive_scan<1024>(s, &chunk_total);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t idx = base + (int64_t)threadIdx.x * 4 + k;
      if (idx < n_blocks) block_sums[idx] = carry + pre;
      pre += v[k];
    }
    carry += chunk_total;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

// Pass 3: per-block exclusive scan plus the block's offset; the Store functor writes results.
struct PlainStore {
  uint32_t* out;
  __device__ void operator()(uint32_t k, uint32_t value, uint32_t prefix) const {
    (void)value;
    out[k] = prefix;
  }
};

template <typename Load, typename Store>
__global__ void __launch_bounds__(kScanThreads) scan_downsweep_kernel(Load load, Store store,
                                                                      int64_t n_cap,
                                                                      const uint32_t* n_dev,
                                                                      const uint32_t* block_sums) {
  chain_wait();
  const uint32_t n = read_count(n_dev, n_cap);
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  if (base >= n) return;
  // Thread t owns the kScanItems consecutive elements base + t * kScanItems + k.
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t idx = base + (int64_t)threadIdx.x * kScanItems + k;
    v[k] = idx < n ? load((uint32_t)idx) : 0u;
    s += v[k];
  }
  uint32_t pre = block_exclusive_scan<kScanThreads>(s, nullptr) + block_sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t idx = base + (int64_t)threadIdx.x * kScanItems + k;
    if (idx < n) store((uint32_t)idx, v[k], pre);
    pre += v[k];
  }
}

// ------------------------------------------------------------------------------------------
// Single-cluster scan: one launch of one cluster of C blocks (16, else 8) of 1024 threads for
// n_cap up to kCscanMaxN (and C * shared memory / sizeof(T)). Block c holds the slice [c S, (c + 1) S),
// S = ceil(n / C), of the loaded values in shared memory (as T: bytes for 0/1 flags); each
// thread sums a contiguous run of it, a block scan gives the runs' offsets and the block total,
// and one cluster barrier lets every block add the totals of the blocks before it (read from
// their shared memory). The runs are then walked again to store the results. Every block
// executes both cluster barriers, also with an empty slice.
// ------------------------------------------------------------------------------------------
constexpr int kCscanThreads = 1024;
constexpr size_t kCscanMaxSmem = 200 * 1024;  // dynamic shared memory per block, at most
constexpr int kCscanUnroll = 16;
// Largest n_cap routed to the single-cluster scan. Measured on GB300: it wins for short inputs
// (a 45k gather scan: 12.6 instead of 18.8 us) but not for long ones (a 144k gather scan: 18.4
// against 18.1 us; a 1.5M flag compaction: 70 against 25 us), where three kernels spread the work
// over every SM.
constexpr int64_t kCscanMaxN = 64 * 1024;

template <typename Load, typename Store, typename T>
__global__ void __launch_bounds__(kCscanThreads, 1) cluster_scan_kernel(Load load, Store store,
                                                                       int64_t n_cap,
                                                                       const uint32_t* n_dev,
                                                                       uint32_t* total) {
  chain_wait();
  extern __shared__ __align__(16) unsigned char cscan_smem[];
  T* buf = reinterpret_cast<T*>(cscan_smem);
  __shared__ uint32_t s_block_total, s_base;
  cg::cluster_group cluster = cg::this_cluster();
  const uint32_t C = cluster.num_blocks(), me = cluster.block_rank();
  const int tid = threadIdx.x;
  const uint32_t n = read_count(n_dev, n_cap);
  const uint32_t S = (n + C - 1) / C;
  const uint32_t lo = me * S;
  const uint32_t cnt = n > lo ? min(S, n - lo) : 0u;
  // Loads in rounds of kCscanUnroll per thread, all issued before any is stored, so that the
  // memory latency is paid once per round rather than once per element.
  for (uint32_t base = 0; base < cnt; base += kCscanThreads * kCscanUnroll) {
    uint32_t v[kCscanUnroll];
#pragma unroll
    for (int u = 0; u < kCscanUnroll; ++u) {
      const uint32_t t = base + (uint32_t)u * kCscanThreads + tid;
      v[u] = t < cnt ? load(lo + t) : 0u;
    }
#pragma unroll
    for (int u = 0; u < kCscanUnroll; ++u) {
      const uint32_t t = base + (uint32_t)u * kCscanThreads + tid;
      if (t < cnt) buf[t] = (T)v[u];
    }
  }
  __syncthreads();
  const uint32_t E = (cnt + kCscanThreads - 1) / kCscanThreads;  // run length per thread
  const uint32_t r0 = min(cnt, (uint32_t)tid * E), r1 = min(cnt, r0 + E);
  uint32_t sum = 0;
  for (uint32_t k = r0; k < r1; ++k) sum += (uint32_t)buf[k];
  uint32_t block_total;
  const uint32_t excl = block_exclusive_scan<kCscanThreads>(sum, &block_total);
  if (tid == 0) s_block_total = block_total;
  cluster.sync();
  if (tid == 0) {
    uint32_t base = 0;
    for (uint32_t r = 0; r < me; ++r) base += *cluster.map_shared_rank(&s_block_total, r);
    s_base = base;
    if (me == C - 1 && total) *total = base + block_total;
  }
  __syncthreads();
  uint32_t run = s_base + excl;
  for (uint32_t k = r0; k < r1; ++k) {
    const uint32_t v = (uint32_t)buf[k];
    store(lo + k, v, run);
    run += v;
  }
  cluster.sync();  // the block totals stay readable until every block has read them
}

// Blocks per cluster of the scan kernel for <Load, Store, T> with up to kCscanMaxSmem bytes of
// dynamic shared memory per block: 16 if one such cluster fits on the device, else 8, else 0
// (per instantiation and device, cached).
template <typename Load, typename Store, typename T>
int cluster_scan_blocks() {
  static std::mutex mu;
  static int cached[64];
  static bool known[64] = {};
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= 64) return 0;
  std::lock_guard<std::mutex> lock(mu);
  if (known[device]) return cached[device];
  auto kernel = cluster_scan_kernel<Load, Store, T>;
  int result = 0;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kCscanMaxSmem) == cudaSuccess &&
      cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
          cudaSuccess) {
    for (const int c : {16, 8}) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(c);
      cfg.blockDim = dim3(kCscanThreads);
      cfg.dynamicSmemBytes = kCscanMaxSmem;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = c;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, kernel, &cfg) == cudaSuccess && clusters > 0) {
        result = c;
        break;
      }
    }
  }
  cudaGetLastError();  // a refused query leaves no sticky error: the three-kernel scan is used
  cached[device] = result;
  known[device] = true;
  return result;
}

// Launches the single-cluster scan if n_cap fits (returns true and the launch status in *e).
template <typename Load, typename Store, typename T>
bool try_cluster_scan(Load load, Store store, int64_t n_cap, const uint32_t* n_dev,
                      uint32_t* total, cudaStream_t stream, cudaError_t* e) {
  if (n_cap <= 0 || n_cap > kCscanMaxN) return false;
  const int blocks = cluster_scan_blocks<Load, Store, T>();
  if (blocks == 0) return false;
  const int64_t slice = (n_cap + blocks - 1) / blocks;
  const size_t smem = (size_t)slice * sizeof(T);
  if (smem > kCscanMaxSmem) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kCscanThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = blocks;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  *e = cudaLaunchKernelEx(&cfg, cluster_scan_kernel<Load, Store, T>, load, store, n_cap, n_dev,
                          total);
  RGS_LAUNCHED();
  return true;
}

// ------------------------------------------------------------------------------------------
// Single-pass scan: the chained scan with decoupled look-back of Merrill and Garland
// ("Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016), in one launch of one
// block per tile of kScanTile elements. A block takes its tile from a ticket counter, so tiles
// are handed out in the order blocks start: a block only ever waits for tiles of blocks that
// are already running, which therefore finish. It scans its tile, publishes the tile total (an
// "aggregate") and, unless it is tile 0, walks back over the earlier tiles 32 at a time (one per
// lane of warp 0), adding aggregates until it meets a published inclusive prefix; then it
// publishes its own inclusive prefix and stores its results. A state word packs the flag in bits 62..63 (0 not yet published, 1 aggregate,
// 2 inclusive prefix) and the value in bits 0..31. It is written and read whole (an aligned
// 64-bit access), and nothing else is published through it, so relaxed accesses suffice. Each
// wait is bounded: past kLookbackSpins polls the block records kStatusScanWait and takes the
// tile as 0 (a wrong result, reported; never expected, since the waited-for block is running).
// ------------------------------------------------------------------------------------------
constexpr unsigned long long kTileAggregate = 1ull << 62, kTileInclusive = 2ull << 62;
constexpr int kLookbackSpins = 1 << 20;  // polls of ~1 us each

__device__ __forceinline__ void store_state(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long load_state(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Takes a tile from the ticket counter (thread 0; the result is broadcast to the block).
__device__ __forceinline__ uint32_t lookback_ticket(const Lookback& lb) {
  __shared__ uint32_t s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(lb.ticket, 1u);
  __syncthreads();
  return s_tile;
}

// Called by the 32 lanes of warp 0 of the block holding tile b, whose elements sum to agg:
// publishes the aggregate, looks back for the exclusive prefix of the tile, publishes the
// inclusive prefix and returns the exclusive one (in every lane).
__device__ uint32_t lookback_prefix(const Lookback& lb, uint32_t b, uint32_t agg) {
  const int lane = threadIdx.x & 31;
  if (b == 0) {
    if (lane == 0) store_state(&lb.tiles[0], kTileInclusive | agg);
    return 0u;
  }
  if (lane == 0) store_state(&lb.tiles[b], kTileAggregate | agg);
  uint32_t prefix = 0;
  bool timed_out = false;
  for (int64_t end = b; end > 0; end -= 32) {
    const int64_t j = end - 1 - lane;  // lane 0 looks at the nearest earlier tile
    unsigned long long w = kTileInclusive;  // before tile 0: an empty inclusive prefix
    if (j >= 0) {
      w = load_state(&lb.tiles[j]);
      for (int spin = 0; (w >> 62) == 0; ++spin) {
        if (spin >= kLookbackSpins) {
          timed_out = true;
          w = kTileInclusive;
          break;
        }
        __nanosleep(32);
        w = load_state(&lb.tiles[j]);
      }
    }
    const uint32_t inclusive = __ballot_sync(0xffffffffu, (w >> 62) == 2ull);
    // Tiles nearer than the nearest inclusive prefix contribute their aggregates, that prefix
    // contributes itself, and the farther tiles nothing.
    const int stop = inclusive ? __ffs(inclusive) - 1 : 32;
    uint32_t x = lane <= stop ? (uint32_t)w : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    prefix += x;
    if (inclusive) break;
  }
  if (__any_sync(0xffffffffu, timed_out) && lane == 0)
    atomicOr(lb.status, (uint32_t)kStatusScanWait);
  if (lane == 0) store_state(&lb.tiles[b], kTileInclusive | (prefix + agg));
  return prefix;
}

template <typename Load, typename Store>
__global__ void __launch_bounds__(kScanThreads) lookback_scan_kernel(Load load, Store store,
                                                                     int64_t n_cap,
                                                                     const uint32_t* n_dev,
                                                                     uint32_t* total,
                                                                     Lookback lb,
                                                                     uint32_t n_tiles) {
  chain_wait();
  __shared__ uint32_t s_prefix;
  const uint32_t b = lookback_ticket(lb);
  if (b >= n_tiles) {  // the ticket counter was not zeroed: report, touch nothing
    if (threadIdx.x == 0) atomicOr(lb.status, (uint32_t)kStatusScanWait);
    return;
  }
  const uint32_t n = read_count(n_dev, n_cap);
  const int64_t base = (int64_t)b * kScanTile;
  // Thread t owns the kScanItems consecutive elements base + t * kScanItems + k.
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t idx = base + (int64_t)threadIdx.x * kScanItems + k;
    v[k] = idx < n ? load((uint32_t)idx) : 0u;
    s += v[k];
  }
  uint32_t agg;
  const uint32_t excl = block_exclusive_scan<kScanThreads>(s, &agg);
  if (threadIdx.x < 32) {
    const uint32_t prefix = lookback_prefix(lb, b, agg);
    if (threadIdx.x == 0) s_prefix = prefix;
  }
  __syncthreads();
  uint32_t pre = s_prefix + excl;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t idx = base + (int64_t)threadIdx.x * kScanItems + k;
    if (idx < n) store((uint32_t)idx, v[k], pre);
    pre += v[k];
  }
  if (b == n_tiles - 1 && threadIdx.x == 0 && total) *total = s_prefix + agg;
}

// ------------------------------------------------------------------------------------------
// Compaction of the visible entries from the visibility bitmask, one single-pass launch. A
// tile is kBitsThreads words, one per thread (coalesced loads). The exclusive prefix of the set
// bits over the threads gives each thread the tile-local position of its first visible entry;
// it writes its entries' indices there, in bit order, into a shared-memory list, while warp 0
// finds the tile's offset by look-back. The block then stores the list with every thread:
// independent loads of the depths, contiguous stores. Words are taken in (view, word) order and
// bits from the lowest, so the output follows (view, Gaussian) order.
// ------------------------------------------------------------------------------------------
constexpr int kBitsThreads = 256;

__global__ void __launch_bounds__(kBitsThreads) compact_bits_kernel(
    const uint32_t* __restrict__ vis_bits, uint32_t n_words, uint32_t words_per_view, uint32_t n,
    const float4* __restrict__ rec2, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
    uint32_t* __restrict__ list, uint32_t* __restrict__ n_out, Lookback lb, uint32_t n_tiles) {
  chain_wait();
  __shared__ uint32_t s_list[kBitsThreads * 32];
  __shared__ uint32_t s_prefix;
  const uint32_t b = lookback_ticket(lb);
  if (b >= n_tiles) {  // the ticket counter was not zeroed: report, touch nothing
    if (threadIdx.x == 0) atomicOr(lb.status, (uint32_t)kStatusScanWait);
    return;
  }
  const uint32_t gw = b * kBitsThreads + threadIdx.x;
  uint32_t m = gw < n_words ? vis_bits[gw] : 0u;
  uint32_t agg;
  uint32_t pos = block_exclusive_scan<kBitsThreads>((uint32_t)__popc(m), &agg);
  if (threadIdx.x < 32) {
    const uint32_t prefix = lookback_prefix(lb, b, agg);
    if (threadIdx.x == 0) s_prefix = prefix;
  }
  if (m) {
    const uint32_t v = gw / words_per_view;
    const uint32_t first = v * n + (gw - v * words_per_view) * 32u;
    while (m) {
      s_list[pos++] = first + (uint32_t)(__ffs(m) - 1);
      m &= m - 1u;
    }
  }
  __syncthreads();
  const uint32_t prefix = s_prefix;
  for (uint32_t t = threadIdx.x; t < agg; t += kBitsThreads) {
    const uint32_t vi = s_list[t];
    keys[prefix + t] = __float_as_uint(rec2[vi].w);
    vals[prefix + t] = vi;
    list[prefix + t] = vi;
  }
  if (b == n_tiles - 1 && threadIdx.x == 0) *n_out = prefix + agg;
}

// Exclusive scan of the loaded values: one single-pass launch when look-back bookkeeping is
// given; else one cluster launch when they fit in a cluster's shared memory (held as T); else
// three kernels.
template <typename Load, typename Store, typename T = uint32_t>
cudaError_t run_scan(Load load, Store store, int64_t n_cap, const uint32_t* n_dev,
                     uint32_t* total, uint32_t* block_sums, cudaStream_t stream,
                     Lookback lb = Lookback{}) {
  const int64_t nb = scan_blocks(n_cap);
  if (nb == 0) {
    if (total) return cudaMemsetAsync(total, 0, sizeof(uint32_t), stream);
    return cudaSuccess;
  }
  cudaError_t e = cudaSuccess;
  if (lb.tiles) {
    if (nb > lb.capacity) return cudaErrorInvalidValue;
    e = launch_chained(lookback_scan_kernel<Load, Store>, dim3((unsigned)nb), dim3(kScanThreads),
                       stream, load, store, n_cap, n_dev, total, lb, (uint32_t)nb);
    RGS_LAUNCHED();
    return e;
  }
  if (try_cluster_scan<Load, Store, T>(load, store, n_cap, n_dev, total, stream, &e)) return e;
  e = launch_chained(scan_reduce_kernel<Load>, dim3((unsigned)nb), dim3(kScanThreads),
                                 stream, load, n_cap, n_dev, block_sums);
  RGS_LAUNCHED();
  if (e == cudaSuccess)
    e = launch_chained(scan_block_sums_kernel, dim3(1), dim3(1024), stream, block_sums, nb, total);
  RGS_LAUNCHED();
  if (e == cudaSuccess)
    e = launch_chained(scan_downsweep_kernel<Load, Store>, dim3((unsigned)nb), dim3(kScanThreads),
                       stream, load, store, n_cap, n_dev, (const uint32_t*)block_sums);
  RGS_LAUNCHED();
  return e;
}

// ------------------------------------------------------------------------------------------
// Radix sort, three kernels per pass:
//   upsweep   per-block digit counts, stored digit-major: hist[d * n_blocks + b];
//   row scan  one block per digit: exclusive scan of its row over the blocks, row total into
//             hist[256 * n_blocks + d];
//   downsweep stable ranks inside the block, a local sort through shared memory, then
//             coalesced stores of each digit's run to its global offset.
// Each block owns kSortTile consecutive keys; warp w of the block owns the contiguous sub-range
// [w * 32 * kSortItems, (w + 1) * 32 * kSortItems) and walks it in rounds of 32 keys (lane l
// takes element r * 32 + l), so warp order, round order and lane order together follow the
// input order, which makes the ranks stable.
// ------------------------------------------------------------------------------------------
template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads) radix_upsweep_kernel(const uint32_t* keys,
                                                                     int64_t n_cap,
                                                                     const uint32_t* n_dev,
                                                                     int shift, uint32_t mask,
                                                                     uint32_t* hist,
                                                                     int64_t n_blocks) {
  chain_wait();
  __shared__ uint32_t counts[kRadixBins];
  const uint32_t n = read_count(n_dev, n_cap);
  for (int d = threadIdx.x; d < kRadixBins; d += kSortThreads) counts[d] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * (kSortThreads * ITEMS);
  if (base < n) {
#pragma unroll 4
    for (int k = 0; k < ITEMS; ++k) {
      const int64_t idx = base + (int64_t)k * kSortThreads + threadIdx.x;
      if (idx < n) atomicAdd(&counts[(keys[idx] >> shift) & mask], 1u);
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadixBins; d += kSortThreads)
    hist[(int64_t)d * n_blocks + blockIdx.x] = counts[d];
}

__global__ void __launch_bounds__(kSortThreads) radix_row_scan_kernel(uint32_t* hist,
                                                                      int64_t n_blocks) {
  chain_wait();
  const int d = blockIdx.x;
  uint32_t* row = hist + (int64_t)d * n_blocks;
  uint32_t carry = 0;
  for (int64_t base = 0; base < n_blocks; base += kSortThreads * 4) {
    uint32_t v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t idx = base + (int64_t)threadIdx.x * 4 + k;
      v[k] = idx < n_blocks ? row[idx] : 0u;
      s += v[k];
    }
    uint32_t chunk_total;
    uint32_t pre = block_exclusive_scan<kSortThreads>(s, &chunk_total);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t idx = base + (int64_t)threadIdx.x * 4 + k;
      if (idx < n_blocks) row[idx] = carry + pre;
      pre += v[k];
    }
    carry += chunk_total;
  }
  if (threadIdx.x == 0) hist[(int64_t)kRadixBins * n_blocks + d] = carry;
}

template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads) radix_downsweep_kernel(
    const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
    int64_t n_cap, const uint32_t* n_dev, int shift, uint32_t mask, const uint32_t* hist,
    int64_t n_blocks) {
  chain_wait();
  static_assert(kSortThreads == kRadixBins, "one thread per digit in the digit scans");
  constexpr int kWarps = kSortThreads / 32;
  constexpr int kTile = kSortThreads * ITEMS;
  __shared__ uint32_t warp_counts[kWarps][kRadixBins];
  __shared__ uint32_t s_keys[kTile];
  __shared__ uint32_t s_vals[kTile];
  __shared__ uint32_t s_digit_start[kRadixBins];   // block-local start of each digit's run
  __shared__ int64_t s_digit_shift[kRadixBins];    // global position minus local position
  const uint32_t n = read_count(n_dev, n_cap);
  const int64_t base = (int64_t)blockIdx.x * kTile;
  if (base >= n) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = lane; d < kRadixBins; d += 32) warp_counts[warp][d] = 0;
  __syncwarp();
  const int64_t wbase = base + (int64_t)warp * 32 * ITEMS;
  uint32_t key[ITEMS], val[ITEMS], rank[ITEMS];
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int nbits = 32 - __clz(mask);  // width of this pass's digit
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const int64_t idx = wbase + r * 32 + lane;
    const bool valid = idx < n;
    key[r] = valid ? keys_in[idx] : 0u;
    val[r] = (valid && vals_in) ? vals_in[idx] : 0u;
    const uint32_t digit = valid ? ((key[r] >> shift) & mask) : kRadixBins;  // kRadixBins = none
    const uint32_t peers = warp_digit_peers(digit, valid, nbits);
    const uint32_t before = __popc(peers & lt_mask);
    uint32_t prior = 0;
    if (valid) prior = warp_counts[warp][digit];
    __syncwarp();
    if (valid && before == 0) warp_counts[warp][digit] = prior + __popc(peers);
    __syncwarp();
    rank[r] = valid ? prior + before : 0xffffffffu;
  }
  __syncthreads();
  {
    // Thread d: exclusive prefix of digit d over the warps, then the block-local and the
    // global start of digit d's run.
    const int d = threadIdx.x;
    uint32_t acc = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = warp_counts[w][d];
      warp_counts[w][d] = acc;
      acc += c;
    }
    const uint32_t local_start = block_exclusive_scan<kSortThreads>(acc, nullptr);
    const uint32_t row_total = hist[(int64_t)kRadixBins * n_blocks + d];
    const uint32_t digit_base = block_exclusive_scan<kSortThreads>(row_total, nullptr);
    s_digit_start[d] = local_start;
    s_digit_shift[d] = (int64_t)digit_base + hist[(int64_t)d * n_blocks + blockIdx.x] -
                       (int64_t)local_start;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    if (rank[r] == 0xffffffffu) continue;
    const uint32_t digit = (key[r] >> shift) & mask;
    const uint32_t local = s_digit_start[digit] + warp_counts[warp][digit] + rank[r];
    s_keys[local] = key[r];
    s_vals[local] = val[r];
  }
  __syncthreads();
  const int count = (int)min((int64_t)kTile, (int64_t)n - base);
  for (int t = threadIdx.x; t < count; t += kSortThreads) {
    const uint32_t k = s_keys[t];
    const int64_t pos = s_digit_shift[(k >> shift) & mask] + t;
    keys_out[pos] = k;
    if (vals_out) vals_out[pos] = s_vals[t];
  }
}

// ------------------------------------------------------------------------------------------
// Wide radix passes for large sorts (the pair list: 10^7 - 10^8 keys): digits of up to 9 bits,
// so that the 17-bit tile ids of a 16-view 1080p window sort in two passes instead of three, and
// blocks of kWideTile = 8192 keys (512 threads x 16), so that each digit's run inside a block is
// long enough for coalesced stores. The same three kernels per pass as above:
//   upsweep   per-block digit counts, digit-major; equal digits of a warp's 32 keys are added
//             once (the keys of one Gaussian's footprint are consecutive tile ids, so the high
//             digits of a warp's keys are mostly equal, and per-key shared-memory atomics would
//             serialise on one address);
//   row scan  one block per digit over the blocks;
//   downsweep stable ranks within each warp's contiguous sub-range (the lanes holding equal
//             digits found by one ballot per digit bit; a match instruction per 32 keys was
//             slower, 2.37 against 1.96 ms for the two passes over 155M pairs), a local sort of
//             keys and values through shared memory (values are read only when they are placed,
//             so the ranking holds keys and ranks only), coalesced stores of each digit's run.
// ------------------------------------------------------------------------------------------
constexpr int kWideThreads = 512;
constexpr int kWideWarps = kWideThreads / 32;
constexpr int kWideItems = 16;
constexpr int kWideTile = kWideThreads * kWideItems;
constexpr int kWideBins = 512;
constexpr int kWideBits = 9;
// Dynamic shared memory of the wide downsweep: per-warp digit counts, the tile's keys and
// values, the per-digit block-local starts and global shifts.
constexpr size_t kWideSmemBytes =
    sizeof(uint32_t) * ((size_t)kWideWarps * kWideBins + 2 * (size_t)kWideTile + 2 * kWideBins);

__global__ void __launch_bounds__(kWideThreads) wide_upsweep_kernel(const uint32_t* keys,
                                                                    int64_t n_cap,
                                                                    const uint32_t* n_dev,
                                                                    int shift, uint32_t mask,
                                                                    uint32_t* hist,
                                                                    int64_t n_blocks) {
  chain_wait();
  __shared__ uint32_t counts[kWideBins];
  const uint32_t n = read_count(n_dev, n_cap);
  for (int d = threadIdx.x; d < kWideBins; d += kWideThreads) counts[d] = 0;
  __syncthreads();
  // Thread t counts the kWideItems consecutive keys base + t * kWideItems + k (four 16-byte
  // loads; the key arrays are 256-byte aligned and blocks hold whole multiples of 16 keys), one
  // shared-memory add per run of equal digits.
  const int64_t first = (int64_t)blockIdx.x * kWideTile + (int64_t)threadIdx.x * kWideItems;
  if (first < n) {
    uint32_t k[kWideItems];
    if (first + kWideItems <= n) {
      const uint4* p4 = reinterpret_cast<const uint4*>(keys + first);
#pragma unroll
      for (int q = 0; q < kWideItems / 4; ++q) {
        const uint4 v = p4[q];
        k[4 * q] = v.x;
        k[4 * q + 1] = v.y;
        k[4 * q + 2] = v.z;
        k[4 * q + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < kWideItems; ++j) k[j] = first + j < n ? keys[first + j] : 0u;
    }
    const int cnt = (int)min((int64_t)kWideItems, (int64_t)n - first);
    uint32_t run_digit = (k[0] >> shift) & mask, run = 1;
#pragma unroll
    for (int j = 1; j < kWideItems; ++j) {
      if (j >= cnt) break;
      const uint32_t d = (k[j] >> shift) & mask;
      if (d == run_digit) {
        ++run;
      } else {
        atomicAdd(&counts[run_digit], run);
        run_digit = d;
        run = 1;
      }
    }
    atomicAdd(&counts[run_digit], run);
  }
  __syncthreads();
  for (int d = threadIdx.x; d <= (int)mask; d += kWideThreads)
    hist[(int64_t)d * n_blocks + blockIdx.x] = counts[d];
}

__global__ void __launch_bounds__(kWideThreads) wide_row_scan_kernel(uint32_t* hist,
                                                                     int64_t n_blocks) {
  chain_wait();
  const int d = blockIdx.x;
  uint32_t* row = hist + (int64_t)d * n_blocks;
  uint32_t carry = 0;
  for (int64_t base = 0; base < n_blocks; base += kWideThreads * 4) {
    uint32_t v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t idx = base + (int64_t)threadIdx.x * 4 + k;
      v[k] = idx < n_blocks ? row[idx] : 0u;
      s += v[k];
    }
    uint32_t chunk_total;
    uint32_t pre = block_exclusive_scan<kWideThreads>(s, &chunk_total);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t idx = base + (int64_t)threadIdx.x * 4 + k;
      if (idx < n_blocks) row[idx] = carry + pre;
      pre += v[k];
    }
    carry += chunk_total;
  }
  if (threadIdx.x == 0) hist[(int64_t)kWideBins * n_blocks + d] = carry;
}

__global__ void __launch_bounds__(kWideThreads, 2) wide_downsweep_kernel(
    const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
    int64_t n_cap, const uint32_t* n_dev, int shift, uint32_t mask, const uint32_t* hist,
    int64_t n_blocks) {
  chain_wait();
  static_assert(kWideThreads == kWideBins, "one thread per digit in the digit scans");
  extern __shared__ uint32_t wide_smem[];
  uint32_t* warp_counts = wide_smem;                                  // [kWideWarps][kWideBins]
  uint32_t* s_keys = warp_counts + kWideWarps * kWideBins;            // [kWideTile]
  uint32_t* s_vals = s_keys + kWideTile;                              // [kWideTile]
  uint32_t* s_digit_start = s_vals + kWideTile;                       // [kWideBins]
  uint32_t* s_digit_shift = s_digit_start + kWideBins;                // [kWideBins]
  const uint32_t n = read_count(n_dev, n_cap);
  const int64_t base = (int64_t)blockIdx.x * kWideTile;
  if (base >= n) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* wc = warp_counts + warp * kWideBins;
  for (int d = lane; d < kWideBins; d += 32) wc[d] = 0;
  __syncwarp();
  const int64_t wbase = base + (int64_t)warp * 32 * kWideItems;
  uint32_t key[kWideItems], rank[kWideItems];
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int nbits = 32 - __clz(mask);
#pragma unroll
  for (int r = 0; r < kWideItems; ++r) {
    const int64_t idx = wbase + r * 32 + lane;
    key[r] = idx < n ? keys_in[idx] : 0u;
  }
#pragma unroll
  for (int r = 0; r < kWideItems; ++r) {
    const int64_t idx = wbase + r * 32 + lane;
    const bool valid = idx < n;
    const uint32_t digit = valid ? ((key[r] >> shift) & mask) : 0u;
    const uint32_t peers = warp_digit_peers(digit, valid, nbits);
    const uint32_t before = __popc(peers & lt_mask);
    uint32_t prior = 0;
    if (valid) prior = wc[digit];
    __syncwarp();
    if (valid && before == 0) wc[digit] = prior + __popc(peers);
    __syncwarp();
    rank[r] = valid ? prior + before : 0xffffffffu;
  }
  __syncthreads();
  {
    // Thread d: exclusive prefix of digit d over the warps, then the block-local start of the
    // digit's run and its global shift (global position minus local position, mod 2^32).
    const int d = threadIdx.x;
    uint32_t acc = 0;
#pragma unroll
    for (int w = 0; w < kWideWarps; ++w) {
      const uint32_t c = warp_counts[w * kWideBins + d];
      warp_counts[w * kWideBins + d] = acc;
      acc += c;
    }
    const uint32_t local_start = block_exclusive_scan<kWideThreads>(acc, nullptr);
    const uint32_t row_total = d <= (int)mask ? hist[(int64_t)kWideBins * n_blocks + d] : 0u;
    const uint32_t digit_base = block_exclusive_scan<kWideThreads>(row_total, nullptr);
    s_digit_start[d] = local_start;
    s_digit_shift[d] = d <= (int)mask
                           ? digit_base + hist[(int64_t)d * n_blocks + blockIdx.x] - local_start
                           : 0u;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kWideItems; ++r) {
    if (rank[r] == 0xffffffffu) continue;
    const uint32_t digit = (key[r] >> shift) & mask;
    const uint32_t local = s_digit_start[digit] + wc[digit] + rank[r];
    s_keys[local] = key[r];
    if (vals_in) s_vals[local] = vals_in[wbase + r * 32 + lane];
  }
  __syncthreads();
  const int count = (int)min((int64_t)kWideTile, (int64_t)n - base);
  for (int t = threadIdx.x; t < count; t += kWideThreads) {
    const uint32_t k = s_keys[t];
    const uint32_t pos = s_digit_shift[(k >> shift) & mask] + (uint32_t)t;
    keys_out[pos] = k;
    if (vals_out) vals_out[pos] = s_vals[t];
  }
}

// ------------------------------------------------------------------------------------------
// Single-cluster radix sort: the whole sort in one launch of one cluster of C blocks (C = 16,
// else 8), for n <= C * kCsSlice; used for n_cap <= kCsMaxN, where it beats three launches per
// pass. Block c owns the slice [c S, (c + 1) S) of the sequence,
// S = ceil(n / C), held in its shared memory. Per 8-bit pass:
//   (a) stable ranks inside the block (warp w owns a contiguous run of the slice and walks it
//       in rounds of 32 elements, as in the multi-kernel downsweep);
//   (b) per-digit counts of the block, published in its shared memory; local digit starts;
//   (c) local sort of the slice into the second buffer;
//   cluster barrier;
//   (e) every block reads all blocks' digit counts (distributed shared memory): the global start
//       of each digit plus the counts of that digit in the blocks before it;
//   (f) each digit's run is stored, in order, at its global position: into the first buffer of
//       the block that owns that position (distributed shared memory), or to the output array
//       after the last pass;
//   cluster barrier.
// Every block executes every barrier, also when its slice is empty.
// ------------------------------------------------------------------------------------------
constexpr int kCsThreads = 1024;
constexpr int kCsWarps = kCsThreads / 32;
constexpr int kCsItems = 11;
constexpr int kCsSlice = kCsThreads * kCsItems;  // elements per block at most
// Dynamic shared memory: two (key, value) buffers of kCsSlice, the per-warp digit counts, the
// block's digit counts, local digit starts and per-digit destination shifts.
constexpr size_t kCsSmemWords = 4 * (size_t)kCsSlice + (size_t)kCsWarps * kRadixBins + 3 * kRadixBins;
constexpr size_t kCsSmemBytes = kCsSmemWords * sizeof(uint32_t);
// Largest n_cap routed to the single-cluster sort. Measured on GB300 with 16-block clusters, a
// pass costs ~6.3 us plus ~0.09 us per 1k elements (latency of the in-block ranking and the
// exchanges on 16 SMs), the three-kernel pass ~10.5 us at these sizes: the cluster wins below
// ~48k elements (2k: 27 vs 39 us for a 31-bit sort; 36k: 39 vs 43 us; 115k: 71 vs 43 us).
constexpr int64_t kCsMaxN = 56 * 1024;

__global__ void __launch_bounds__(kCsThreads, 1) cluster_sort_kernel(
    const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
    int64_t n_cap, const uint32_t* n_dev, int begin_bit, int end_bit) {
  chain_wait();
  extern __shared__ uint32_t cs_smem[];
  uint32_t* a_keys = cs_smem;
  uint32_t* a_vals = a_keys + kCsSlice;
  uint32_t* b_keys = a_vals + kCsSlice;
  uint32_t* b_vals = b_keys + kCsSlice;
  uint32_t* warp_counts = b_vals + kCsSlice;  // [kCsWarps][kRadixBins]
  uint32_t* cta_counts = warp_counts + kCsWarps * kRadixBins;
  uint32_t* local_start = cta_counts + kRadixBins;
  uint32_t* digit_shift = local_start + kRadixBins;
  cg::cluster_group cluster = cg::this_cluster();
  const uint32_t C = cluster.num_blocks(), me = cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t n = read_count(n_dev, n_cap);
  const uint32_t S = (n + C - 1) / C;
  const uint32_t lo = me * S;
  const uint32_t cnt = n > lo ? min(S, n - lo) : 0u;
  const bool has_vals = vals_in != nullptr;
  for (uint32_t t = tid; t < cnt; t += kCsThreads) {
    a_keys[t] = keys_in[lo + t];
    if (has_vals) a_vals[t] = vals_in[lo + t];
  }
  __syncthreads();
  const int bits = end_bit - begin_bit;
  const int passes = (bits + 7) / 8;
  const int per_pass = (bits + passes - 1) / passes;
  const uint32_t rounds = (cnt + kCsThreads - 1) / kCsThreads;  // rounds of 32 per warp
  const uint32_t wbase = (uint32_t)warp * 32u * rounds;
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t* my_counts = warp_counts + warp * kRadixBins;
  for (int p = 0; p < passes; ++p) {
    const int shift = begin_bit + p * per_pass;
    const int w = (shift + per_pass <= end_bit) ? per_pass : end_bit - shift;
    const uint32_t mask = (w >= 32) ? 0xffffffffu : ((1u << w) - 1u);
    // (a) Stable ranks within the warp's run.
    for (int d = lane; d < kRadixBins; d += 32) my_counts[d] = 0;
    __syncwarp();
    uint32_t key[kCsItems], val[kCsItems], rank[kCsItems];
#pragma unroll
    for (int r = 0; r < kCsItems; ++r) {
      rank[r] = 0xffffffffu;
      key[r] = val[r] = 0u;
      if ((uint32_t)r < rounds) {  // warp-uniform
        const uint32_t e = wbase + (uint32_t)r * 32u + lane;
        const bool valid = e < cnt;
        if (valid) {
          key[r] = a_keys[e];
          if (has_vals) val[r] = a_vals[e];
        }
        const uint32_t digit = valid ? ((key[r] >> shift) & mask) : (uint32_t)kRadixBins;
        const uint32_t peers = warp_digit_peers(digit, valid, w);
        const uint32_t before = __popc(peers & lt_mask);
        const uint32_t prior = valid ? my_counts[digit] : 0u;
        __syncwarp();
        if (valid && before == 0) my_counts[digit] = prior + __popc(peers);
        __syncwarp();
        if (valid) rank[r] = prior + before;
      }
    }
    __syncthreads();
    // (b) Digit d: exclusive prefix over the warps, block total, local start.
    uint32_t total = 0;
    if (tid < kRadixBins) {
      for (int w2 = 0; w2 < kCsWarps; ++w2) {
        const uint32_t c2 = warp_counts[w2 * kRadixBins + tid];
        warp_counts[w2 * kRadixBins + tid] = total;
        total += c2;
      }
    }
    const uint32_t ls = block_exclusive_scan<kCsThreads>(tid < kRadixBins ? total : 0u, nullptr);
    if (tid < kRadixBins) {
      local_start[tid] = ls;
      cta_counts[tid] = total;
    }
    __syncthreads();
    // (c) Local sort into the second buffer.
#pragma unroll
    for (int r = 0; r < kCsItems; ++r) {
      if (rank[r] == 0xffffffffu) continue;
      const uint32_t d = (key[r] >> shift) & mask;
      const uint32_t pos = local_start[d] + my_counts[d] + rank[r];
      b_keys[pos] = key[r];
      b_vals[pos] = val[r];
    }
    cluster.sync();
    // (e) Global start of each digit's run of this block.
    uint32_t all = 0, before_me = 0;
    if (tid < kRadixBins) {
      for (uint32_t r2 = 0; r2 < C; ++r2) {
        const uint32_t v = cluster.map_shared_rank(cta_counts, r2)[tid];
        all += v;
        if (r2 < me) before_me += v;
      }
    }
    const uint32_t gstart = block_exclusive_scan<kCsThreads>(tid < kRadixBins ? all : 0u, nullptr);
    if (tid < kRadixBins) digit_shift[tid] = gstart + before_me - local_start[tid];  // mod 2^32
    __syncthreads();
    // (f) Runs to their global positions.
    const bool last = p == passes - 1;
    for (uint32_t t = tid; t < cnt; t += kCsThreads) {
      const uint32_t k = b_keys[t];
      const uint32_t dest = digit_shift[(k >> shift) & mask] + t;
      if (last) {
        keys_out[dest] = k;
        if (has_vals) vals_out[dest] = b_vals[t];
      } else {
        const uint32_t owner = dest / S;
        const uint32_t off = dest - owner * S;
        cluster.map_shared_rank(a_keys, owner)[off] = k;
        if (has_vals) cluster.map_shared_rank(a_vals, owner)[off] = b_vals[t];
      }
    }
    cluster.sync();
  }
}

}  // namespace

cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n_cap,
                                  const uint32_t* n_dev, uint32_t* total, uint32_t* block_sums,
                                  cudaStream_t stream) {
  return run_scan(PlainLoad{in}, PlainStore{out}, n_cap, n_dev, total, block_sums, stream);
}

cudaError_t launch_exclusive_scan_single_pass(const uint32_t* in, uint32_t* out, int64_t n,
                                              uint32_t* total, Lookback lb, cudaStream_t stream) {
  return run_scan(PlainLoad{in}, PlainStore{out}, n, nullptr, total, nullptr, stream, lb);
}

cudaError_t launch_compact_visible(const uint32_t* vis_bits, int n_views, int n,
                                   const float4* rec2, uint32_t* keys, uint32_t* vals,
                                   uint32_t* list, uint32_t* n_out, Lookback lb,
                                   cudaStream_t stream) {
  const int64_t words = (int64_t)n_views * vis_bit_words_per_view(n);
  if (words == 0) return cudaMemsetAsync(n_out, 0, sizeof(uint32_t), stream);
  const int64_t tiles = (words + kBitsThreads - 1) / kBitsThreads;
  if (tiles > lb.capacity) return cudaErrorInvalidValue;
  const cudaError_t e = launch_chained(
      compact_bits_kernel, dim3((unsigned)tiles), dim3(kBitsThreads), stream, vis_bits,
      (uint32_t)words, (uint32_t)vis_bit_words_per_view(n), (uint32_t)n, rec2, keys, vals, list,
      n_out, lb, (uint32_t)tiles);
  RGS_LAUNCHED();
  return e;
}

cudaError_t launch_gather_scan(const uint32_t* ntiles, const uint32_t* order, int64_t n_cap,
                               const uint32_t* n_dev, uint32_t* offs, uint32_t* total,
                               uint32_t* block_sums, Lookback lb, cudaStream_t stream) {
  return run_scan(GatherLoad{ntiles, order}, PlainStore{offs}, n_cap, n_dev, total, block_sums,
                  stream, lb);
}

// Sorts of at least this many keys (capacity) take the wide passes.
constexpr int64_t kWideMinN = 4 << 20;

cudaError_t radix_sort_wide(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                            int64_t n_cap, const uint32_t* n_dev, int begin_bit, int end_bit,
                            uint32_t* hist, bool* result_in_alt, cudaStream_t stream) {
  *result_in_alt = false;
  const int64_t nb = (n_cap + kWideTile - 1) / kWideTile;
  if (nb == 0 || end_bit <= begin_bit) return cudaSuccess;
  {
    // The kernel's dynamic shared memory limit is raised once per device, before its first use.
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t ea = cudaGetDevice(&dev);
    if (ea != cudaSuccess) return ea;
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64 || !done[dev]) {
      ea = cudaFuncSetAttribute(wide_downsweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kWideSmemBytes);
      if (ea != cudaSuccess) return ea;
      if (dev >= 0 && dev < 64) done[dev] = true;
    }
  }
  const int bits = end_bit - begin_bit;
  const int passes = (bits + kWideBits - 1) / kWideBits;
  const int per_pass = (bits + passes - 1) / passes;
  uint32_t *kin = keys, *vin = vals, *kout = keys_alt, *vout = vals ? vals_alt : nullptr;
  for (int p = 0; p < passes; ++p) {
    const int shift = begin_bit + p * per_pass;
    const int w = (shift + per_pass <= end_bit) ? per_pass : end_bit - shift;
    const uint32_t mask = (1u << w) - 1u;
    cudaError_t e = launch_chained(wide_upsweep_kernel, dim3((unsigned)nb), dim3(kWideThreads),
                                   stream, (const uint32_t*)kin, n_cap, n_dev, shift, mask, hist,
                                   nb);
    RGS_LAUNCHED();
    if (e == cudaSuccess)
      e = launch_chained(wide_row_scan_kernel, dim3(mask + 1), dim3(kWideThreads), stream, hist,
                         nb);
    RGS_LAUNCHED();
    if (e == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)nb);
      cfg.blockDim = dim3(kWideThreads);
      cfg.dynamicSmemBytes = kWideSmemBytes;
      cfg.stream = stream;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, wide_downsweep_kernel, (const uint32_t*)kin,
                             (const uint32_t*)vin, kout, vout, n_cap, n_dev, shift, mask,
                             (const uint32_t*)hist, nb);
    }
    RGS_LAUNCHED();
    if (e != cudaSuccess) return e;
    uint32_t* t = kin;
    kin = kout;
    kout = t;
    t = vin;
    vin = vout;
    vout = t;
    *result_in_alt = !*result_in_alt;
  }
  return cudaGetLastError();
}

template <int ITEMS>
cudaError_t radix_sort_t(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                         int64_t n_cap, const uint32_t* n_dev, int begin_bit, int end_bit,
                         uint32_t* hist, bool* result_in_alt, cudaStream_t stream) {
  *result_in_alt = false;
  const int64_t nb = sort_blocks(n_cap, ITEMS);
  if (nb == 0 || end_bit <= begin_bit) return cudaSuccess;
  const int bits = end_bit - begin_bit;
  const int passes = (bits + 7) / 8;
  const int per_pass = (bits + passes - 1) / passes;
  uint32_t *kin = keys, *vin = vals, *kout = keys_alt, *vout = vals ? vals_alt : nullptr;
  for (int p = 0; p < passes; ++p) {
    const int shift = begin_bit + p * per_pass;
    const int w = (shift + per_pass <= end_bit) ? per_pass : end_bit - shift;
    const uint32_t mask = (w >= 32) ? 0xffffffffu : ((1u << w) - 1u);
    cudaError_t e = launch_chained(radix_upsweep_kernel<ITEMS>, dim3((unsigned)nb),
                                   dim3(kSortThreads), stream, (const uint32_t*)kin, n_cap, n_dev,
                                   shift, mask, hist, nb);
    RGS_LAUNCHED();
    if (e == cudaSuccess)
      e = launch_chained(radix_row_scan_kernel, dim3(kRadixBins), dim3(kSortThreads), stream,
                         hist, nb);
    RGS_LAUNCHED();
    if (e == cudaSuccess)
      e = launch_chained(radix_downsweep_kernel<ITEMS>, dim3((unsigned)nb), dim3(kSortThreads),
                         stream, (const uint32_t*)kin, (const uint32_t*)vin, kout, vout, n_cap,
                         n_dev, shift, mask, (const uint32_t*)hist, nb);
    RGS_LAUNCHED();
    if (e != cudaSuccess) return e;
    uint32_t* t = kin;
    kin = kout;
    kout = t;
    t = vin;
    vin = vout;
    vout = t;
    *result_in_alt = !*result_in_alt;
  }
  return cudaGetLastError();
}

int cluster_sort_blocks(int device) {
  // Per device: 16 blocks per cluster if one such cluster fits on the GPU, else 8, else 0.
  static std::mutex mu;
  static int cached[64];
  static bool known[64] = {};
  if (device < 0 || device >= 64) return 0;
  std::lock_guard<std::mutex> lock(mu);
  if (known[device]) return cached[device];
  int result = 0;
  int prev = 0;
  if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(device) == cudaSuccess &&
      cudaFuncSetAttribute(cluster_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kCsSmemBytes) == cudaSuccess &&
      cudaFuncSetAttribute(cluster_sort_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed,
                           1) == cudaSuccess) {
    for (const int c : {16, 8}) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(c);
      cfg.blockDim = dim3(kCsThreads);
      cfg.dynamicSmemBytes = kCsSmemBytes;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = c;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, cluster_sort_kernel, &cfg) == cudaSuccess &&
          clusters > 0) {
        result = c;
        break;
      }
    }
  }
  cudaGetLastError();  // a refused query leaves no sticky error: fall back to the multi-kernel sort
  cudaSetDevice(prev);
  cached[device] = result;
  known[device] = true;
  return result;
}

int64_t cluster_sort_capacity(int device) {
  return std::min<int64_t>((int64_t)cluster_sort_blocks(device) * kCsSlice, kCsMaxN);
}

cudaError_t launch_radix_sort(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                              uint32_t* vals_alt, int64_t n_cap, const uint32_t* n_dev,
                              int begin_bit, int end_bit, uint32_t* hist, uint32_t* block_sums,
                              bool* result_in_alt, cudaStream_t stream, int items) {
  (void)block_sums;
  int device = 0;
  if (n_cap > 0 && end_bit > begin_bit && cudaGetDevice(&device) == cudaSuccess) {
    const int blocks = cluster_sort_blocks(device);
    if (blocks > 0 && n_cap <= std::min<int64_t>((int64_t)blocks * kCsSlice, kCsMaxN)) {
      // One launch: (keys, vals) -> (keys_alt, vals_alt).
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(blocks);
      cfg.blockDim = dim3(kCsThreads);
      cfg.dynamicSmemBytes = kCsSmemBytes;
      cfg.stream = stream;
      cudaLaunchAttribute attr[2];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = blocks;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[1].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 2;
      const cudaError_t e = cudaLaunchKernelEx(&cfg, cluster_sort_kernel, (const uint32_t*)keys,
                                               (const uint32_t*)vals, keys_alt,
                                               vals ? vals_alt : nullptr, n_cap, n_dev,
                                               begin_bit, end_bit);
      RGS_LAUNCHED();
      *result_in_alt = true;
      return e;
    }
  }
  // The wide upsweep reads keys with 16-byte loads: both key buffers must be 16-byte aligned.
  const bool aligned16 = reinterpret_cast<uintptr_t>(keys) % 16 == 0 &&
                         reinterpret_cast<uintptr_t>(keys_alt) % 16 == 0;
  if (n_cap >= kWideMinN && items == kSortItems && aligned16)
    return radix_sort_wide(keys, vals, keys_alt, vals_alt, n_cap, n_dev, begin_bit, end_bit, hist,
                           result_in_alt, stream);
  if (items == kSortItemsSmall)
    return radix_sort_t<kSortItemsSmall>(keys, vals, keys_alt, vals_alt, n_cap, n_dev, begin_bit,
                                         end_bit, hist, result_in_alt, stream);
  return radix_sort_t<kSortItems>(keys, vals, keys_alt, vals_alt, n_cap, n_dev, begin_bit,
                                  end_bit, hist, result_in_alt, stream);
}

}  // namespace rgs
