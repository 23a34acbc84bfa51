// static_scan.cu -- rgs_exclusive_scan_u32_static: the exclusive scan of rgs_exclusive_scan_u32
// with its scratch in a fixed device array of this file instead of memory from cudaMalloc.
//
// Some callers cannot allocate device memory at call time: a real-time tracking loop that must
// not block on the driver's allocator in the middle of a frame, or a process whose device
// memory is already reserved in full by another framework's caching allocator. This entry point
// serves them: it runs the same three scan kernels, and the only scratch it needs (one partial
// sum per 4096-element block) lives in `g_scan_block_sums` below, which every GPU that loads the
// library holds (64 KiB) until the process exits.
#include "rgs_internal.cuh"

namespace {

constexpr int64_t kStaticScanMax = RGS_STATIC_SCAN_MAX_N;
constexpr int64_t kStaticScanBlocks = (kStaticScanMax + rgs::kScanTile - 1) / rgs::kScanTile;

// Per-block partial sums of the scan (one u32 per 4096 elements, plus the grand-total slot).
// Shared by every call on a device; each call overwrites what it reads, so nothing needs to be
// cleared between calls.
static __device__ __align__(256) uint32_t g_scan_block_sums[kStaticScanBlocks + 1];

// Device address of the scratch array in the current context. In host code `g_scan_block_sums`
// names a host-side stand-in, never the device memory itself. The lookup is repeated on every
// call (it is a cheap table lookup once the module is loaded), so a reset device or another
// current context never sees a stale address.
cudaError_t scratch_on_current_device(uint32_t** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_scan_block_sums);
  if (e != cudaSuccess) return e;
  *out = static_cast<uint32_t*>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" rgs_status rgs_exclusive_scan_u32_static(const uint32_t* in, uint32_t* out, int64_t n,
                                                    uint32_t* total_out, void* stream) {
  if (n < 0 || (n > 0 && (!in || !out))) return RGS_ERR_INVALID_ARG;
  if (n > kStaticScanMax) return RGS_ERR_TOO_LARGE;
  uint32_t* scratch = nullptr;
  if (scratch_on_current_device(&scratch) != cudaSuccess) return RGS_ERR_CUDA;
  const cudaError_t e = rgs::launch_exclusive_scan(in, out, n, nullptr, total_out, scratch,
                                                   static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? RGS_OK : RGS_ERR_CUDA;
}
