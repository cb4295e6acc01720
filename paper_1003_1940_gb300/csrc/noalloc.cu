// noalloc.cu -- dbg_rle_u64_noalloc: the run-length reduce of sorted 64-bit
// keys with no memory allocation at all, for callers that cannot allocate
// device memory themselves or let a library do it (see include/dbg.h).
//
// The reduce is k_rle, a single pass with decoupled look-back.  dbg_build
// does not launch it: the build counts each key's copies inside the local
// pass of its hybrid sort (or, with every digit sorted globally, reduces by
// a counting pass, a scan and a writing pass), which yields the same
// distinct keys and multiplicities; the test of this entry point checks it
// against dbg_build's edges.  k_rle's scratch -- the per-tile look-back
// status words, the tile ticket, the unique-key total and the device error
// word -- lives in one file-scope __device__ array instead of memory from an
// allocator.
#include <mutex>

#include "k_build.cuh"

namespace dbg {
namespace {

// Largest input of one call.  With SCAN_TILE keys per tile the status words
// need MAX_KEYS / SCAN_TILE entries.
constexpr uint64_t kNoAllocMaxKeys = 1ull << 26;
constexpr uint64_t kNoAllocTiles = kNoAllocMaxKeys / SCAN_TILE;
// layout (64-bit words): [0, tiles) status words, then ticket/total/error
constexpr uint64_t kNoAllocWords = kNoAllocTiles + 8;

static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
uint64_t *g_scratch_addr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// Device address of the scratch array on `dev` (host code cannot use the
// array's name as a device pointer).  Looked up once per device.
dbg_status scratch_address(int dev, uint64_t **out) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d outside [0, %d)", dev, kMaxDevices);
    return DBG_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      set_error("cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return DBG_ECUDA;
    }
    g_scratch_addr[dev] = static_cast<uint64_t *>(p);
  }
  *out = g_scratch_addr[dev];
  return DBG_OK;
}

}  // namespace
}  // namespace dbg

using namespace dbg;

extern "C" dbg_status dbg_rle_u64_noalloc(const uint64_t *keys, uint64_t n, uint64_t *uniq, uint32_t *run_start,
                                          uint64_t *count, void *stream) {
  if (!count || !run_start || (n > 0 && (!keys || !uniq))) {
    set_error("dbg_rle_u64_noalloc: NULL argument");
    return DBG_EINVAL;
  }
  if (n > kNoAllocMaxKeys) {
    set_error("dbg_rle_u64_noalloc: n = %llu exceeds the maximum of %llu keys", (unsigned long long)n,
              (unsigned long long)kNoAllocMaxKeys);
    return DBG_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  DBG_CUDA_TRY(cudaGetDevice(&dev));
  uint64_t *scratch = nullptr;
  DBG_TRY(scratch_address(dev, &scratch));
  uint64_t *status = scratch;
  uint32_t *small = reinterpret_cast<uint32_t *>(scratch + kNoAllocTiles);  // ticket, total, err
  if (n == 0) {
    // run_start holds n + 1 = 1 entry: the end of the (empty) input
    DBG_CUDA_TRY(cudaMemsetAsync(run_start, 0, sizeof(uint32_t), s));
    DBG_CUDA_TRY(cudaStreamSynchronize(s));
    *count = 0;
    return DBG_OK;
  }
  const uint64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  // the array keeps the previous call's words: clear what this call reads
  DBG_CUDA_TRY(cudaMemsetAsync(status, 0, tiles * sizeof(uint64_t), s));
  DBG_CUDA_TRY(cudaMemsetAsync(small, 0, 4 * sizeof(uint32_t), s));
  k_rle<uint64_t><<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(keys, n, uniq, run_start, status, small, 1u, 1u << 22,
                                                        small + 2, small + 1);
  DBG_CUDA_TRY(cudaGetLastError());
  uint32_t host[2] = {0, 0};
  DBG_CUDA_TRY(cudaMemcpyAsync(host, small + 1, sizeof(host), cudaMemcpyDeviceToHost, s));
  DBG_CUDA_TRY(cudaStreamSynchronize(s));
  if (host[1] != 0) {
    set_error("dbg_rle_u64_noalloc: a device-side wait reached its spin limit");
    return DBG_ETIMEOUT;
  }
  *count = host[0];
  return DBG_OK;
}
