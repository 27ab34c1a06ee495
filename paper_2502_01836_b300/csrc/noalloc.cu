// leafi_leaf_lower_bounds_noalloc: the leaf lower bounds without any device
// allocation, for callers that must not call cudaMalloc: a host program whose
// GPU memory is reserved up front by another allocator (a framework's caching
// pool that owns the device), or a latency-critical loop that cannot accept
// cudaMalloc's implicit device-wide synchronisation on its path.
//
// The bound kernels need scratch memory (float64 prefix sums of the queries,
// per-interval query statistics, per-node bounds).  Here that scratch is a
// file-scope __device__ array of kNoAllocScratchBytes; every GPU that loads the
// library holds it until the process exits.  Host code cannot use the array's
// name as a device address, so the first call on each device looks the
// address up with cudaGetSymbolAddress (with that device current) and caches
// it; make that first call before any stream capture.  All calls share the
// array: calls that overlap on the GPU (other streams, other threads) race on
// it.  Every scratch byte the kernels read is written earlier in the same
// call, so nothing has to be cleared between calls.
#include <mutex>

#include "internal.h"

namespace leafi {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// device address of the scratch array on `dev` (which must be current)
unsigned char* scratch_on(int dev) {
  if (dev < 0 || dev >= kMaxDevices) fail(LEAFI_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      fail(LEAFI_ECUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
           cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  return static_cast<unsigned char*>(g_scratch_addr[dev]);
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// true iff p is device (or managed) memory of GPU `dev`: the kernels read and
// write it in place, so memory of another GPU is refused rather than reached
// through peer access (or faulting without it)
bool is_device_pointer_on(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace
}  // namespace leafi

using namespace leafi;

extern "C" leafi_status leafi_leaf_lower_bounds_noalloc(leafi_index* index, const float* queries,
                                                        int64_t nq, double* lb2) {
  try {
    if (!index) fail(LEAFI_EINVAL, "index is NULL");
    if (index->device < 0) fail(LEAFI_EINVAL, "index was built host-only (device -1)");
    if (nq < 0) fail(LEAFI_EINVAL, "nq < 0");
    if (nq == 0) return LEAFI_OK;
    if (!queries || !lb2) fail(LEAFI_EINVAL, "queries / lb2 is NULL");
    // every query needs at least 16 bytes of prefix sums, so this bound keeps
    // the size arithmetic below far from overflow and nq within int range
    if ((uint64_t)nq > kNoAllocScratchBytes / 16)
      fail(LEAFI_EINVAL, "nq = %lld exceeds the no-allocation scratch (%zu bytes)",
           (long long)nq, kNoAllocScratchBytes);
    std::lock_guard<std::mutex> lk(index->mu);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != index->device) LF_CUDA(cudaSetDevice(index->device));
    struct Restore {
      int dev;
      ~Restore() {
        if (dev >= 0) cudaSetDevice(dev);
      }
    } restore{prev != index->device ? prev : -1};
    if (!is_device_pointer_on(queries, index->device) ||
        !is_device_pointer_on(lb2, index->device))
      fail(LEAFI_EINVAL,
           "queries and lb2 must be device arrays on the index's GPU %d (nothing is staged)",
           index->device);
    if (reinterpret_cast<uintptr_t>(queries) % 4 || reinterpret_cast<uintptr_t>(lb2) % 8)
      fail(LEAFI_EINVAL, "misaligned queries / lb2");
    const HostTree& t = index->tree;
    const int m = index->m;
    // scratch layout: prefix sums, then the tree-specific statistics
    const size_t bP = align256(sizeof(double) * (size_t)nq * 2 * (m + 1));
    size_t need = bP;
    size_t bA = 0, bB = 0;
    if (t.type == LEAFI_DSTREE) {
      bA = align256(sizeof(double) * ds_ivstat_doubles(nq, t.iv_s.size()));
      bB = align256(sizeof(double) * (size_t)nq * t.n_nodes);
    } else {
      bA = align256(sizeof(double) * isax_paa_doubles(nq, t.w));
    }
    need += bA + bB;
    if (need > kNoAllocScratchBytes)
      fail(LEAFI_EINVAL,
           "nq = %lld needs %zu bytes of scratch; the no-allocation path holds %zu bytes "
           "(at most %lld queries for this index)",
           (long long)nq, need, kNoAllocScratchBytes,
           (long long)((double)kNoAllocScratchBytes / ((double)need / (double)nq)));
    unsigned char* base = scratch_on(index->device);
    double* P = reinterpret_cast<double*>(base);
    double* A = reinterpret_cast<double*>(base + bP);
    double* B = reinterpret_cast<double*>(base + bP + bA);
    // queries are read in place with their own row stride m
    launch_prefix(queries, (int)nq, m, m, P, index->stream);
    if (t.type == LEAFI_DSTREE)
      launch_ds_bounds(index->ds(), P, (int)nq, m, A, B, lb2, nullptr, index->stream);
    else
      launch_isax_bounds(index->isax(), P, (int)nq, m, A, lb2, nullptr, index->stream);
    return LEAFI_OK;
  } catch (const Failure& e) {
    set_last_error(e.msg);
    return e.status;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return LEAFI_EINTERNAL;
  }
}
