// noalloc.cu -- sstep_block_gram_noalloc: the block Gram products of sstep_block_gram for
// callers that cannot allocate device memory when they call us.
//
// sstep_block_gram needs scratch for its per-CTA partial sums and its completion ticket and
// obtains it with cudaMallocAsync on every call.  Some callers cannot do that: programs whose
// framework has already reserved the device's memory in its own pool (an extra allocation
// fails or fragments that pool), and latency-sensitive callers that must not pay for the
// allocator or let a free wait on the device.  This variant uses one fixed scratch area that
// lives in the library image instead: a file-scope __device__ array of kScratchBytes
// (about 1.06 MB), present on every GPU that loads the library until the process exits.
//
// Limits: ne <= kNoAllocMaxEntries (256) products per call, and devices with at most
// kNoAllocMaxCtas / 2 SMs (the Gram grid is two CTAs per SM of the current device).  All calls
// share the one array and it keeps the previous call's contents, so each call first zeroes the
// ticket and flags it relies on.  Calls that run concurrently on the GPU (on different streams,
// or from different threads without ordering) race on the array and give wrong sums; order
// them.
//
// Set-up: the first call on a device, with that device current, looks up the array's device
// address (cudaGetSymbolAddress) and keeps it for later calls on that device ordinal; make that
// first call before any stream capture.  The address belongs to the device's primary context:
// after cudaDeviceReset on a device the kept address is stale, so do not call this entry point
// on that device again in the same process.
#include <mutex>
#include <string>

#include "common.cuh"

using namespace sstep;

namespace {

constexpr int kNoAllocMaxEntries = 256;
constexpr int kNoAllocMaxCtas = 512;
constexpr int kMaxDevices = 64;
constexpr size_t kCtrlBytes = (sizeof(Ctrl) + 255) / 256 * 256;
constexpr size_t kScratchBytes =
    kCtrlBytes + sizeof(double) * (size_t)kNoAllocMaxCtas * kNoAllocMaxEntries;

// The scratch: control block (ticket, flags, sums) followed by the partial-sum table.
static __device__ __align__(256) unsigned char g_gram_scratch[kScratchBytes];

std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device.  In host code the array's name is only
// a host-side stand-in, so the address is looked up once per device, with that device current,
// and kept per device ordinal.
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_gram_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

sstep_status fail(sstep_status st, const std::string& msg) {
  set_last_error(msg.c_str());  // reported by sstep_last_error()
  return st;
}

}  // namespace

extern "C" SSTEP_API sstep_status sstep_block_gram_noalloc(int64_t n, int nl, const double* const* L,
                                                 int nr, const double* const* R, int ne,
                                                 const int* pairs, double* out, void* stream) {
  if (n < 1 || nl < 1 || nr < 1 || nl > kMaxGramVecs || nr > kMaxGramVecs || ne < 1 || !L || !R ||
      !pairs || !out)
    return fail(SSTEP_ERR_INVALID, "bad block_gram_noalloc arguments");
  if (ne > kNoAllocMaxEntries)
    return fail(SSTEP_ERR_INVALID, "block_gram_noalloc: at most 256 products per call (ne = " +
                                       std::to_string(ne) + ")");
  // the grid launch_gram uses on the current device must fit the partial-sum table
  if (gram_ctas() > kNoAllocMaxCtas)
    return fail(SSTEP_ERR_UNSUPPORTED, "block_gram_noalloc: the device has more SMs than the "
                                       "fixed scratch area serves (at most 256)");
  GramArgs g{};
  g.n = n;
  g.nl = nl;
  g.nr = nr;
  g.ne = ne;
  for (int i = 0; i < nl; ++i) g.L[i] = L[i];
  for (int i = 0; i < nr; ++i) g.R[i] = R[i];
  for (int e = 0; e < ne; ++e) {
    if (pairs[2 * e] < 0 || pairs[2 * e] >= nl || pairs[2 * e + 1] < 0 || pairs[2 * e + 1] >= nr)
      return fail(SSTEP_ERR_INVALID, "block_gram_noalloc: pair index out of range");
    g.pairs[e] = (unsigned short)((pairs[2 * e] << 8) | pairs[2 * e + 1]);
  }
  g.mode = GM_SUMS;
  g.out = out;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(SSTEP_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(SSTEP_ERR_UNSUPPORTED, "device ordinal >= 64");
  void* base = nullptr;
  e = scratch_address(dev, &base);
  if (e != cudaSuccess)
    return fail(SSTEP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  e = gram_init();  // sets a kernel attribute; allocates nothing
  if (e != cudaSuccess) return fail(SSTEP_ERR_CUDA, cudaGetErrorString(e));
  cudaStream_t st = (cudaStream_t)stream;
  Ctrl* ctrl = (Ctrl*)base;
  // The ticket and the early-exit flag must start at zero; the array holds the last call's data.
  e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st);
  if (e != cudaSuccess) return fail(SSTEP_ERR_CUDA, cudaGetErrorString(e));
  g.ctrl = ctrl;
  g.partials = (double*)((unsigned char*)base + kCtrlBytes);
  e = launch_gram(g, st);
  if (e != cudaSuccess) return fail(SSTEP_ERR_CUDA, cudaGetErrorString(e));
  set_last_error("");
  return SSTEP_OK;
}
