// pf_noalloc.cu -- pf_resample_noalloc: the per-group systematic resampler
// of pf_resample, with its scratch memory in a fixed device array instead of
// a workspace the caller allocates.
//
// It exists for callers that cannot allocate device memory when they need
// to resample: code that runs under a fixed memory budget reserved up front,
// code inside a framework whose caching allocator must not be bypassed, and
// latency-critical loops where cudaMalloc's implicit device synchronisation
// is not acceptable.  Such a caller still provides the inputs and outputs.
//
// The scratch (an error word, the group table and the group state, about
// 96 KB) is the file-scope array g_scratch.  Every GPU that loads this
// library holds it until the process exits.  On the host the name g_scratch
// is only a host-side stand-in, not a device address; host code never hands
// it to a kernel.  The device address is looked up with cudaGetSymbolAddress
// on the first call made on each device (with that device current), checked,
// and cached; that first call should therefore come before any stream
// capture.  The cache remembers the CUDA context it was taken in: after
// cudaDeviceReset (or any other end of the device's primary context) the
// next call sees a new context and looks the address up again.  All calls
// share the one array and it keeps the last call's contents: each call
// clears the error word and rewrites the group table before the resampler
// reads them, and calls that overlap on the GPU (on different streams
// without ordering) race on it.  The resampler's device-side error word
// stays in the array until the next call clears it; pf_resample_check(NULL,
// stream) reads it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/pfarna.h"
#include "pf_device.cuh"
#include "pf_launch.h"

using namespace pf;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kOffDesc = align_up(sizeof(DevState));
constexpr size_t kOffState = kOffDesc + align_up(sizeof(GroupDesc) * PF_NOALLOC_MAX_GROUPS);
constexpr size_t kScratchBytes = kOffState + align_up(sizeof(GroupState) * PF_NOALLOC_MAX_GROUPS);

// The scratch every call shares.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_dev_ptr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};  // context the cached address belongs to
std::mutex g_mutex;

// Unique id of the calling thread's current CUDA context (0 if none or if
// the driver does not say), through the runtime's driver entry points.
unsigned long long current_context_id() {
  typedef CUresult (*get_current_t)(CUcontext*);
  typedef CUresult (*get_id_t)(CUcontext, unsigned long long*);
  static get_current_t get_current = nullptr;
  static get_id_t get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (get_current_t)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (get_id_t)f;
    resolved = true;
  }
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c != nullptr && get_id(c, &id) == CUDA_SUCCESS)
    return id;
  return 0;
}

pf_status fail(pf_status st, const std::string& msg) {
  set_handleless_error(msg.c_str());
  return st;
}

// The group table of G equal groups of Np particles, written on the device.
__global__ void k_noalloc_groups(GroupDesc* gd, int G, int Np) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    GroupDesc d{};
    d.base = (long long)g * Np;
    d.Np = Np;
    d.g = g;
    gd[g] = d;
  }
}

// Device address of g_scratch on the current device, looked up once.
pf_status scratch_on_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(PF_ERR_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mutex);
  const unsigned long long ctx = current_context_id();
  if (g_dev_ptr[dev] == nullptr || ctx == 0 || ctx != g_ctx_id[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(PF_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_dev_ptr[dev] = p;
    g_ctx_id[dev] = current_context_id();  // the lookup made the device's context current
  }
  *out = static_cast<unsigned char*>(g_dev_ptr[dev]);
  return PF_OK;
}

}  // namespace

namespace pf {
int noalloc_error_word(const DevState** out) {
  unsigned char* base = nullptr;
  const pf_status st = scratch_on_current_device(&base);
  if (st != PF_OK) return st;
  *out = reinterpret_cast<const DevState*>(base);
  return PF_OK;
}
}  // namespace pf

extern "C" pf_status pf_resample_noalloc(const float* logw, const uint32_t* u, int32_t G, int32_t Np, uint32_t* anc,
                                         uint64_t* q, void* stream) {
  if (!logw || !u || !anc) return fail(PF_ERR_ARG, "pf_resample_noalloc: NULL pointer");
  if (G < 1 || G > PF_NOALLOC_MAX_GROUPS)
    return fail(PF_ERR_ARG, "pf_resample_noalloc: G must be in [1, " + std::to_string(PF_NOALLOC_MAX_GROUPS) +
                                "] (the size of its fixed scratch)");
  if (Np < 1 || Np > (1 << 20) || (long long)G * Np >= (1ll << 31))
    return fail(PF_ERR_ARG, "pf_resample_noalloc: Np must be in [1, 2^20] and G*Np < 2^31");
  unsigned char* base = nullptr;
  const pf_status st = scratch_on_current_device(&base);
  if (st != PF_OK) return st;
  DevState* ds = reinterpret_cast<DevState*>(base);
  GroupDesc* gd = reinterpret_cast<GroupDesc*>(base + kOffDesc);
  GroupState* gs = reinterpret_cast<GroupState*>(base + kOffState);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the error word must start at zero; the group table is rewritten in full
  cudaError_t e = cudaMemsetAsync(ds, 0, sizeof(DevState), s);
  if (e != cudaSuccess) return fail(PF_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  k_noalloc_groups<<<(G + 255) / 256, 256, 0, s>>>(gd, G, Np);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return fail(PF_ERR_CUDA, std::string("k_noalloc_groups: ") + cudaGetErrorString(e));
  ResampleArgs ra{gd, gs, nullptr, logw, nullptr, anc, 0, reinterpret_cast<unsigned long long*>(q), u, 1,
                  resample_coeffs(), ds};
  ra.n_groups = G;
  ra.max_np = Np;
  ra.lean = q ? 0 : 1;  // without codes to store, the lean instance when the chunks fit
  if ((e = launch_resample(ra, G, resample_cluster_size(Np), false, s)) != cudaSuccess)
    return fail(PF_ERR_CUDA, std::string("k_resample: ") + cudaGetErrorString(e));
  return PF_OK;
}
