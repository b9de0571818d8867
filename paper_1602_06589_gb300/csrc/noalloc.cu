// noalloc.cu -- hsgen_coefficients_noalloc: the A/B coefficient step with no
// device allocation at all.
//
// Why it exists: hsgen_coefficients takes its scratch (the per-species radial
// factors) from a workspace that the library grows with cudaMalloc on first
// use. Some callers cannot let a library do that: code that runs under
// another framework's memory manager (which has already reserved the GPU's
// memory, so a cudaMalloc from here may fail), and latency-critical loops in
// which cudaMalloc's implicit device synchronisation is not acceptable. This
// entry point takes its scratch from a fixed array in device memory that is
// part of the loaded library instead.
//
// The array below is allocated by the CUDA runtime when the library's device
// code is loaded into a context on a device (with the runtime's default lazy
// loading that happens at the first call of this entry point on that device,
// not when the library is loaded into the process) and stays there until the
// context ends, normally at process exit, on every GPU that uses it. Host code
// cannot use its name as a device address (on the host the name is only a
// stand-in), so the device address is fetched with cudaGetSymbolAddress, with
// that device current, during the first call on that device, and again after
// the device's context has been replaced (for example by cudaDeviceReset).
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace hsg {

// 16 MiB: radial factors for n_types * n_g <= 95325 species-plane-wave pairs.
constexpr size_t kNoallocScratchBytes = 16u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};  // context the address belongs to

// Device address of the scratch array on `device`, which must be current
// (looked up on first use, and again when the device's context changed).
cudaError_t scratch_address(int device, void **out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  // the driver's context calls, fetched at run time (the library does not
  // link the driver library itself)
  typedef CUresult (*GetCurrentFn)(CUcontext *);
  typedef CUresult (*GetIdFn)(CUcontext, unsigned long long *);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  cudaError_t e = cudaSuccess;
  if (!get_current || !get_id) {
    void *p1 = nullptr, *p2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p1, 12000, cudaEnableDefault, &q1);
    if (e != cudaSuccess || q1 != cudaDriverEntryPointSuccess) return e != cudaSuccess ? e : cudaErrorNotSupported;
    e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &p2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess || q2 != cudaDriverEntryPointSuccess) return e != cudaSuccess ? e : cudaErrorNotSupported;
    get_current = (GetCurrentFn)p1;
    get_id = (GetIdFn)p2;
  }
  // cudaSetDevice (called before this) has made the device's primary context current
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  if (!g_scratch_addr[device] || g_scratch_ctx[device] != id) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = p;
    g_scratch_ctx[device] = id;
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}
}  // namespace

}  // namespace hsg

using namespace hsg;

extern "C" hsgen_status hsgen_coefficients_noalloc(hsgen_ctx *ctx, int n_g, const double *kvec, void *W,
                                                   long long ldw, void *cuda_stream) {
  if (!ctx) return HSGEN_EINVAL;
  if (!ctx->have_system) return set_err(ctx, HSGEN_EINVAL, "coefficients_noalloc: no system set");
  if (n_g < 0 || !kvec || !W) return set_err(ctx, HSGEN_EINVAL, "coefficients_noalloc: bad argument");
  if (ldw < ctx->depth) return set_err(ctx, HSGEN_EINVAL, "coefficients_noalloc: ldw < depth");
  if (n_g == 0) return HSGEN_OK;
  const int nt = (int)ctx->types.size();
  const size_t need = sizeof(double2) * (size_t)nt * (size_t)n_g * kRadStride;
  if (need > kNoallocScratchBytes)
    return set_err(ctx, HSGEN_EINVAL,
                   "coefficients_noalloc: n_types * n_g = " + std::to_string((long long)nt * n_g) +
                       " exceeds the fixed scratch (16 MiB: n_types * n_g <= " +
                       std::to_string(kNoallocScratchBytes / (sizeof(double2) * kRadStride)) + ")");
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, kvec) != cudaSuccess ||
      !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) {
    cudaGetLastError();
    return set_err(ctx, HSGEN_EINVAL, "coefficients_noalloc: kvec must be a device pointer");
  }
  if (cudaPointerGetAttributes(&a, W) != cudaSuccess ||
      !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) {
    cudaGetLastError();
    return set_err(ctx, HSGEN_EINVAL, "coefficients_noalloc: W must be a device pointer");
  }
  if (on_other_device(kvec, ctx->device) || on_other_device(W, ctx->device))
    return set_err(ctx, HSGEN_EINVAL, "coefficients_noalloc: kvec or W lives on another GPU than the context's");
  HSG_CUDA(ctx, cudaSetDevice(ctx->device));
  void *scratch = nullptr;
  HSG_CUDA(ctx, scratch_address(ctx->device, &scratch));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // Every factor that the coefficient kernel reads is written by the radial
  // kernel earlier in this call, so nothing left by an earlier call is read
  // and nothing needs clearing.
  double2 *F = (double2 *)scratch;
  ctx->launches = 0;
  HSG_LAUNCH(ctx, launch_radial(n_g, kvec, nt, ctx->d_radial, F, s));
  for (int t = 0; t < nt; ++t) {
    int n = (int)ctx->atoms_of_type[t].size();
    if (!n) continue;
    HSG_LAUNCH(ctx, launch_coefficients(ctx->types[t].lc, n_g, kvec, F + (size_t)t * n_g * kRadStride,
                                        ctx->d_atoms_by_type + ctx->atoms_by_type_start[t], n, ctx->d_pos,
                                        ctx->d_rot, ctx->d_off, 0, ctx->types[t].dpad, (double2 *)W, ldw, s));
  }
  return HSGEN_OK;
}
