// noalloc.cu -- D^dag D for one lattice without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside a host
// framework which owns every byte of device memory through its own pool, code
// that must not trigger the device-wide synchronisation that cudaMalloc and
// cudaFree can imply (for example between the launches of a latency-critical
// loop), or plugins that are not allowed to create allocations of their own.
// sm_apply_DdagD needs a workspace (for t = D in) and a lattice object, and
// sm_lattice_create allocates the geometry tables.  The entry point below
// takes the geometry of a single L x T lattice by value and keeps t in a
// file-scope device array, so it allocates nothing.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace sm {

// Scratch for t = D in: 8 MiB, i.e. 262144 sites in FP64 (32 B/site) or
// 524288 sites in FP32 (16 B/site).  Every GPU that loads this library holds
// it until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
// The array's device address, per device, with the unique id of the context
// it was looked up in.  After cudaDeviceReset (or any other teardown of the
// primary context) the library's module is loaded again in a new context and
// the array gets a new address: the id no longer matches and the address is
// looked up again.
struct ScratchAddr {
  unsigned long long ctx_id;
  void* ptr;
};
static ScratchAddr g_scratch[kMaxDevices];
static std::mutex g_scratch_mu;

// The unique id of the calling thread's current context (driver entry
// points, no link against the driver library); false if none is current or
// the driver does not offer the calls.
static bool current_context_id(unsigned long long* id) {
  static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
  });
  if (!get_current || !get_id) return false;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

// The device address of the scratch array on the current device (host code
// cannot use the array's name as an address).  Looked up with
// cudaGetSymbolAddress the first time a device's context calls, which also
// initialises that context if the runtime has not yet; later calls in the
// same context reuse it.  Where the context id cannot be read, every call
// looks the address up.
static int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(SM_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(SM_ERR_ARG, "device ordinal %d too large", dev);
  unsigned long long id = 0;
  bool have_id = current_context_id(&id);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (have_id && g_scratch[dev].ptr && g_scratch[dev].ctx_id == id) {
    *out = g_scratch[dev].ptr;
    return SM_OK;
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess)
    return fail(SM_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
  if (!have_id) have_id = current_context_id(&id);  // the lookup made the context current
  g_scratch[dev] = have_id ? ScratchAddr{id, p} : ScratchAddr{0, nullptr};
  *out = p;
  return SM_OK;
}

// out = D in (DAG = false) or D^dag in, one L x T lattice, one site per thread.
template <typename R, bool DAG>
__global__ void __launch_bounds__(kBlock) k_dslash_single(int L, int T, R diag,
                                                          const R* __restrict__ U,
                                                          const R* __restrict__ in,
                                                          R* __restrict__ out) {
  const long long n = (long long)blockIdx.x * kBlock + threadIdx.x;
  if (n >= (long long)L * T) return;
  const int t = (int)(n / L), x = (int)(n - (long long)t * L);
  const long long row = (long long)t * L;
  const long long nxp = row + (x + 1 == L ? 0 : x + 1), nxm = row + (x == 0 ? L - 1 : x - 1);
  const long long ntp = (long long)(t + 1 == T ? 0 : t + 1) * L + x;
  const long long ntm = (long long)(t == 0 ? T - 1 : t - 1) * L + x;
  const Lk<R> u = ld_lk(U, n);
  const Sp<R> o = hop_sum<DAG, R>(ld_sp(in, nxp), ld_sp(in, nxm), ld_sp(in, ntp), ld_sp(in, ntm),
                                  u.x, ld_lk(U, nxm).x, u.t, ld_lk(U, ntm).t);
  st_sp(out, n, diag * ld_sp(in, n) - (R)0.5 * o);
}

template <typename R>
static int ddagd_single(int L, int T, double m0, const R* U, const R* in, R* out, R* t,
                        cudaStream_t s) {
  const long long V = (long long)L * T;
  const unsigned grid = (unsigned)((V + kBlock - 1) / kBlock);
  const R diag = (R)(2.0 + m0);
  k_dslash_single<R, false><<<grid, kBlock, 0, s>>>(L, T, diag, U, in, t);
  const int rc = launched(nullptr, "dslash_single");
  if (rc) return rc;
  k_dslash_single<R, true><<<grid, kBlock, 0, s>>>(L, T, diag, U, t, out);
  return launched(nullptr, "dslash_single");
}

}  // namespace sm

using namespace sm;

extern "C" int sm_apply_DdagD_noalloc(int L, int T, double m0, const void* U, const void* in,
                                      void* out, int prec, void* stream) {
  if (L < 2 || T < 2) return fail(SM_ERR_ARG, "sm_apply_DdagD_noalloc: sides must be >= 2");
  if (!U || !in || !out) return fail(SM_ERR_ARG, "sm_apply_DdagD_noalloc: NULL field");
  if ((((uintptr_t)U) | ((uintptr_t)in) | ((uintptr_t)out)) & 15)
    return fail(SM_ERR_ARG, "sm_apply_DdagD_noalloc: field not 16-byte aligned");
  if (in == out) return fail(SM_ERR_ARG, "sm_apply_DdagD_noalloc: in and out alias");
  if (prec != SM_F64 && prec != SM_F32)
    return fail(SM_ERR_ARG, "sm_apply_DdagD_noalloc: prec must be SM_F64 or SM_F32");
  const size_t site_bytes = prec == SM_F64 ? 32 : 16;
  const long long V = (long long)L * T;
  if ((size_t)V > kNoAllocScratchBytes / site_bytes)
    return fail(SM_ERR_ARG,
                "sm_apply_DdagD_noalloc: %d x %d = %lld sites exceed the %zu-site maximum of the "
                "built-in scratch for this precision",
                L, T, V, kNoAllocScratchBytes / site_bytes);
  void* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
#ifdef SM_DEBUG
  dbg::set_sites(V, s);
#endif
  if (prec == SM_F64)
    return ddagd_single<double>(L, T, m0, (const double*)U, (const double*)in, (double*)out,
                                (double*)scratch, s);
  return ddagd_single<float>(L, T, m0, (const float*)U, (const float*)in, (float*)out,
                             (float*)scratch, s);
}
