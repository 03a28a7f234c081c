// tprod_noalloc.cu -- t-product C = A * B for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) around the
// computation: code running inside a memory-pool or arena that must not grow,
// plug-ins hosted by a process that owns all device allocations, or real-time
// loops where an allocation would stall.  They still own the inputs and the
// output; this entry point takes its scratch (the three Fourier-domain
// operands and the split-K partial sums) from a fixed array in this file
// instead of a caller workspace.
//
// Costs and rules of the fixed array:
//  * every GPU that loads the library keeps TPROD_NOALLOC_SCRATCH_BYTES (16 MiB)
//    of device memory reserved until the process exits;
//  * all calls share it and it keeps the last call's contents; nothing in it
//    has to start at zero (every byte a call reads was written earlier by the
//    same call), so nothing is cleared;
//  * calls whose kernels overlap on the GPU (different streams, or different
//    host threads, without ordering between them) race on the array;
//  * the array lives in this file's own module, which holds no kernel; under
//    CUDA's lazy module loading (the default) that module, and with it the
//    16 MiB, is loaded on a device at the first call there (the address
//    lookup below), so make that first call before sealing a pool or arena
//    that must not grow afterwards, and before any CUDA graph capture;
//  * every call outside stream capture looks the address up again
//    (cudaGetSymbolAddress allocates nothing once the module is loaded), so a
//    device reset that reloads the module at another address is followed;
//    inside a capture the address of the last uncaptured call on the device
//    is used.
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace tsvd {

constexpr size_t TPROD_NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;

// The scratch itself.  Host code must not pass `g_tprod_scratch` to a kernel:
// on the host the name is only a stand-in; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_tprod_scratch[TPROD_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
static void* g_scratch_ptr[kMaxDevices];  // last looked-up device address of g_tprod_scratch per device

// The device address of the array on the current device: looked up on every
// call outside stream capture (a context re-created after a device reset can
// place the module elsewhere), the cached one inside a capture.
static int scratch_address(cudaStream_t s, void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TSVD_ERR_CUDA;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    cap = cudaStreamCaptureStatusActive;  // cannot tell: do not call into the runtime's module tables
  }
  void* p = nullptr;
  if (cap == cudaStreamCaptureStatusNone) {
    if (cudaGetSymbolAddress(&p, g_tprod_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return TSVD_ERR_CUDA;
    }
    __atomic_store_n(&g_scratch_ptr[dev], p, __ATOMIC_RELEASE);
  } else {
    p = __atomic_load_n(&g_scratch_ptr[dev], __ATOMIC_ACQUIRE);
    if (!p) return TSVD_ERR_CUDA;  // no uncaptured call on this device yet
  }
  *out = p;
  return TSVD_OK;
}

template <typename T>
static int tprod_noalloc_run(const T* A, const T* B, T* Cout, int n1, int n2, int n4, int n3, cudaStream_t s) {
  using C = cx_t<T>;
  const size_t h = n3 / 2 + 1;
  // each operand's size in floating point first: the size_t products below
  // could wrap for very large dimensions and pass the limit check
  const double lim = (double)TPROD_NOALLOC_SCRATCH_BYTES / sizeof(C);
  if ((double)h * n1 * n2 > lim || (double)h * n2 * n4 > lim || (double)h * n1 * n4 > lim)
    return TSVD_ERR_UNSUPPORTED;
  Carver cv(nullptr);
  cv.take<C>(h * n1 * n2);
  cv.take<C>(h * n2 * n4);
  cv.take<C>(h * n1 * n4);
  const size_t operands = cv.bytes();
  if (operands > TPROD_NOALLOC_SCRATCH_BYTES) return TSVD_ERR_UNSUPPORTED;
  void* base = nullptr;
  TSVD_TRY(scratch_address(s, &base));
  Carver w(base);
  C* Ah = w.take<C>(h * n1 * n2);
  C* Bh = w.take<C>(h * n2 * n4);
  C* Ch = w.take<C>(h * n1 * n4);
  const size_t used = w.bytes();
  C* sk = (C*)((char*)base + used);
  const size_t sk_elems = (TPROD_NOALLOC_SCRATCH_BYTES - used) / sizeof(C);
  TSVD_TRY(launch_rfft3<T>(A, Ah, (long)n1 * n2, n3, s));
  TSVD_TRY(launch_rfft3<T>(B, Bh, (long)n2 * n4, n3, s));
  GemmArgs g;
  g.opA = 'N';
  g.opB = 'N';
  g.M = n1;
  g.N = n4;
  g.K = n2;
  g.alpha = 1.0;
  g.beta = 0.0;
  g.A = Ah;
  g.lda = n2;
  g.sA = (long)n1 * n2;
  g.B = Bh;
  g.ldb = n4;
  g.sB = (long)n2 * n4;
  g.C = Ch;
  g.ldc = n4;
  g.sC = (long)n1 * n4;
  g.batch = (int)h;
  TSVD_TRY(cgemm<C>(g, sk_elems > 0 ? sk : nullptr, sk_elems, s));
  TSVD_TRY(launch_irfft3<T>(Ch, Cout, (long)n1 * n4, n3, s));
  return TSVD_OK;
}

}  // namespace tsvd

using namespace tsvd;

extern "C" int tprod_noalloc(const void* A, const void* B, void* C, int n1, int n2, int n4, int n3, int precision,
                             void* stream) {
  if (!A || !B || !C || n1 < 1 || n2 < 1 || n4 < 1 || n3 < 1) return TSVD_ERR_INVALID_ARG;
  if (precision != TSVD_FP64 && precision != TSVD_FP32) return TSVD_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == TSVD_FP64)
    return tprod_noalloc_run<double>((const double*)A, (const double*)B, (double*)C, n1, n2, n4, n3, s);
  return tprod_noalloc_run<float>((const float*)A, (const float*)B, (float*)C, n1, n2, n4, n3, s);
}
