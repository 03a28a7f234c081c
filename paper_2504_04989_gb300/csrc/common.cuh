// common.cuh -- shared device helpers of libtsvd (complex arithmetic on
// double2 / float2, launch checks, workspace carving).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstddef>

#include "../../include/tsvd.h"

namespace tsvd {

// complex element type for a real type
template <typename T>
struct Cx;
template <>
struct Cx<double> {
  using type = double2;
};
template <>
struct Cx<float> {
  using type = float2;
};
template <typename T>
using cx_t = typename Cx<T>::type;

__host__ __device__ __forceinline__ double2 mkc(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ float2 mkc(float r, float i) { return make_float2(r, i); }

template <typename T>
__host__ __device__ __forceinline__ cx_t<T> czero() {
  return mkc(T(0), T(0));
}

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// acc += a * b
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }

__device__ __forceinline__ double2 to_c64(double2 a) { return a; }
__device__ __forceinline__ double2 to_c64(float2 a) { return make_double2(a.x, a.y); }
template <typename C>
__device__ __forceinline__ C from_c64(double2 a);
template <>
__device__ __forceinline__ double2 from_c64<double2>(double2 a) {
  return a;
}
template <>
__device__ __forceinline__ float2 from_c64<float2>(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}

// warp reductions
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double2 warp_sum(double2 v) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  return v;
}

// Block-wide sum of a double (all threads get the result).  `red` must hold
// blockDim.x / 32 doubles; the block size is a multiple of 32.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (lane < nw) ? red[lane] : 0.0;
  t = warp_sum(t);
  return t;
}
__device__ __forceinline__ double2 block_sum2(double2 v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) {
    red[2 * wid] = v.x;
    red[2 * wid + 1] = v.y;
  }
  __syncthreads();
  double2 t = (lane < nw) ? make_double2(red[2 * lane], red[2 * lane + 1]) : make_double2(0, 0);
  return warp_sum(t);
}

// Philox4x32-10 (Salmon et al., SC'11): per round, the two products of the
// even counter words with the round multipliers give (hi, lo) halves that are
// mixed with the odd words and the key; the key advances by the Weyl constants.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Host-side workspace carving: consecutive 256-byte aligned regions.
struct Carver {
  char* base;
  size_t off;
  explicit Carver(void* b) : base((char*)b), off(0) {}
  template <typename P>
  P* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    P* p = base ? (P*)(base + off) : nullptr;
    off += count * sizeof(P);
    return p;
  }
  size_t bytes() const { return (off + 255) & ~(size_t)255; }
};

inline int launch_status() { return cudaGetLastError() == cudaSuccess ? TSVD_OK : TSVD_ERR_CUDA; }

#define TSVD_TRY(expr)          \
  do {                          \
    int _rc = (expr);           \
    if (_rc != TSVD_OK) return _rc; \
  } while (0)

// counts every kernel launch of the library (profile.cu)
void count_launch();

#define TSVD_LAUNCHED()                                          \
  do {                                                           \
    ::tsvd::count_launch();                                      \
    if (cudaPeekAtLastError() != cudaSuccess) {                  \
      cudaGetLastError();                                        \
      return TSVD_ERR_CUDA;                                      \
    }                                                            \
  } while (0)

inline unsigned cdiv(long a, long b) { return (unsigned)((a + b - 1) / b); }

}  // namespace tsvd
