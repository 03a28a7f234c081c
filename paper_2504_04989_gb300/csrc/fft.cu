// fft.cu -- mode-3 transforms and the Gaussian test tensor.
//
// rFFT along mode 3 (Sec. 2, Definition of F_n: omega = exp(-2 pi i/n3),
// unnormalised) keeping the h = floor(n3/2)+1 non-redundant slices (Alg. TP),
// and its inverse from the half spectrum (the conjugate mirror of Alg. TP
// followed by F^{-1} = F^*/n3; the imaginary parts of the DC and Nyquist
// slices are ignored, i.e. the real part of the mirrored inverse).
//
// Layout: the plane index e = i*n2 + j runs fastest, so a CTA that owns a tile
// of consecutive e for every t reads and writes whole cache lines; the
// transform of one tube runs out of shared memory.
#include "common.cuh"
#include "kernels.cuh"

namespace tsvd {

// omega^p with omega = exp(sign * 2 pi i / n); exact on the axes so that the DC
// and Nyquist slices of a real tensor come out exactly real.
template <typename T>
__device__ __forceinline__ cx_t<T> twiddle(int p, int n, int sign) {
  p %= n;
  if (p == 0) return mkc(T(1), T(0));
  if (2 * p == n) return mkc(T(-1), T(0));
  if (4 * p == n) return mkc(T(0), T(sign));
  if (4 * p == 3 * n) return mkc(T(0), T(-sign));
  double s, c;
  sincospi(2.0 * (double)p / (double)n, &s, &c);
  return mkc((T)c, (T)(sign * s));
}

template <typename T>
__global__ void __launch_bounds__(256) k_rfft3(const T* __restrict__ X, cx_t<T>* __restrict__ Xh, long plane,
                                               int n3, int te) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using C = cx_t<T>;
  C* tw = (C*)smem_raw;          // [n3]
  T* xs = (T*)(tw + n3);         // [n3][te]
  const long e0 = (long)blockIdx.x * te;
  for (int p = threadIdx.x; p < n3; p += blockDim.x) tw[p] = twiddle<T>(p, n3, -1);
  for (int idx = threadIdx.x; idx < n3 * te; idx += blockDim.x) {
    const int t = idx / te, e = idx - t * te;
    const long ge = e0 + e;
    xs[idx] = (ge < plane) ? __ldg(X + (long)t * plane + ge) : T(0);
  }
  __syncthreads();
  const int h = n3 / 2 + 1;
  const int e = threadIdx.x % te, kg = threadIdx.x / te, nkg = blockDim.x / te;
  const long ge = e0 + e;
  for (int k = kg; k < h; k += nkg) {
    T re = 0, im = 0;
    int p = 0;
    for (int t = 0; t < n3; ++t) {
      const T x = xs[t * te + e];
      const C w = tw[p];
      re = fma(x, w.x, re);
      im = fma(x, w.y, im);
      p += k;
      if (p >= n3) p -= n3;
    }
    if (ge < plane) Xh[(long)k * plane + ge] = mkc(re, im);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_irfft3(const cx_t<T>* __restrict__ Xh, T* __restrict__ X, long plane,
                                                int n3, int te) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using C = cx_t<T>;
  const int h = n3 / 2 + 1;
  C* tw = (C*)smem_raw;  // [n3]
  C* xs = tw + n3;       // [h][te]
  const long e0 = (long)blockIdx.x * te;
  for (int p = threadIdx.x; p < n3; p += blockDim.x) tw[p] = twiddle<T>(p, n3, +1);
  for (int idx = threadIdx.x; idx < h * te; idx += blockDim.x) {
    const int k = idx / te, e = idx - k * te;
    const long ge = e0 + e;
    xs[idx] = (ge < plane) ? Xh[(long)k * plane + ge] : mkc(T(0), T(0));
  }
  __syncthreads();
  const bool even = (n3 % 2) == 0;
  const int kint = even ? h - 1 : h;  // interior slices 1..kint-1 appear twice in the full spectrum
  const T inv = T(1) / T(n3);
  const int e = threadIdx.x % te, tg = threadIdx.x / te, ntg = blockDim.x / te;
  const long ge = e0 + e;
  for (int t = tg; t < n3; t += ntg) {
    T acc = xs[e].x;  // DC
    int p = t;
    for (int k = 1; k < kint; ++k) {
      const C x = xs[k * te + e];
      const C w = tw[p];
      acc = fma(T(2) * x.x, w.x, acc);
      acc = fma(T(-2) * x.y, w.y, acc);
      p += t;
      if (p >= n3) p -= n3;
    }
    if (even) {
      const T xn = xs[(h - 1) * te + e].x;
      acc += (t & 1) ? -xn : xn;
    }
    if (ge < plane) X[(long)t * plane + ge] = acc * inv;
  }
}

static int tile_e(int n3, size_t elem, size_t celem, bool inverse) {
  // largest power-of-two tile (<= 128, >= 32) whose shared footprint stays under 96 KB
  const int h = n3 / 2 + 1;
  for (int te = 128; te >= 32; te >>= 1) {
    size_t bytes = (size_t)n3 * celem + (size_t)(inverse ? h * celem : n3 * elem) * te;
    if (bytes <= 96 * 1024) return te;
  }
  return 32;
}

template <typename T>
int launch_rfft3(const T* X, cx_t<T>* Xh, long plane, int n3, cudaStream_t s) {
  if (plane <= 0) return TSVD_OK;
  const int te = tile_e(n3, sizeof(T), sizeof(cx_t<T>), false);
  const size_t smem = (size_t)n3 * sizeof(cx_t<T>) + (size_t)n3 * te * sizeof(T);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_rfft3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_rfft3<T><<<cdiv(plane, te), 256, smem, s>>>(X, Xh, plane, n3, te);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

template <typename T>
int launch_irfft3(const cx_t<T>* Xh, T* X, long plane, int n3, cudaStream_t s) {
  if (plane <= 0) return TSVD_OK;
  const int h = n3 / 2 + 1;
  const int te = tile_e(n3, sizeof(T), sizeof(cx_t<T>), true);
  const size_t smem = (size_t)n3 * sizeof(cx_t<T>) + (size_t)h * te * sizeof(cx_t<T>);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_irfft3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_irfft3<T><<<cdiv(plane, te), 256, smem, s>>>(Xh, X, plane, n3, te);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

template int launch_rfft3<double>(const double*, double2*, long, int, cudaStream_t);
template int launch_rfft3<float>(const float*, float2*, long, int, cudaStream_t);
template int launch_irfft3<double>(const double2*, double*, long, int, cudaStream_t);
template int launch_irfft3<float>(const float2*, float*, long, int, cudaStream_t);

// Element e of stream (seed, stream_id, tensor_id) is Box-Muller output e%4 of
// Philox call e/4; the two uniforms of a pair are (x + 1) 2^-32 in (0, 1].
template <typename T>
__global__ void k_gaussian(uint64_t seed, uint32_t stream_id, uint32_t tensor_id, long n, T* __restrict__ out) {
  const long call = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * call >= n) return;
  const uint4 x = philox10(make_uint4((uint32_t)call, (uint32_t)((unsigned long long)call >> 32), stream_id, tensor_id),
                           (uint32_t)seed, (uint32_t)(seed >> 32));
  const double inv32 = 1.0 / 4294967296.0;
  const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
  for (int pair = 0; pair < 2; ++pair) {
    const double u1 = ((double)w[2 * pair] + 1.0) * inv32;
    const double u2 = ((double)w[2 * pair + 1] + 1.0) * inv32;
    const double r = sqrt(-2.0 * log(u1));
    const double th = 2.0 * 3.141592653589793 * u2;
    const long e = 4 * call + 2 * pair;
    if (e < n) out[e] = (T)(r * cos(th));
    if (e + 1 < n) out[e + 1] = (T)(r * sin(th));
  }
}

__global__ void k_philox_words(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3, long n,
                               uint32_t* __restrict__ out) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 x = philox10(make_uint4((uint32_t)i, c1, c2, c3), k0, k1);
  out[4 * i + 0] = x.x;
  out[4 * i + 1] = x.y;
  out[4 * i + 2] = x.z;
  out[4 * i + 3] = x.w;
}

template <typename T>
int launch_gaussian(uint64_t seed, uint32_t stream_id, uint32_t tensor_id, long n, T* out, cudaStream_t s) {
  if (n <= 0) return TSVD_OK;
  const long calls = (n + 3) / 4;
  k_gaussian<T><<<cdiv(calls, 256), 256, 0, s>>>(seed, stream_id, tensor_id, n, out);
  TSVD_LAUNCHED();
  return TSVD_OK;
}
template int launch_gaussian<double>(uint64_t, uint32_t, uint32_t, long, double*, cudaStream_t);
template int launch_gaussian<float>(uint64_t, uint32_t, uint32_t, long, float*, cudaStream_t);

}  // namespace tsvd

extern "C" int tsvd_gaussian(uint64_t seed, uint32_t stream_id, uint32_t tensor_id, long n, double* out,
                             void* stream) {
  if (n < 0 || (n > 0 && !out)) return TSVD_ERR_INVALID_ARG;
  return tsvd::launch_gaussian<double>(seed, stream_id, tensor_id, n, out, (cudaStream_t)stream);
}

extern "C" int tsvd_philox_words(const uint32_t key[2], uint32_t ctr1, uint32_t ctr2, uint32_t ctr3, long n,
                                 uint32_t* out, void* stream) {
  if (!key || n < 0 || (n > 0 && !out)) return TSVD_ERR_INVALID_ARG;
  if (n == 0) return TSVD_OK;
  tsvd::k_philox_words<<<tsvd::cdiv(n, 256), 256, 0, (cudaStream_t)stream>>>(key[0], key[1], ctr1, ctr2, ctr3, n, out);
  TSVD_LAUNCHED();
  return TSVD_OK;
}
