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
  if (sizeof(T) == sizeof(float)) {
    float s, c;
    sincospif(2.0f * (float)p / (float)n, &s, &c);
    return mkc((T)c, (T)(sign * s));
  }
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

// ---------------------------------------------------------------------------
// Mixed-radix FFT of the tubes (Stockham autosort, radices 4, 2, 3, 5 and any
// remaining prime).  A CTA owns a tile of FFT_TUBES consecutive tubes; two real
// tubes are packed into one complex sequence z = x + i y and each warp
// transforms whole sequences in shared memory (lane-parallel butterflies,
// warp barriers between passes).  The half spectra are separated as
// X_k = (Z_k + conj Z_{n-k}) / 2, Y_k = (Z_k - conj Z_{n-k}) / (2i); the inverse
// packs Z = X + i Y over the full (Hermitian) spectrum.  Global reads and writes
// run along the plane index, so they stay coalesced.
// ---------------------------------------------------------------------------
constexpr int FFT_WARPS = 8;
constexpr int FFT_LOADS = 8;
constexpr int FFT_MAXR = 24;
// sequences a warp transforms together
constexpr int fft_seqs(int n) { return n < 1 ? 1 : (256 / n < 1 ? 1 : (256 / n > 4 ? 4 : 256 / n)); }
struct FftPlan {
  int n, nr, tubes;
  int seqs;  // sequences a warp transforms together (every pass has seqs * n / R independent butterflies)
  int radix[FFT_MAXR];
};

static bool make_plan(int n, FftPlan* p) {
  p->n = n;
  p->nr = 0;
  p->seqs = fft_seqs(n);
  int m = n;
  while (m % 4 == 0) { p->radix[p->nr++] = 4; m /= 4; }
  while (m % 2 == 0) { p->radix[p->nr++] = 2; m /= 2; }
  for (int f = 3; m > 1; f += 2) {
    while (m % f == 0) {
      if (p->nr >= FFT_MAXR) return false;
      p->radix[p->nr++] = f;
      m /= f;
    }
  }
  return true;
}

// one Stockham pass of radix R (sign of the exponent in tw): in -> out
template <typename C, int R>
__device__ __forceinline__ void fft_pass_fixed(const C* __restrict__ in0, C* __restrict__ out0,
                                               const C* __restrict__ tw, int n, int Ns, int lane, int nseq) {
  const int nR = n / R, tstep = n / (Ns * R);
  for (int jj = lane; jj < nseq * nR; jj += 32) {
    const int sq = jj / nR, j = jj - sq * nR;
    const C* __restrict__ in = in0 + sq * n;
    C* __restrict__ out = out0 + sq * n;
    const int k = j % Ns;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      v[r] = in[j + r * nR];
      if (r > 0) v[r] = cmul(v[r], tw[(r * k * tstep) % n]);
    }
    C o[R];
    if (R == 2) {
      o[0] = cadd(v[0], v[1]);
      o[1] = csub(v[0], v[1]);
    } else if (R == 4) {
      // omega_4 = tw[n/4] is exactly +-i
      const C w = tw[n / 4];
      const C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
      const C c = cadd(v[1], v[3]), d = cmul(csub(v[1], v[3]), w);
      o[0] = cadd(a, c);
      o[2] = csub(a, c);
      o[1] = cadd(b, d);
      o[3] = csub(b, d);
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        C acc = v[0];
#pragma unroll
        for (int r = 1; r < R; ++r) acc = cadd(acc, cmul(v[r], tw[((q * r) % R) * (n / R)]));
        o[q] = acc;
      }
    }
    const int idxD = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[idxD + r * Ns] = o[r];
  }
}

template <typename C>
__device__ void fft_pass_generic(const C* __restrict__ in0, C* __restrict__ out0, const C* __restrict__ tw, int n,
                                 int Ns, int R, int lane, int nseq) {
  const int nR = n / R, tstep = n / (Ns * R);
  for (int jj = lane; jj < nseq * nR; jj += 32) {
    const int sq = jj / nR, j = jj - sq * nR;
    const C* __restrict__ in = in0 + sq * n;
    C* __restrict__ out = out0 + sq * n;
    const int k = j % Ns;
    const int idxD = (j / Ns) * Ns * R + k;
    for (int q = 0; q < R; ++q) {
      C acc = in[j];
      for (int r = 1; r < R; ++r) {
        const C vr = cmul(in[j + r * nR], tw[(r * k * tstep) % n]);
        acc = cadd(acc, cmul(vr, tw[((q * r) % R) * (n / R)]));
      }
      out[idxD + q * Ns] = acc;
    }
  }
}

// in-place (ping-pong) FFT of nseq length-n sequences (stride n) in a / b;
// returns the buffer holding the result
template <typename C>
__device__ C* fft_run(C* a, C* b, const C* tw, const FftPlan& P, int lane, int nseq) {
  int Ns = 1;
  for (int s = 0; s < P.nr; ++s) {
    const int R = P.radix[s];
    if (R == 4) fft_pass_fixed<C, 4>(a, b, tw, P.n, Ns, lane, nseq);
    else if (R == 2) fft_pass_fixed<C, 2>(a, b, tw, P.n, Ns, lane, nseq);
    else if (R == 3) fft_pass_fixed<C, 3>(a, b, tw, P.n, Ns, lane, nseq);
    else if (R == 5) fft_pass_fixed<C, 5>(a, b, tw, P.n, Ns, lane, nseq);
    else fft_pass_generic<C>(a, b, tw, P.n, Ns, R, lane, nseq);
    __syncwarp();
    C* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// The same transform for a length known at compile time (powers of two up to
// 128): the pass sequence (radix 4 while possible, then 2, as make_plan) is
// unrolled and every index division and modulus becomes a shift or a mask.
template <typename C, int N, int NS>
__device__ __forceinline__ C* fft_run_c(C* a, C* b, const C* tw, int lane, int nseq) {
  if constexpr (NS >= N) {
    return a;
  } else {
    constexpr int R = ((N / NS) % 4 == 0) ? 4 : 2;
    fft_pass_fixed<C, R>(a, b, tw, N, NS, lane, nseq);
    __syncwarp();
    return fft_run_c<C, N, NS * R>(b, a, tw, lane, nseq);
  }
}

template <typename T>
constexpr size_t fft_smem_c(int n, int tt) {
  return sizeof(cx_t<T>) * ((size_t)n + (size_t)FFT_WARPS * 2 * fft_seqs(n) * n + (size_t)(n / 2 + 1) * (tt + 1)) +
         sizeof(T) * (size_t)n * (tt + 1);
}
// tubes per CTA (the choice fft_setup makes at run time): the widest tile that leaves room for
// three CTAs per SM (measured: n = 128 in FP32 went from 64 tubes, two CTAs per SM, to 32),
// else the widest within 110 KB
constexpr size_t FFT_SMEM_3 = 72 * 1024, FFT_SMEM_MAX = 110 * 1024;
constexpr int fft_pick_tt(size_t s64, size_t s32, size_t s16) {
  return s64 <= FFT_SMEM_3 ? 64 : s32 <= FFT_SMEM_3 ? 32 : s16 <= FFT_SMEM_3 ? 16 :
         s64 <= FFT_SMEM_MAX ? 64 : s32 <= FFT_SMEM_MAX ? 32 : s16 <= FFT_SMEM_MAX ? 16 : 0;
}
template <typename T>
constexpr int fft_tt(int n) {
  return fft_pick_tt(fft_smem_c<T>(n, 64), fft_smem_c<T>(n, 32), fft_smem_c<T>(n, 16));
}

template <typename T, int NC>  // NC: compile-time length (0: the plan's)
__global__ void __launch_bounds__(FFT_WARPS * 32) k_rfft3_fft(const T* __restrict__ X, cx_t<T>* __restrict__ Xh,
                                                              long plane, FftPlan P) {
  using C = cx_t<T>;
  extern __shared__ __align__(16) unsigned char fsm[];
  const int n = NC ? NC : P.n, h = n / 2 + 1, TT = NC ? fft_tt<T>(NC) : P.tubes;
  C* tw = (C*)fsm;                                  // [n]
  C* zb = tw + n;                                   // [FFT_WARPS][2][seqs][n]
  const int LD = TT + 1;                            // padded row stride: conflict-free column walks
  C* otile = zb + (size_t)FFT_WARPS * 2 * (NC ? fft_seqs(NC) : P.seqs) * n;  // [h][LD] complex
  T* itile = (T*)(otile + (size_t)h * LD);          // [n][LD] real
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long e0 = (long)blockIdx.x * TT;
  for (int p = threadIdx.x; p < n; p += blockDim.x) tw[p] = twiddle<T>(p, n, -1);
  if (sizeof(T) == 4 && (plane & 3) == 0 && ((uintptr_t)X & 15) == 0 && e0 + TT <= plane) {
    // whole tile, FP32: 16-byte loads of four consecutive tubes, FFT_LOADS in flight per thread
    const int q4 = TT / 4, total = n * q4;
    for (int base = threadIdx.x; base < total; base += FFT_LOADS * blockDim.x) {
      float4 v[FFT_LOADS];
#pragma unroll
      for (int u = 0; u < FFT_LOADS; ++u) {
        const int idx = base + u * blockDim.x;
        const int t = idx / q4, e = 4 * (idx - t * q4);
        v[u] = (idx < total) ? __ldg((const float4*)(X + (long)t * plane + e0 + e)) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < FFT_LOADS; ++u) {
        const int idx = base + u * blockDim.x;
        if (idx < total) {
          const int t = idx / q4, e = 4 * (idx - t * q4);
          T* d = itile + t * LD + e;
          d[0] = (T)v[u].x;
          d[1] = (T)v[u].y;
          d[2] = (T)v[u].z;
          d[3] = (T)v[u].w;
        }
      }
    }
  } else {
    // FFT_LOADS independent loads in flight per thread (memory-level parallelism)
    const int total = n * TT;
    for (int base = threadIdx.x; base < total; base += FFT_LOADS * blockDim.x) {
      T v[FFT_LOADS];
#pragma unroll
      for (int u = 0; u < FFT_LOADS; ++u) {
        const int idx = base + u * blockDim.x;
        const int t = idx / TT, e = idx - t * TT;
        const long ge = e0 + e;
        v[u] = (idx < total && ge < plane) ? __ldg(X + (long)t * plane + ge) : T(0);
      }
#pragma unroll
      for (int u = 0; u < FFT_LOADS; ++u) {
        const int idx = base + u * blockDim.x;
        if (idx < total) itile[(idx / TT) * LD + idx % TT] = v[u];
      }
    }
  }
  __syncthreads();
  const int B = NC ? fft_seqs(NC) : P.seqs;
  C* za = zb + (size_t)warp * 2 * B * n;
  C* zc = za + (size_t)B * n;
  const T hf = T(0.5);
  for (int s0 = warp * B; s0 < TT / 2; s0 += FFT_WARPS * B) {
    const int nseq = min(B, TT / 2 - s0);
    for (int q = lane; q < nseq * n; q += 32) {
      const int sq = q / n, t = q - sq * n, s = s0 + sq;
      za[q] = mkc(itile[t * LD + 2 * s], itile[t * LD + 2 * s + 1]);
    }
    __syncwarp();
    const C* Z;
    if constexpr (NC > 0) Z = fft_run_c<C, NC, 1>(za, zc, tw, lane, nseq);
    else Z = fft_run<C>(za, zc, tw, P, lane, nseq);
    for (int q = lane; q < nseq * h; q += 32) {
      const int sq = q / h, k = q - sq * h, s = s0 + sq;
      const C zk = Z[sq * n + k], zn = Z[sq * n + (n - k) % n];
      otile[k * LD + 2 * s] = mkc(hf * (zk.x + zn.x), hf * (zk.y - zn.y));      // X_k
      otile[k * LD + 2 * s + 1] = mkc(hf * (zk.y + zn.y), hf * (zn.x - zk.x));  // Y_k
    }
    __syncwarp();
  }
  __syncthreads();
  if (sizeof(T) == 4 && (plane & 1) == 0 && ((uintptr_t)Xh & 15) == 0 && e0 + TT <= plane) {
    // whole tile, FP32: 16-byte stores of two consecutive complex values
    const int q2 = TT / 2;
    for (int idx = threadIdx.x; idx < h * q2; idx += blockDim.x) {
      const int k = idx / q2, e = 2 * (idx - k * q2);
      const C a = otile[k * LD + e], c = otile[k * LD + e + 1];
      *(float4*)(Xh + (long)k * plane + e0 + e) = make_float4((float)a.x, (float)a.y, (float)c.x, (float)c.y);
    }
  } else {
    for (int idx = threadIdx.x; idx < h * TT; idx += blockDim.x) {
      const int k = idx / TT, e = idx - k * TT;
      const long ge = e0 + e;
      if (ge < plane) Xh[(long)k * plane + ge] = otile[k * LD + e];
    }
  }
}

template <typename T, int NC>  // NC: compile-time length (0: the plan's)
__global__ void __launch_bounds__(FFT_WARPS * 32) k_irfft3_fft(const cx_t<T>* __restrict__ Xh, T* __restrict__ X,
                                                               long plane, FftPlan P) {
  using C = cx_t<T>;
  extern __shared__ __align__(16) unsigned char fsm[];
  const int n = NC ? NC : P.n, h = n / 2 + 1, TT = NC ? fft_tt<T>(NC) : P.tubes;
  C* tw = (C*)fsm;                                  // [n]
  C* zb = tw + n;                                   // [FFT_WARPS][2][seqs][n]
  const int LD = TT + 1;                            // padded row stride: conflict-free column walks
  C* itile = zb + (size_t)FFT_WARPS * 2 * (NC ? fft_seqs(NC) : P.seqs) * n;  // [h][LD] complex
  T* otile = (T*)(itile + (size_t)h * LD);          // [n][LD] real
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long e0 = (long)blockIdx.x * TT;
  for (int p = threadIdx.x; p < n; p += blockDim.x) tw[p] = twiddle<T>(p, n, +1);
  {
    const int total = h * TT;
    for (int base = threadIdx.x; base < total; base += FFT_LOADS * blockDim.x) {
      C v[FFT_LOADS];
#pragma unroll
      for (int u = 0; u < FFT_LOADS; ++u) {
        const int idx = base + u * blockDim.x;
        const int k = idx / TT, e = idx - k * TT;
        const long ge = e0 + e;
        v[u] = mkc(T(0), T(0));
        if (idx < total && ge < plane) v[u] = Xh[(long)k * plane + ge];
        if (k == 0 || 2 * k == n) v[u].y = T(0);  // c2r: the DC and Nyquist slices are real
      }
#pragma unroll
      for (int u = 0; u < FFT_LOADS; ++u) {
        const int idx = base + u * blockDim.x;
        if (idx < total) itile[(idx / TT) * LD + idx % TT] = v[u];
      }
    }
  }
  __syncthreads();
  const int B = NC ? fft_seqs(NC) : P.seqs;
  C* za = zb + (size_t)warp * 2 * B * n;
  C* zc = za + (size_t)B * n;
  const T inv = T(1) / T(n);
  for (int s0 = warp * B; s0 < TT / 2; s0 += FFT_WARPS * B) {
    const int nseq = min(B, TT / 2 - s0);
    for (int q = lane; q < nseq * n; q += 32) {
      const int sq = q / n, k = q - sq * n, s = s0 + sq;
      C x, y;
      if (k < h) {
        x = itile[k * LD + 2 * s];
        y = itile[k * LD + 2 * s + 1];
      } else {
        x = cconj(itile[(n - k) * LD + 2 * s]);
        y = cconj(itile[(n - k) * LD + 2 * s + 1]);
      }
      za[q] = mkc(x.x - y.y, x.y + y.x);  // Z = X + i Y
    }
    __syncwarp();
    const C* z;
    if constexpr (NC > 0) z = fft_run_c<C, NC, 1>(za, zc, tw, lane, nseq);
    else z = fft_run<C>(za, zc, tw, P, lane, nseq);
    for (int q = lane; q < nseq * n; q += 32) {
      const int sq = q / n, t = q - sq * n, s = s0 + sq;
      otile[t * LD + 2 * s] = z[q].x * inv;
      otile[t * LD + 2 * s + 1] = z[q].y * inv;
    }
    __syncwarp();
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * TT; idx += blockDim.x) {
    const int t = idx / TT, e = idx - t * TT;
    const long ge = e0 + e;
    if (ge < plane) X[(long)t * plane + ge] = otile[t * LD + e];
  }
}

// shared bytes of the FFT kernels for tile width tt (0 when the plan does not exist)
template <typename T>
static size_t fft_smem(int n, int tt, int seqs) {
  const int h = n / 2 + 1;
  return sizeof(cx_t<T>) * ((size_t)n + (size_t)FFT_WARPS * 2 * seqs * n + (size_t)h * (tt + 1)) +
         sizeof(T) * (size_t)n * (tt + 1);
}

template <typename T>
static bool fft_setup(int n, FftPlan* P, size_t* smem) {
  if (!make_plan(n, P)) return false;
  const int tt = fft_pick_tt(fft_smem<T>(n, 64, P->seqs), fft_smem<T>(n, 32, P->seqs), fft_smem<T>(n, 16, P->seqs));
  if (tt == 0) return false;
  P->tubes = tt;
  *smem = fft_smem<T>(n, tt, P->seqs);
  return true;
}

template <typename T>
int launch_rfft3(const T* X, cx_t<T>* Xh, long plane, int n3, cudaStream_t s) {
  if (plane <= 0) return TSVD_OK;
  FftPlan P;
  size_t smem;
  if (fft_setup<T>(n3, &P, &smem)) {
    auto go = [&](auto kern) {
      if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      kern<<<cdiv(plane, P.tubes), FFT_WARPS * 32, smem, s>>>(X, Xh, plane, P);
      TSVD_LAUNCHED();
      return TSVD_OK;
    };
    switch (n3) {  // compile-time lengths (same tile width as the plan's)
      case 4: return go(k_rfft3_fft<T, 4>);
      case 8: return go(k_rfft3_fft<T, 8>);
      case 16: return go(k_rfft3_fft<T, 16>);
      case 32: return go(k_rfft3_fft<T, 32>);
      case 64: return go(k_rfft3_fft<T, 64>);
      case 128: return go(k_rfft3_fft<T, 128>);
      default: return go(k_rfft3_fft<T, 0>);
    }
  }
  // very long tubes: direct transform
  const int te = tile_e(n3, sizeof(T), sizeof(cx_t<T>), false);
  const size_t sm = (size_t)n3 * sizeof(cx_t<T>) + (size_t)n3 * te * sizeof(T);
  if (sm > 227 * 1024) return TSVD_ERR_UNSUPPORTED;
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_rfft3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_rfft3<T><<<cdiv(plane, te), 256, sm, s>>>(X, Xh, plane, n3, te);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

template <typename T>
int launch_irfft3(const cx_t<T>* Xh, T* X, long plane, int n3, cudaStream_t s) {
  if (plane <= 0) return TSVD_OK;
  FftPlan P;
  size_t smem;
  if (fft_setup<T>(n3, &P, &smem)) {
    auto go = [&](auto kern) {
      if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      kern<<<cdiv(plane, P.tubes), FFT_WARPS * 32, smem, s>>>(Xh, X, plane, P);
      TSVD_LAUNCHED();
      return TSVD_OK;
    };
    switch (n3) {
      case 4: return go(k_irfft3_fft<T, 4>);
      case 8: return go(k_irfft3_fft<T, 8>);
      case 16: return go(k_irfft3_fft<T, 16>);
      case 32: return go(k_irfft3_fft<T, 32>);
      case 64: return go(k_irfft3_fft<T, 64>);
      case 128: return go(k_irfft3_fft<T, 128>);
      default: return go(k_irfft3_fft<T, 0>);
    }
  }
  const int h = n3 / 2 + 1;
  const int te = tile_e(n3, sizeof(T), sizeof(cx_t<T>), true);
  const size_t sm = (size_t)n3 * sizeof(cx_t<T>) + (size_t)h * te * sizeof(cx_t<T>);
  if (sm > 227 * 1024) return TSVD_ERR_UNSUPPORTED;
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_irfft3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_irfft3<T><<<cdiv(plane, te), 256, sm, s>>>(Xh, X, plane, n3, te);
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
  const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
  for (int pair = 0; pair < 2; ++pair) {
    const long e = 4 * call + 2 * pair;
    T g0, g1;
    if constexpr (sizeof(T) == sizeof(float)) {
      // FP32 stream: the same definition evaluated in FP32 (its values are FP32 anyway; FP64
      // transcendentals run at 1/64 of the FP32 rate here)
      const float u1 = fmaf((float)w[2 * pair], 0x1p-32f, 0x1p-32f);
      const float u2 = fmaf((float)w[2 * pair + 1], 0x1p-32f, 0x1p-32f);
      const float r = sqrtf(-2.0f * logf(u1));
      float sn, cs;
      sincospif(2.0f * u2, &sn, &cs);
      g0 = r * cs;
      g1 = r * sn;
    } else {
      const double inv32 = 1.0 / 4294967296.0;
      const double u1 = ((double)w[2 * pair] + 1.0) * inv32;
      const double u2 = ((double)w[2 * pair + 1] + 1.0) * inv32;
      const double r = sqrt(-2.0 * log(u1));
      const double th = 2.0 * 3.141592653589793 * u2;
      g0 = (T)(r * cos(th));
      g1 = (T)(r * sin(th));
    }
    if (e < n) out[e] = g0;
    if (e + 1 < n) out[e + 1] = g1;
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

// The mode-3 transforms on their own (Sec. 2, Def. of F_n; Alg. TP first and
// last lines), for callers that move Fourier slices between devices.
extern "C" int tsvd_rfft3(const void* X, long plane, int n3, int precision, void* Xhat, void* stream) {
  if (!X || !Xhat || plane < 1 || n3 < 1) return TSVD_ERR_INVALID_ARG;
  if (precision == TSVD_FP64)
    return tsvd::launch_rfft3<double>((const double*)X, (double2*)Xhat, plane, n3, (cudaStream_t)stream);
  if (precision == TSVD_FP32)
    return tsvd::launch_rfft3<float>((const float*)X, (float2*)Xhat, plane, n3, (cudaStream_t)stream);
  return TSVD_ERR_INVALID_ARG;
}

extern "C" int tsvd_irfft3(const void* Xhat, long plane, int n3, int precision, void* X, void* stream) {
  if (!X || !Xhat || plane < 1 || n3 < 1) return TSVD_ERR_INVALID_ARG;
  if (precision == TSVD_FP64)
    return tsvd::launch_irfft3<double>((const double2*)Xhat, (double*)X, plane, n3, (cudaStream_t)stream);
  if (precision == TSVD_FP32)
    return tsvd::launch_irfft3<float>((const float2*)Xhat, (float*)X, plane, n3, (cudaStream_t)stream);
  return TSVD_ERR_INVALID_ARG;
}
