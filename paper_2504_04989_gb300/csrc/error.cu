// error.cu -- the approximation error ||X - U * S * V^T||_F^2 of a truncated
// T-SVD (the quantity the experiments of Sec. 5 report), evaluated in the
// Fourier domain.  By Parseval (Sec. 2: ||X||_F^2 = (1/n3) sum_k ||X_k||_F^2
// over the Fourier slices) and the conjugate symmetry of the slices of a real
// tensor, only the h = floor(n3/2)+1 leading slices are needed: weight 1 for
// slice 0 (and for slice n3/2 when n3 is even), 2 for the others.
// One fused pass per slice: E_k = X_k - U_k diag(s_k) V_k^H is formed tile by
// tile in registers and only w_k |E|^2 / n3 is accumulated (FP64); the
// reconstruction is never written to memory.
#include "common.cuh"
#include "kernels.cuh"

namespace tsvd {

constexpr int FE_TILE = 64;  // output tile FE_TILE x FE_TILE per CTA, 4 x 4 per thread
constexpr int FE_RC = 16;    // rank columns staged per round

template <typename T>
__global__ void __launch_bounds__(256, 1) k_fro_error(const cx_t<T>* __restrict__ Xh, const cx_t<T>* __restrict__ Uh,
                                                   const cx_t<T>* __restrict__ Sh, const cx_t<T>* __restrict__ Vh,
                                                   int n1, int n2, int R, int n3, double* __restrict__ partial) {
  using C = cx_t<T>;
  __shared__ C Us[FE_RC][FE_TILE];  // U(i, r) s(r)
  __shared__ C Vs[FE_RC][FE_TILE];  // conj(V(l, r))
  __shared__ double red[8];
  const int k = blockIdx.z;
  const int i0 = blockIdx.y * FE_TILE, l0 = blockIdx.x * FE_TILE;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const C* U = Uh + (long)k * n1 * R;
  const C* V = Vh + (long)k * n2 * R;
  const C* s = Sh + (long)k * R;
  C acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = C{0, 0};
  for (int r0 = 0; r0 < R; r0 += FE_RC) {
    for (int e = threadIdx.x; e < FE_RC * FE_TILE; e += 256) {
      const int rr = e / FE_TILE, ii = e % FE_TILE, r = r0 + rr;
      C u = C{0, 0}, v = C{0, 0};
      if (r < R) {
        if (i0 + ii < n1) u = cmul(U[(long)(i0 + ii) * R + r], s[r]);
        if (l0 + ii < n2) v = cconj(V[(long)(l0 + ii) * R + r]);
      }
      Us[rr][ii] = u;
      Vs[rr][ii] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < FE_RC; ++rr) {
      C uu[4], vv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) uu[a] = Us[rr][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) vv[b] = Vs[rr][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) cfma(acc[a][b], uu[a], vv[b]);
    }
    __syncthreads();
  }
  const C* X = Xh + (long)k * n1 * n2;
  double e2 = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty + 16 * a;
    if (i >= n1) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int l = l0 + tx + 16 * b;
      if (l >= n2) continue;
      const C x = X[(long)i * n2 + l];
      const double er = (double)x.x - (double)acc[a][b].x, ei = (double)x.y - (double)acc[a][b].y;
      e2 = fma(er, er, fma(ei, ei, e2));
    }
  }
  const double tot = block_sum(e2, red);
  if (threadIdx.x == 0) {
    const double wk = (k == 0 || 2 * k == n3) ? 1.0 : 2.0;
    partial[((long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = tot * wk / n3;
  }
}

__global__ void k_sum_error_partials(const double* __restrict__ partial, long n, double* __restrict__ out) {
  __shared__ double red[8];
  double acc = 0;
  for (long i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) *out = s;
}

template <typename T>
struct ErrWs {
  cx_t<T>* Xh;
  cx_t<T>* Uh;
  cx_t<T>* Vh;
  cx_t<T>* Sh;
  double* partial;
};

static dim3 error_grid(int n1, int n2, int n3) { return dim3(cdiv(n2, FE_TILE), cdiv(n1, FE_TILE), n3 / 2 + 1); }

template <typename T>
static ErrWs<T> carve_error(void* base, int n1, int n2, int n3, int R, size_t* bytes) {
  using C = cx_t<T>;
  const size_t h = n3 / 2 + 1;
  const dim3 g = error_grid(n1, n2, n3);
  Carver cv(base);
  ErrWs<T> w;
  w.Xh = cv.take<C>(h * n1 * n2);
  w.Uh = cv.take<C>(h * n1 * R);
  w.Vh = cv.take<C>(h * n2 * R);
  w.Sh = cv.take<C>(h * R);
  w.partial = cv.take<double>((size_t)g.x * g.y * g.z);
  if (bytes) *bytes = cv.bytes();
  return w;
}

template <typename T>
static int error_run(const T* X, const T* U, const T* S, const T* V, int n1, int n2, int n3, int R, double* err2,
                     void* ws, cudaStream_t s) {
  ErrWs<T> w = carve_error<T>(ws, n1, n2, n3, R, nullptr);
  TSVD_TRY(launch_rfft3<T>(X, w.Xh, (long)n1 * n2, n3, s));
  TSVD_TRY(launch_rfft3<T>(U, w.Uh, (long)n1 * R, n3, s));
  TSVD_TRY(launch_rfft3<T>(V, w.Vh, (long)n2 * R, n3, s));
  TSVD_TRY(launch_rfft3<T>(S, w.Sh, (long)R, n3, s));
  const dim3 g = error_grid(n1, n2, n3);
  {
    TSVD_STAGE("error_fused", s);
    k_fro_error<T><<<g, 256, 0, s>>>(w.Xh, w.Uh, w.Sh, w.Vh, n1, n2, R, n3, w.partial);
    TSVD_LAUNCHED();
  }
  k_sum_error_partials<<<1, 256, 0, s>>>(w.partial, (long)g.x * g.y * g.z, err2);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

static int error_check(int n1, int n2, int n3, int R, int precision) {
  if (n1 < 1 || n2 < 1 || n3 < 1 || R < 1) return TSVD_ERR_INVALID_ARG;
  if (precision < TSVD_FP64 || precision > TSVD_MIXED_BF16) return TSVD_ERR_INVALID_ARG;
  if (n3 / 2 + 1 > 65535) return TSVD_ERR_UNSUPPORTED;
  return TSVD_OK;
}

}  // namespace tsvd

using namespace tsvd;

extern "C" int tsvd_error_workspace_size(int n1, int n2, int n3, int R, int precision, size_t* bytes) {
  if (!bytes) return TSVD_ERR_INVALID_ARG;
  TSVD_TRY(error_check(n1, n2, n3, R, precision));
  if (precision == TSVD_FP64) carve_error<double>(nullptr, n1, n2, n3, R, bytes);
  else carve_error<float>(nullptr, n1, n2, n3, R, bytes);
  return TSVD_OK;
}

extern "C" int tsvd_error(const void* X, const void* U, const void* S, const void* V, int n1, int n2, int n3, int R,
                          int precision, double* err2, void* ws, size_t ws_bytes, void* stream) {
  if (!X || !U || !S || !V || !err2 || !ws) return TSVD_ERR_INVALID_ARG;
  size_t need = 0;
  TSVD_TRY(tsvd_error_workspace_size(n1, n2, n3, R, precision, &need));
  if (ws_bytes < need) return TSVD_ERR_WORKSPACE;
  if (((uintptr_t)ws & 255) != 0) return TSVD_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == TSVD_FP64)
    return error_run<double>((const double*)X, (const double*)U, (const double*)S, (const double*)V, n1, n2, n3, R,
                             err2, ws, s);
  return error_run<float>((const float*)X, (const float*)U, (const float*)S, (const float*)V, n1, n2, n3, R, err2, ws,
                          s);
}
