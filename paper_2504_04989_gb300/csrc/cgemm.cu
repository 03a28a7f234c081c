// cgemm.cu -- batched complex GEMM on the SIMT FP64 / FP32 pipes.
//
// One CTA computes a 64 x 64 tile of one slice's product with 256 threads,
// each holding a 4 x 4 complex register tile (rows ty + 16 i, columns
// tx + 16 j, so a warp's shared-memory reads are contiguous).  op(A) and op(B)
// tiles are staged in shared memory k-major, in two stages: the next k-tile is
// loaded into registers while the current one is multiplied; the conjugate
// transpose is taken while staging, reading the stored matrix along its
// contiguous dimension.
// Thin products (long K, small M x N) split K across CTAs and reduce the
// partial tiles in a fixed order (deterministic, no atomics).
#include "common.cuh"
#include "kernels.cuh"

namespace tsvd {

template <typename C>
struct GemmCfg;
template <>
struct GemmCfg<double2> {
  static constexpr int BK = 8;
  using R = double;
};
template <>
struct GemmCfg<float2> {
  static constexpr int BK = 16;
  using R = float;
};

constexpr int GBM = 64, GBN = 64;

template <typename C, bool AH, bool BH>
__global__ void __launch_bounds__(256) k_cgemm(GemmArgs g, C* __restrict__ ws, int ksplit, int kchunk, int tiles_m,
                                               int herm_upper) {
  constexpr int BK = GemmCfg<C>::BK;
  constexpr int NA = GBM * BK / 256, NB = GBN * BK / 256;  // staged elements per thread
  using R = typename GemmCfg<C>::R;
  // two stages; rows padded by one element so the transposed stores hit distinct banks
  __shared__ __align__(16) C As[2][BK][GBM + 1];
  __shared__ __align__(16) C Bs[2][BK][GBN + 1];
  const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
  if (herm_upper && tm > tn) return;  // Hermitian product: the lower tiles are mirrored afterwards
  const int bi = blockIdx.z / ksplit, kz = blockIdx.z % ksplit;
  const int m0 = tm * GBM, n0 = tn * GBN;
  const C* __restrict__ A = (const C*)g.A + (long)bi * g.sA;
  const C* __restrict__ B = (const C*)g.B + (long)bi * g.sB;
  const int kb = kz * kchunk, ke = min(g.K, kb + kchunk);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  C acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mkc(R(0), R(0));

  // the next k-tile is fetched into registers while the current one is multiplied
  C ra[NA], rb[NB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int t = 0; t < NA; ++t) {
      const int idx = tid + 256 * t;
      int mm, kk;
      if (!AH) { kk = idx % BK; mm = idx / BK; }
      else { mm = idx % GBM; kk = idx / GBM; }
      const int gm = m0 + mm, gk = k0 + kk;
      C v = mkc(R(0), R(0));
      if (gm < g.M && gk < ke) v = AH ? cconj(A[(long)gk * g.lda + gm]) : A[(long)gm * g.lda + gk];
      ra[t] = v;
    }
#pragma unroll
    for (int t = 0; t < NB; ++t) {
      const int idx = tid + 256 * t;
      int nn, kk;
      if (!BH) { nn = idx % GBN; kk = idx / GBN; }
      else { kk = idx % BK; nn = idx / BK; }
      const int gn = n0 + nn, gk = k0 + kk;
      C v = mkc(R(0), R(0));
      if (gn < g.N && gk < ke) v = BH ? cconj(B[(long)gn * g.ldb + gk]) : B[(long)gk * g.ldb + gn];
      rb[t] = v;
    }
  };
  auto stash = [&](int st) {
#pragma unroll
    for (int t = 0; t < NA; ++t) {
      const int idx = tid + 256 * t;
      if (!AH) As[st][idx % BK][idx / BK] = ra[t];
      else As[st][idx / GBM][idx % GBM] = ra[t];
    }
#pragma unroll
    for (int t = 0; t < NB; ++t) {
      const int idx = tid + 256 * t;
      if (!BH) Bs[st][idx / GBN][idx % GBN] = rb[t];
      else Bs[st][idx % BK][idx / BK] = rb[t];
    }
  };
  if (kb < ke) fetch(kb);
  int st = 0;
  for (int k0 = kb; k0 < ke; k0 += BK) {
    stash(st);
    __syncthreads();  // stage st complete; the stage written next was last read before this barrier
    if (k0 + BK < ke) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      C a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[st][kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[st][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
    }
    st ^= 1;
  }
  C* __restrict__ Cm = (C*)g.C + (long)bi * g.sC;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= g.N) continue;
      if (ksplit > 1) {
        ws[(((long)kz * g.batch + bi) * g.M + gm) * g.N + gn] = acc[i][j];
      } else {
        C r = cscale(acc[i][j], (R)g.alpha);
        if (g.beta != 0.0) r = cadd(r, cscale(Cm[(long)gm * g.ldc + gn], (R)g.beta));
        Cm[(long)gm * g.ldc + gn] = r;
      }
    }
  }
}

// FP32 (float2) products other than the Hermitian form: 128 x 64 tiles, each
// of the 256 threads holding an 8 x 4 complex register tile (rows 8 ty .. +7,
// columns 4 tx .. +3), read from shared memory in 16-byte pieces: 6 loads per
// 128 FMAs instead of 8 per 64.  Rows of the staged tiles are padded by 16
// bytes, which keeps the 16-byte reads aligned and spreads the transposed
// stores of consecutive k over distinct banks.  Same staging, split-K and
// epilogue as k_cgemm.
constexpr int WBM = 128, WBN = 64, WBK = 8, WPAD = 2;

template <bool AH, bool BH>
__global__ void __launch_bounds__(256, 2) k_cgemm_w(GemmArgs g, float2* __restrict__ ws, int ksplit, int kchunk,
                                                    int tiles_m) {
  constexpr int NA = WBM * WBK / 256, NB = WBN * WBK / 256;  // staged elements per thread
  __shared__ __align__(16) float2 As[2][WBK][WBM + WPAD];
  __shared__ __align__(16) float2 Bs[2][WBK][WBN + WPAD];
  const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
  const int bi = blockIdx.z / ksplit, kz = blockIdx.z % ksplit;
  const int m0 = tm * WBM, n0 = tn * WBN;
  const float2* __restrict__ A = (const float2*)g.A + (long)bi * g.sA;
  const float2* __restrict__ B = (const float2*)g.B + (long)bi * g.sB;
  const int kb = kz * kchunk, ke = min(g.K, kb + kchunk);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float2 acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  float2 ra[NA], rb[NB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int t = 0; t < NA; ++t) {
      const int idx = tid + 256 * t;
      int mm, kk;
      if (!AH) { kk = idx % WBK; mm = idx / WBK; }
      else { mm = idx % WBM; kk = idx / WBM; }
      const int gm = m0 + mm, gk = k0 + kk;
      float2 v = make_float2(0.f, 0.f);
      if (gm < g.M && gk < ke) v = AH ? cconj(A[(long)gk * g.lda + gm]) : A[(long)gm * g.lda + gk];
      ra[t] = v;
    }
#pragma unroll
    for (int t = 0; t < NB; ++t) {
      const int idx = tid + 256 * t;
      int nn, kk;
      if (!BH) { nn = idx % WBN; kk = idx / WBN; }
      else { kk = idx % WBK; nn = idx / WBK; }
      const int gn = n0 + nn, gk = k0 + kk;
      float2 v = make_float2(0.f, 0.f);
      if (gn < g.N && gk < ke) v = BH ? cconj(B[(long)gn * g.ldb + gk]) : B[(long)gk * g.ldb + gn];
      rb[t] = v;
    }
  };
  auto stash = [&](int st) {
#pragma unroll
    for (int t = 0; t < NA; ++t) {
      const int idx = tid + 256 * t;
      if (!AH) As[st][idx % WBK][idx / WBK] = ra[t];
      else As[st][idx / WBM][idx % WBM] = ra[t];
    }
#pragma unroll
    for (int t = 0; t < NB; ++t) {
      const int idx = tid + 256 * t;
      if (!BH) Bs[st][idx / WBN][idx % WBN] = rb[t];
      else Bs[st][idx % WBK][idx / WBK] = rb[t];
    }
  };
  if (kb < ke) fetch(kb);
  int st = 0;
  for (int k0 = kb; k0 < ke; k0 += WBK) {
    stash(st);
    __syncthreads();  // stage st complete; the stage written next was last read before this barrier
    if (k0 + WBK < ke) fetch(k0 + WBK);
#pragma unroll
    for (int kk = 0; kk < WBK; ++kk) {
      float2 a[8], b[4];
      const float4* ap = reinterpret_cast<const float4*>(&As[st][kk][8 * ty]);
      const float4* bp = reinterpret_cast<const float4*>(&Bs[st][kk][4 * tx]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 x = ap[u];
        a[2 * u] = make_float2(x.x, x.y);
        a[2 * u + 1] = make_float2(x.z, x.w);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float4 x = bp[u];
        b[2 * u] = make_float2(x.x, x.y);
        b[2 * u + 1] = make_float2(x.z, x.w);
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
    }
    st ^= 1;
  }
  float2* __restrict__ Cm = (float2*)g.C + (long)bi * g.sC;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gm = m0 + 8 * ty + i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + 4 * tx + j;
      if (gn >= g.N) continue;
      if (ksplit > 1) {
        ws[(((long)kz * g.batch + bi) * g.M + gm) * g.N + gn] = acc[i][j];
      } else {
        float2 r = cscale(acc[i][j], (float)g.alpha);
        if (g.beta != 0.0) r = cadd(r, cscale(Cm[(long)gm * g.ldc + gn], (float)g.beta));
        Cm[(long)gm * g.ldc + gn] = r;
      }
    }
  }
}

template <typename C>
__global__ void k_splitk_reduce(const C* __restrict__ ws, int ksplit, GemmArgs g) {
  using R = typename GemmCfg<C>::R;
  const long total = (long)g.batch * g.M * g.N;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int n = idx % g.N;
    const long r = idx / g.N;
    const int m = r % g.M;
    const int bi = r / g.M;
    C s = mkc(R(0), R(0));
    for (int kz = 0; kz < ksplit; ++kz) s = cadd(s, ws[(long)kz * total + idx]);
    C* Cm = (C*)g.C + (long)bi * g.sC + (long)m * g.ldc + n;
    C out = cscale(s, (R)g.alpha);
    if (g.beta != 0.0) out = cadd(out, cscale(*Cm, (R)g.beta));
    *Cm = out;
  }
}

int choose_ksplit(int M, int N, int K, int batch, size_t splitk_elems) {
  const long tiles = (long)cdiv(M, GBM) * cdiv(N, GBN) * batch;
  const long target = 2 * 152;
  int ks = (int)std::max(1L, std::min(16L, target / std::max(1L, tiles)));
  ks = std::min(ks, std::max(1, K / 64));
  while (ks > 1 && (size_t)ks * batch * M * N > splitk_elems) --ks;
  while (ks > 1 && (long)ks * batch > 65535) --ks;
  return ks;
}

// lower triangle of each slice's square C from the conjugate of the upper one
template <typename C>
__global__ void k_mirror_lower(C* __restrict__ Cm, long ldc, long sC, int n, int batch) {
  const long total = (long)batch * n * n;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int j = idx % n;
    const long t = idx / n;
    const int i = t % n;
    const int b = t / n;
    if (i > j) Cm[(long)b * sC + (long)i * ldc + j] = cconj(Cm[(long)b * sC + (long)j * ldc + i]);
  }
}

// k_cgemm_w over the FP32 product g: split-K until about two waves of two CTAs per SM
static int cgemm_wide(const GemmArgs& g, float2* ws, size_t splitk_elems, cudaStream_t s) {
  const long tiles = (long)cdiv(g.M, WBM) * cdiv(g.N, WBN) * g.batch;
  int ks = (int)std::max(1L, std::min(16L, (4L * 152 + tiles - 1) / tiles));
  ks = std::min(ks, std::max(1, g.K / 64));
  if (!ws) ks = 1;
  while (ks > 1 && (size_t)ks * g.batch * g.M * g.N > splitk_elems) --ks;
  while (ks > 1 && (long)ks * g.batch > 65535) --ks;
  int kchunk = (g.K + ks - 1) / ks;
  kchunk = (kchunk + WBK - 1) / WBK * WBK;
  if (kchunk == 0) kchunk = WBK;
  ks = std::max(1, (g.K + kchunk - 1) / kchunk);
  const int tiles_m = cdiv(g.M, WBM), tiles_n = cdiv(g.N, WBN);
  dim3 grid(tiles_m * tiles_n, 1, g.batch * ks);
  const bool ah = (g.opA == 'H'), bh = (g.opB == 'H');
  if (!ah && !bh) k_cgemm_w<false, false><<<grid, 256, 0, s>>>(g, ws, ks, kchunk, tiles_m);
  else if (ah && !bh) k_cgemm_w<true, false><<<grid, 256, 0, s>>>(g, ws, ks, kchunk, tiles_m);
  else if (!ah && bh) k_cgemm_w<false, true><<<grid, 256, 0, s>>>(g, ws, ks, kchunk, tiles_m);
  else k_cgemm_w<true, true><<<grid, 256, 0, s>>>(g, ws, ks, kchunk, tiles_m);
  TSVD_LAUNCHED();
  if (ks > 1) {
    const long total = (long)g.batch * g.M * g.N;
    k_splitk_reduce<float2><<<std::min<long>(cdiv(total, 256), 4096), 256, 0, s>>>(ws, ks, g);
    TSVD_LAUNCHED();
  }
  return TSVD_OK;
}

template <typename C>
static int cgemm_impl(const GemmArgs& g, void* splitk_ws, size_t splitk_elems, cudaStream_t s, int herm) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return TSVD_OK;
  if (g.batch > 65535) return TSVD_ERR_UNSUPPORTED;
  if (g.beta != 0.0 && g.beta != 1.0) return TSVD_ERR_INVALID_ARG;
  if constexpr (std::is_same<C, float2>::value) {
    // the wide tiles where they fill the GPU (two CTAs per SM), directly or by splitting a long K;
    // smaller products keep the 64 x 64 tiles (measured faster there)
    const long wtiles = (long)cdiv(g.M, WBM) * cdiv(g.N, WBN) * g.batch;
    if (!herm && g.K > 0 && (wtiles >= 2L * 152 || (g.K >= 1024 && splitk_ws)))
      return cgemm_wide(g, (float2*)splitk_ws, splitk_ws ? splitk_elems : 0, s);
  }
  int ks = (g.K > 0) ? choose_ksplit(g.M, g.N, g.K, g.batch, splitk_ws ? splitk_elems : 0) : 1;
  constexpr int BK = GemmCfg<C>::BK;
  int kchunk = (g.K + ks - 1) / ks;
  kchunk = (kchunk + BK - 1) / BK * BK;
  if (kchunk == 0) kchunk = BK;
  ks = (g.K + kchunk - 1) / kchunk;
  if (ks < 1) ks = 1;
  const int tiles_m = cdiv(g.M, GBM), tiles_n = cdiv(g.N, GBN);
  dim3 grid(tiles_m * tiles_n, 1, g.batch * ks);
  const bool ah = (g.opA == 'H'), bh = (g.opB == 'H');
  C* ws = (C*)splitk_ws;
  if (!ah && !bh) k_cgemm<C, false, false><<<grid, 256, 0, s>>>(g, ws, ks, kchunk, tiles_m, herm);
  else if (ah && !bh) k_cgemm<C, true, false><<<grid, 256, 0, s>>>(g, ws, ks, kchunk, tiles_m, herm);
  else if (!ah && bh) k_cgemm<C, false, true><<<grid, 256, 0, s>>>(g, ws, ks, kchunk, tiles_m, herm);
  else k_cgemm<C, true, true><<<grid, 256, 0, s>>>(g, ws, ks, kchunk, tiles_m, herm);
  TSVD_LAUNCHED();
  if (ks > 1) {
    const long total = (long)g.batch * g.M * g.N;
    k_splitk_reduce<C><<<std::min<long>(cdiv(total, 256), 4096), 256, 0, s>>>(ws, ks, g);
    TSVD_LAUNCHED();
  }
  if (herm) {
    const long total = (long)g.batch * g.M * g.M;
    k_mirror_lower<C><<<std::min<long>(cdiv(total, 256), 8192), 256, 0, s>>>((C*)g.C, g.ldc, g.sC, g.M, g.batch);
    TSVD_LAUNCHED();
  }
  return TSVD_OK;
}

template <typename C>
int cgemm(const GemmArgs& g, void* splitk_ws, size_t splitk_elems, cudaStream_t s) {
  return cgemm_impl<C>(g, splitk_ws, splitk_elems, s, 0);
}

template <typename C>
int cgemm_herm(const GemmArgs& g, void* splitk_ws, size_t splitk_elems, cudaStream_t s) {
  if (g.M != g.N || g.beta != 0.0) return TSVD_ERR_INVALID_ARG;
  return cgemm_impl<C>(g, splitk_ws, splitk_elems, s, 1);
}
template int cgemm_herm<double2>(const GemmArgs&, void*, size_t, cudaStream_t);
template int cgemm_herm<float2>(const GemmArgs&, void*, size_t, cudaStream_t);
template int cgemm<double2>(const GemmArgs&, void*, size_t, cudaStream_t);
template int cgemm<float2>(const GemmArgs&, void*, size_t, cudaStream_t);

// ---------------------------------------------------------------------------
template <typename S, typename D>
__global__ void k_convert(const S* __restrict__ src, long lds, long ss, D* __restrict__ dst, long ldd, long sd,
                          int rows, int cols, int batch) {
  const long total = (long)batch * rows * cols;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int c = idx % cols;
    const long r = idx / cols;
    const int row = r % rows;
    const int b = r / rows;
    const S v = src[(long)b * ss + (long)row * lds + c];
    D o;
    o.x = v.x;
    o.y = v.y;
    dst[(long)b * sd + (long)row * ldd + c] = o;
  }
}

template <typename S, typename D>
static int convert(const S* src, long lds, long ss, D* dst, long ldd, long sd, int rows, int cols, int batch,
                   cudaStream_t s) {
  const long total = (long)batch * rows * cols;
  if (total <= 0) return TSVD_OK;
  k_convert<S, D><<<std::min<long>(cdiv(total, 256), 8192), 256, 0, s>>>(src, lds, ss, dst, ldd, sd, rows, cols, batch);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

int convert_c64_to_c32(const double2* src, long lds, long ss, float2* dst, long ldd, long sd, int rows, int cols,
                       int batch, cudaStream_t s) {
  return convert(src, lds, ss, dst, ldd, sd, rows, cols, batch, s);
}
int convert_c32_to_c64(const float2* src, long lds, long ss, double2* dst, long ldd, long sd, int rows, int cols,
                       int batch, cudaStream_t s) {
  return convert(src, lds, ss, dst, ldd, sd, rows, cols, batch, s);
}
template <typename C>
int copy_cx(const C* src, long lds, long ss, C* dst, long ldd, long sd, int rows, int cols, int batch, cudaStream_t s) {
  return convert(src, lds, ss, dst, ldd, sd, rows, cols, batch, s);
}
template int copy_cx<double2>(const double2*, long, long, double2*, long, long, int, int, int, cudaStream_t);
template int copy_cx<float2>(const float2*, long, long, float2*, long, long, int, int, int, cudaStream_t);

}  // namespace tsvd
