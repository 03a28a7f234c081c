// gram_int.cu -- the Hermitian Gram G = C C^H of the small SVD of Alg. 2
// (T-SVD(C) through the eigenpairs of C C^H) on the FP32 path, summed exactly
// in integer arithmetic.
//
// C^H (n2 x m per slice) holds FP32 data.  Each column i is written as
// 2^(e_i - B) times a vector of integers of at most B+1 bits (one power of two
// per column, e_i the exponent of the column's largest component), which moves
// every entry by at most 2^(e_i - B - 1): a perturbation of C of the size of its
// own FP32 rounding.  The Gram of the scaled integers is then exact in 64-bit
// integer multiply-adds, and G_ij = 2^(e_i + e_j - 2B) sum_l conj(q_li) q_lj is
// rounded once, to FP64.  An FP32 Gram would put rounding errors of the order
// eps32 ||C||^2 on the small eigenvalues sigma_i^2 the method keeps; this form
// keeps the error at the level of a perturbation of C itself, as the FP64 Gram
// does, while running on the integer pipe instead of GB300's narrow FP64 unit.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace tsvd {

// mantissa bits B: 2 products per component and n2 terms must stay below 2^63
static int gram_bits(int n2) {
  int lg = 0;
  while ((1L << lg) < n2) ++lg;
  return std::min(23, (61 - lg) / 2);
}

// columns of one slice in tiles of 32, 8 row groups per column: exponent of the
// column's largest |component| (max over the groups in shared memory), then
// the scaled integers (round to nearest even)
__global__ void __launch_bounds__(256) k_gram_quantize(const float2* __restrict__ CH, long ldc, long sC, int n2,
                                                       int m, int B, int2* __restrict__ Q, int* __restrict__ colexp) {
  __shared__ float smx[8][32];
  const int cx = threadIdx.x & 31, ry = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + cx;
  const int k = blockIdx.y;
  const bool ok = i < m;
  const float2* src = CH + (long)k * sC + i;
  float mx = 0.0f;
  if (ok)
    for (int l = ry; l < n2; l += 8) {
      const float2 x = src[(long)l * ldc];
      mx = fmaxf(mx, fmaxf(fabsf(x.x), fabsf(x.y)));
    }
  smx[ry][cx] = mx;
  __syncthreads();
  float cm = 0.0f;
#pragma unroll
  for (int r = 0; r < 8; ++r) cm = fmaxf(cm, smx[r][cx]);
  if (!ok) return;
  int e = 0;
  if (cm > 0.0f) frexpf(cm, &e);  // cm < 2^e
  if (ry == 0) colexp[(long)k * m + i] = e;
  if (!Q) return;  // the exponents only (the sliced form quantizes as it writes its digits)
  int2* dst = Q + (long)k * n2 * m + i;
  for (int l = ry; l < n2; l += 8) {
    const float2 x = src[(long)l * ldc];
    dst[(long)l * m] = make_int2((int)rintf(ldexpf(x.x, B - e)), (int)rintf(ldexpf(x.y, B - e)));
  }
}

// ---------------------------------------------------------------------------
// The same exact Gram on the BF16 tensor cores.  Every integer q (|q| <= 2^B,
// B <= 23) is split into four signed base-64 digits, q = sum_s d_s 64^(3-s),
// |d_s| <= 63: exact in BF16, and a digit product summed over n2 <= 4096 terms
// stays below 2^24, so the FP32 accumulation of the tensor cores adds exact
// integers and is exact.  The digits of the real and imaginary parts of every
// column i of C^H are rows s 2m + 2i (real) and s 2m + 2i + 1 (imaginary) of D
// (8m x n2 per slice), P = D D^T holds all 16 digit pairs (s, t) of the
// de-interleaved real products, and
//   sum_l conj(q_li) q_lj = sum_(s,t) 64^(6-s-t) (P[2i][2j] + P[2i+1][2j+1]
//                                  + i (P[2i][2j+1] - P[2i+1][2j]))   (block s, t)
// is summed in 64-bit integers and rounded once, as above: G is bitwise the
// integer kernel's.
// ---------------------------------------------------------------------------
constexpr int GS_DIGITS = 4, GS_DBITS = 6;

// digits of the quantized C^H: 32 columns x 32 rows of C^H per block, transposed
// through shared memory so that the rows of D are written along l
__global__ void k_gram_digits(const float2* __restrict__ CH, long ldc, long sC, int n2, int m, int B,
                              const int* __restrict__ colexp, __nv_bfloat16* __restrict__ D, long ldd, long sD) {
  __shared__ int2 t[32][33];
  const int b = blockIdx.z, i0 = blockIdx.x * 32, l0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int rr = ty; rr < 32; rr += blockDim.y) {
    const int l = l0 + rr, i = i0 + tx;
    int2 q = make_int2(0, 0);
    if (l < n2 && i < m) {
      const float2 x = CH[(long)b * sC + (long)l * ldc + i];
      const int sh = B - colexp[(long)b * m + i];
      q = make_int2((int)rintf(ldexpf(x.x, sh)), (int)rintf(ldexpf(x.y, sh)));
    }
    t[rr][tx] = q;
  }
  __syncthreads();
  __nv_bfloat16* Db = D + (long)b * sD;
  for (int cc = ty; cc < 32; cc += blockDim.y) {
    const int i = i0 + cc, l = l0 + tx;
    if (i >= m || l >= n2) continue;
    const int2 q = t[tx][cc];
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      const int v = part ? q.y : q.x;
      const int mag = v < 0 ? -v : v;
#pragma unroll
      for (int sd = 0; sd < GS_DIGITS; ++sd) {
        const int d = (mag >> (GS_DBITS * (GS_DIGITS - 1 - sd))) & ((1 << GS_DBITS) - 1);
        Db[(long)(sd * 2 * m + 2 * i + part) * ldd + l] = __int2bfloat16_rn(v < 0 ? -d : d);
      }
    }
  }
}

// G_ij from the 16 digit-pair blocks of P (exact integers in FP32), summed in 64 bits
// (P holds only the tiles of 128 rows x bn columns not wholly below its diagonal; an
// element of a skipped tile is read at its transposed place, whose tile is always there)
__global__ void k_gram_combine(const float* __restrict__ P, long ldp, long sP, int m, int B,
                               const int* __restrict__ colexp, double2* __restrict__ G, long ldg, long sG,
                               int batch, int bn) {
  const long total = (long)batch * m * m;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int j = idx % m;
    const long r = idx / m;
    const int i = r % m;
    const int b = r / m;
    const float* Pb = P + (long)b * sP;
    long long re = 0, im = 0;
#pragma unroll
    for (int sd = 0; sd < GS_DIGITS; ++sd)
#pragma unroll
      for (int td = 0; td < GS_DIGITS; ++td) {
        const int a = sd * 2 * m + 2 * i, c = td * 2 * m + 2 * j;  // the even-aligned 2 x 2 block (a, c)
        float q00, q01, q10, q11;
        if ((c / bn + 1) * bn <= (a / 128) * 128) {  // its tile was skipped: P is symmetric
          const float* t0 = Pb + (long)c * ldp + a;
          const float* t1 = t0 + ldp;
          q00 = t0[0];
          q01 = t1[0];
          q10 = t0[1];
          q11 = t1[1];
        } else {
          const float* p0 = Pb + (long)a * ldp + c;
          const float* p1 = p0 + ldp;
          q00 = p0[0];
          q01 = p0[1];
          q10 = p1[0];
          q11 = p1[1];
        }
        const long long w = 1LL << (GS_DBITS * (2 * GS_DIGITS - 2 - sd - td));
        re += ((long long)q00 + (long long)q11) * w;
        im += ((long long)q01 - (long long)q10) * w;
      }
    const int sc = colexp[(long)b * m + i] + colexp[(long)b * m + j] - 2 * B;
    G[(long)b * sG + (long)i * ldg + j] = make_double2(ldexp((double)re, sc), ldexp((double)im, sc));
  }
}

constexpr int GI_TILE = 64;
constexpr int GI_KC = 16;

// Upper-triangle tiles (ti <= tj) of G per slice; each thread 4 x 4 entries
// with 64-bit accumulators; the tile and its conjugate transpose are written.
__global__ void __launch_bounds__(256) k_gram_int(const int2* __restrict__ Q, const int* __restrict__ colexp, int n2,
                                                  int m, int B, double2* __restrict__ G, long ldg, long sG) {
  __shared__ int2 Qa[GI_KC][GI_TILE];
  __shared__ int2 Qb[GI_KC][GI_TILE];
  const int nt = (m + GI_TILE - 1) / GI_TILE;
  int ti = 0, rem = blockIdx.x;
  while (rem >= nt - ti) {
    rem -= nt - ti;
    ++ti;
  }
  const int tj = ti + rem;
  const int k = blockIdx.y;
  const int i0 = ti * GI_TILE, j0 = tj * GI_TILE;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int2* Qk = Q + (long)k * n2 * m;
  long long re[4][4], im[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) re[a][b] = im[a][b] = 0;
  for (int l0 = 0; l0 < n2; l0 += GI_KC) {
    for (int e = threadIdx.x; e < GI_KC * GI_TILE; e += 256) {
      const int ll = e / GI_TILE, c = e % GI_TILE, l = l0 + ll;
      const bool lok = l < n2;
      Qa[ll][c] = (lok && i0 + c < m) ? Qk[(long)l * m + i0 + c] : make_int2(0, 0);
      Qb[ll][c] = (lok && j0 + c < m) ? Qk[(long)l * m + j0 + c] : make_int2(0, 0);
    }
    __syncthreads();
#pragma unroll 4
    for (int ll = 0; ll < GI_KC; ++ll) {
      int2 a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Qa[ll][ty + 16 * u];
#pragma unroll
      for (int u = 0; u < 4; ++u) b[u] = Qb[ll][tx + 16 * u];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int nai = -a[u].y;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          // conj(a) b = (ar br + ai bi) + i (ar bi - ai br)
          re[u][v] += (long long)a[u].x * b[v].x;
          re[u][v] += (long long)a[u].y * b[v].y;
          im[u][v] += (long long)a[u].x * b[v].y;
          im[u][v] += (long long)nai * b[v].x;
        }
      }
    }
    __syncthreads();
  }
  const int* ek = colexp + (long)k * m;
  double2* Gk = G + (long)k * sG;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + ty + 16 * u;
    if (i >= m) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = j0 + tx + 16 * v;
      if (j >= m) continue;
      const int sc = ek[i] + ek[j] - 2 * B;
      const double2 g = make_double2(ldexp((double)re[u][v], sc), ldexp((double)im[u][v], sc));
      Gk[(long)i * ldg + j] = g;
      if (ti != tj) Gk[(long)j * ldg + i] = make_double2(g.x, -g.y);
    }
  }
}

int gram_int_fp32(const float2* CH, long ldc, long sC, int n2, int m, int batch, int2* Q, int* colexp, double2* G,
                  long ldg, long sG, cudaStream_t s) {
  if (n2 <= 0 || m <= 0 || batch <= 0) return TSVD_OK;
  if (batch > 65535) return TSVD_ERR_UNSUPPORTED;
  const int B = gram_bits(n2);
  k_gram_quantize<<<dim3(cdiv(m, 32), batch), 256, 0, s>>>(CH, ldc, sC, n2, m, B, Q, colexp);
  TSVD_LAUNCHED();
  const int nt = cdiv(m, GI_TILE);
  k_gram_int<<<dim3(nt * (nt + 1) / 2, batch), 256, 0, s>>>(Q, colexp, n2, m, B, G, ldg, sG);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

// the sliced form: for n2 <= 4096 (the digit products' sums stay below 2^24)
bool gram_sliced_ok(int n2, int m) { return n2 >= 1 && n2 <= 4096 && m >= 1 && 8L * m <= 65535; }
long gram_sliced_ldd(int n2) { return (n2 + 7) / 8 * 8; }
size_t gram_sliced_bytes(int n2, int m, int batch) {
  return (size_t)batch * 8 * m * gram_sliced_ldd(n2) * sizeof(__nv_bfloat16) +
         (size_t)batch * 64 * m * m * sizeof(float) + 512;
}

int gram_sliced_fp32(const float2* CH, long ldc, long sC, int n2, int m, int batch, int* colexp, void* ws,
                     double2* G, long ldg, long sG, int* err, cudaStream_t s) {
  if (n2 <= 0 || m <= 0 || batch <= 0) return TSVD_OK;
  if (batch > 65535 || !gram_sliced_ok(n2, m)) return TSVD_ERR_UNSUPPORTED;
  const int B = gram_bits(n2);
  const long ldd = gram_sliced_ldd(n2), sD = 8L * m * ldd, sP = 64L * m * m;
  __nv_bfloat16* D = (__nv_bfloat16*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  float* P = (float*)(((uintptr_t)(D + (size_t)batch * sD) + 255) & ~(uintptr_t)255);
  k_gram_quantize<<<dim3(cdiv(m, 32), batch), 256, 0, s>>>(CH, ldc, sC, n2, m, B, nullptr, colexp);
  TSVD_LAUNCHED();
  k_gram_digits<<<dim3(cdiv(m, 32), cdiv(n2, 32), batch), dim3(32, 8), 0, s>>>(CH, ldc, sC, n2, m, B, colexp, D,
                                                                              ldd, sD);
  TSVD_LAUNCHED();
  TSVD_TRY(tc_gemm(D, ldd, sD, 8 * m, D, ldd, sD, 8 * m, n2, P, 8L * m, sP, batch, true, err, s, true));
  const int bn = tc_gemm_tile_n(8 * m, true);
  const long total = (long)batch * m * m;
  k_gram_combine<<<(unsigned)std::min<long>(cdiv(total, 256), 8192), 256, 0, s>>>(P, 8L * m, sP, m, B, colexp, G,
                                                                                  ldg, sG, batch, bn);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

}  // namespace tsvd
