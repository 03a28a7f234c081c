// cholqr.cu -- block orthonormalisation pieces of the Krylov basis (the T-QR
// step of Alg. 2, per Fourier slice): Cholesky of a Gram matrix (optionally
// shifted), the right triangular solve W <- W R^{-1}, and the replacement of
// numerically dependent columns by fresh orthonormal directions.
//
// The Gram matrix, its Cholesky factorisation and the triangular solve all run
// in the precision of the basis (FP64, or FP32 on the FP32 / mixed paths), as
// in the analysis of shifted CholeskyQR (Fukaya et al.), which takes every step
// in the working precision.
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace tsvd {

__device__ __forceinline__ int pidx(int i, int j, int n) { return i * n - (i * (i - 1)) / 2 + (j - i); }

// ---------------------------------------------------------------------------
// Cholesky (upper, right-looking) R^H R = G + s I of one nb x nb Gram matrix
// per CTA, in the Gram's own precision.  s = shift_rel * trace(G).
// Pivot test: shifted pass -> dead iff d_j <= 0; plain pass -> dead iff
// d_j <= dead_rel * G_jj.  Dead columns get R_jj = 1 and R_jk = 0.
// One barrier per column: the scaling of row j is folded into the trailing
// update S(i,k) -= conj(S(j,i)) S(j,k) / d_j, and row j is scaled by
// 1/sqrt(d_j) at the end.
// ---------------------------------------------------------------------------
template <typename GC>
__global__ void __launch_bounds__(512) k_chol_upper(const GC* __restrict__ G, long ldg, long sG,
                                                    double2* __restrict__ Rm, long ldr, long sR, int nb,
                                                    double shift_rel, double dead_rel,
                                                    uint32_t* __restrict__ dead_out) {
  using Rt = decltype(GC().x);
  extern __shared__ __align__(16) unsigned char chsm[];
  const int np = nb * (nb + 1) / 2;
  GC* S = (GC*)chsm;                                  // packed upper triangle
  unsigned char* rowof = (unsigned char*)(S + np);    // row of each packed index (nb <= 128)
  __shared__ Rt dg[128];      // diagonal of G (pivot test of the plain passes)
  __shared__ Rt dj[128];      // pivots d_j (0 for a dead column)
  __shared__ double red[16];
  const int b = blockIdx.x, tid = threadIdx.x;
  G += (long)b * sG;
  Rm += (long)b * sR;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e - i * nb;
    if (j >= i) {
      S[pidx(i, j, nb)] = G[(long)i * ldg + j];
      rowof[pidx(i, j, nb)] = (unsigned char)i;
    }
  }
  if (tid < nb) dg[tid] = G[(long)tid * ldg + tid].x;
  __syncthreads();
  const double trace = block_sum(tid < nb ? (double)dg[tid] : 0.0, red);
  const Rt sft = (shift_rel > 0.0) ? (Rt)(shift_rel * trace) : Rt(0);
  if (tid < nb) S[pidx(tid, tid, nb)].x += sft;
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    const int offj = pidx(j, j, nb);
    const Rt d = S[offj].x;
    const bool dead = (shift_rel > 0.0) ? !(d > Rt(0)) : !(d > (Rt)dead_rel * dg[j]);
    if (tid == 0) dj[j] = dead ? Rt(0) : d;
    if (!dead && j + 1 < nb) {
      // trailing triangle (rows i > j) = the packed suffix from pidx(j+1, j+1), flattened over the CTA
      const Rt inv = Rt(1) / d;
      for (int p = pidx(j + 1, j + 1, nb) + tid; p < np; p += blockDim.x) {
        const int i = rowof[p];
        const int k = p - pidx(i, i, nb) + i;
        GC a = S[offj + (i - j)];  // S(j, i); the update uses conj(a) / d
        const GC cjk = S[offj + (k - j)];
        a.x *= inv;
        a.y *= inv;
        GC t = S[p];
        t.x = fma(-a.x, cjk.x, t.x);
        t.x = fma(-a.y, cjk.y, t.x);
        t.y = fma(-a.x, cjk.y, t.y);
        t.y = fma(a.y, cjk.x, t.y);
        S[p] = t;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, k = e - i * nb;
    double2 r = make_double2(0, 0);
    const Rt d = dj[i];
    if (k == i) {
      r.x = (d > Rt(0)) ? sqrt((double)d) : 1.0;
    } else if (k > i && d > Rt(0)) {
      const double sc = 1.0 / sqrt((double)d);
      const GC v = S[pidx(i, k, nb)];
      r = make_double2((double)v.x * sc, (double)v.y * sc);
    }
    Rm[(long)i * ldr + k] = r;
  }
  if (tid < 4) {
    uint32_t msk = 0;
    for (int q = 0; q < 32; ++q) {
      const int jj = tid * 32 + q;
      if (jj < nb && !(dj[jj] > Rt(0))) msk |= 1u << q;
    }
    dead_out[b * 4 + tid] = msk;
  }
}

template <typename GC>
int chol_upper(const GC* G, long ldg, long sG, double2* Rm, long ldr, long sR, int nb, int batch, double shift_rel,
               double dead_rel, uint32_t* dead, cudaStream_t s) {
  if (nb <= 0 || batch <= 0) return TSVD_OK;
  if (nb > 128) return TSVD_ERR_UNSUPPORTED;
  const size_t np = (size_t)nb * (nb + 1) / 2;
  const size_t smem = np * sizeof(GC) + np;  // packed triangle + row table
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_chol_upper<GC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_chol_upper<GC><<<batch, 512, smem, s>>>(G, ldg, sG, Rm, ldr, sR, nb, shift_rel, dead_rel, dead);
  TSVD_LAUNCHED();
  return TSVD_OK;
}
template int chol_upper<double2>(const double2*, long, long, double2*, long, long, int, int, double, double,
                                 uint32_t*, cudaStream_t);
template int chol_upper<float2>(const float2*, long, long, double2*, long, long, int, int, double, double, uint32_t*,
                                cudaStream_t);

// ---------------------------------------------------------------------------
// W <- W R^{-1} by forward substitution x R = w, one warp per TS_ROWS rows of
// W: lane l keeps columns l, l+32, l+64, l+96 of its rows in registers; for
// each j the solved x_j is broadcast by a shuffle and every lane updates its
// columns k > j with R(j, k) (R packed in shared memory, diagonal stored as
// 1/R_jj, 0 for a dead column).
// ---------------------------------------------------------------------------
// rows per warp (more rows raise the registers past one wave of CTAs)
template <typename C>
constexpr int ts_rows() { return 4; }
constexpr int TS_WARPS = 8;

template <typename C, int NU>  // NU = ceil(nb / 32) column slots per lane
__global__ void __launch_bounds__(TS_WARPS * 32) k_trsm_right_upper(C* __restrict__ W, long ldw, long sW,
                                                                   const double2* __restrict__ Rm, long ldr, long sR,
                                                                   int n1, int nb, const uint32_t* __restrict__ dead) {
  using R = decltype(C().x);
  extern __shared__ __align__(16) unsigned char smraw[];
  C* Rp = (C*)smraw;  // packed upper, nb(nb+1)/2
  const int b = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  W += (long)b * sW;
  Rm += (long)b * sR;
  uint32_t dm[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) dm[q] = dead[b * 4 + q];
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e - i * nb;
    if (j < i) continue;
    const double2 v = Rm[(long)i * ldr + j];
    C out;
    if (j == i) {
      const bool isdead = (dm[j >> 5] >> (j & 31)) & 1u;
      out.x = isdead ? R(0) : (R)(1.0 / v.x);
      out.y = R(0);
    } else {
      out.x = (R)v.x;
      out.y = (R)v.y;
    }
    Rp[pidx(i, j, nb)] = out;
  }
  __syncthreads();
  constexpr int TS_ROWS = ts_rows<C>();
  const int r0 = (blockIdx.x * TS_WARPS + warp) * TS_ROWS;
  if (r0 >= n1) return;
  C x[TS_ROWS][NU];
#pragma unroll
  for (int r = 0; r < TS_ROWS; ++r)
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      const int k = lane + 32 * u;
      x[r][u] = (r0 + r < n1 && k < nb) ? W[(long)(r0 + r) * ldw + k] : C{R(0), R(0)};
    }
#pragma unroll
  for (int u = 0; u < NU; ++u) {
    for (int jj = 0; jj < 32; ++jj) {
      const int j = 32 * u + jj;
      if (j >= nb) break;
      const int offj = pidx(j, j, nb);
      const R rinv = Rp[offj].x;
      C xj[TS_ROWS];
#pragma unroll
      for (int r = 0; r < TS_ROWS; ++r) {
        xj[r].x = __shfl_sync(0xffffffffu, x[r][u].x, jj) * rinv;
        xj[r].y = __shfl_sync(0xffffffffu, x[r][u].y, jj) * rinv;
        if (lane == jj) x[r][u] = xj[r];
      }
#pragma unroll
      for (int v = u; v < NU; ++v) {
        const int k = lane + 32 * v;
        if (k > j && k < nb) {
          const C rjk = Rp[offj + (k - j)];
#pragma unroll
          for (int r = 0; r < TS_ROWS; ++r) {
            x[r][v].x -= xj[r].x * rjk.x - xj[r].y * rjk.y;
            x[r][v].y -= xj[r].x * rjk.y + xj[r].y * rjk.x;
          }
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < TS_ROWS; ++r)
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      const int k = lane + 32 * u;
      if (r0 + r < n1 && k < nb) W[(long)(r0 + r) * ldw + k] = x[r][u];
    }
}

template <typename C>
int trsm_right_upper(C* W, long ldw, long sW, const double2* Rm, long ldr, long sR, int n1, int nb, int batch,
                     const uint32_t* dead, cudaStream_t s) {
  if (nb <= 0 || n1 <= 0 || batch <= 0) return TSVD_OK;
  if (nb > 128) return TSVD_ERR_UNSUPPORTED;
  const size_t smem = (size_t)nb * (nb + 1) / 2 * sizeof(C);
  dim3 grid(cdiv(n1, ts_rows<C>() * TS_WARPS), batch);
  auto go = [&](auto kern) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return TSVD_ERR_CUDA;
    }
    kern<<<grid, TS_WARPS * 32, smem, s>>>(W, ldw, sW, Rm, ldr, sR, n1, nb, dead);
    TSVD_LAUNCHED();
    return TSVD_OK;
  };
  switch ((nb + 31) / 32) {
    case 1: return go(k_trsm_right_upper<C, 1>);
    case 2: return go(k_trsm_right_upper<C, 2>);
    case 3: return go(k_trsm_right_upper<C, 3>);
    default: return go(k_trsm_right_upper<C, 4>);
  }
}
template int trsm_right_upper<double2>(double2*, long, long, const double2*, long, long, int, int, int,
                                       const uint32_t*, cudaStream_t);
template int trsm_right_upper<float2>(float2*, long, long, const double2*, long, long, int, int, int,
                                      const uint32_t*, cudaStream_t);

// ---------------------------------------------------------------------------
// Dependent Krylov columns (exact low rank, zero data): replace column c+j by
// a Philox Gaussian direction (stream 3) projected twice against every other
// live column of the basis, then normalised.  Any orthonormal completion of
// span(K) leaves the Rayleigh-Ritz result of Alg. 2 optimal (eq. mn39).
// ---------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(256) k_repair_dead(C* __restrict__ Q, long ldq, long sQ, int n1, int c, int nb,
                                                     const uint32_t* __restrict__ dead, uint64_t seed, int block_id,
                                                     int* __restrict__ dead_count) {
  using R = decltype(C().x);
  __shared__ double red[32];
  const int b = blockIdx.x, tid = threadIdx.x;
  uint32_t dm[4];
  int ndead = 0;
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    dm[w] = dead[b * 4 + w];
    ndead += __popc(dm[w]);
  }
  if (ndead == 0) return;
  Q += (long)b * sQ;
  if (tid == 0) atomicAdd(dead_count, ndead);
  uint32_t pending[4] = {dm[0], dm[1], dm[2], dm[3]};
  for (int j = 0; j < nb; ++j) {
    if (!((dm[j >> 5] >> (j & 31)) & 1u)) continue;
    const int col = c + j;
    for (int attempt = 0; attempt < 4; ++attempt) {
      for (int i = tid; i < n1; i += blockDim.x) {
        const uint4 x = philox10(make_uint4((uint32_t)i, (uint32_t)col | ((uint32_t)attempt << 24),
                                            (uint32_t)block_id, 3u + ((uint32_t)b << 8)),
                                 (uint32_t)seed, (uint32_t)(seed >> 32));
        const double u1 = ((double)x.x + 1.0) * (1.0 / 4294967296.0);
        const double u2 = ((double)x.y + 1.0) * (1.0 / 4294967296.0);
        const double r = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        C v;
        v.x = (R)(r * cs);
        v.y = (R)(r * sn);
        Q[(long)i * ldq + col] = v;
      }
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {
        for (int l = 0; l < c + nb; ++l) {
          if (l == col) continue;
          if (l >= c && ((pending[(l - c) >> 5] >> ((l - c) & 31)) & 1u)) continue;
          double2 part = make_double2(0, 0);
          for (int i = tid; i < n1; i += blockDim.x)
            cfmac(part, to_c64(Q[(long)i * ldq + l]), to_c64(Q[(long)i * ldq + col]));
          const double2 dot = block_sum2(part, red);
          for (int i = tid; i < n1; i += blockDim.x) {
            double2 q = to_c64(Q[(long)i * ldq + col]);
            const double2 ql = to_c64(Q[(long)i * ldq + l]);
            q.x -= dot.x * ql.x - dot.y * ql.y;
            q.y -= dot.x * ql.y + dot.y * ql.x;
            Q[(long)i * ldq + col] = from_c64<C>(q);
          }
          __syncthreads();
        }
      }
      double part = 0;
      for (int i = tid; i < n1; i += blockDim.x) part += cabs2(to_c64(Q[(long)i * ldq + col]));
      const double nrm = sqrt(block_sum(part, red));
      const bool ok = nrm > 1e-3;
      for (int i = tid; i < n1; i += blockDim.x)
        Q[(long)i * ldq + col] = ok ? from_c64<C>(cscale(to_c64(Q[(long)i * ldq + col]), 1.0 / nrm))
                                    : from_c64<C>(make_double2(0, 0));
      __syncthreads();
      if (ok) break;
    }
    pending[j >> 5] &= ~(1u << (j & 31));
  }
}

template <typename C>
int repair_dead(C* Q, long ldq, long sQ, int n1, int c, int nb, const uint32_t* dead, int batch, uint64_t seed,
                int block_id, int* dead_count, cudaStream_t s) {
  if (nb <= 0 || batch <= 0) return TSVD_OK;
  k_repair_dead<C><<<batch, 256, 0, s>>>(Q, ldq, sQ, n1, c, nb, dead, seed, block_id, dead_count);
  TSVD_LAUNCHED();
  return TSVD_OK;
}
template int repair_dead<double2>(double2*, long, long, int, int, int, const uint32_t*, int, uint64_t, int, int*,
                                  cudaStream_t);
template int repair_dead<float2>(float2*, long, long, int, int, int, const uint32_t*, int, uint64_t, int, int*,
                                 cudaStream_t);

}  // namespace tsvd
