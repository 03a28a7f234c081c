// cholqr.cu -- block orthonormalisation pieces of the Krylov basis (the T-QR
// step of Alg. 2, per Fourier slice): Cholesky of a Gram matrix (optionally
// shifted), the right triangular solve W <- W R^{-1}, and the replacement of
// numerically dependent columns by fresh orthonormal directions.
//
// The Gram matrix and the triangular solve run in the precision of the basis
// (FP64, or FP32 on the FP32 / mixed paths); the small Cholesky itself always
// runs in FP64.
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace tsvd {

__device__ __forceinline__ int pidx(int i, int j, int n) { return i * n - (i * (i - 1)) / 2 + (j - i); }

// ---------------------------------------------------------------------------
// Cholesky (upper, right-looking) R^H R = G + s I of one nb x nb Gram matrix
// per CTA, in FP64 from a Gram of either precision.  s = shift_rel * trace(G).
// Pivot test: shifted pass -> dead iff d_j <= 0; plain pass -> dead iff
// d_j <= dead_rel * G_jj.  Dead columns get R_jj = 1 and R_jk = 0.
// ---------------------------------------------------------------------------
template <typename GC>
__global__ void __launch_bounds__(256) k_chol_upper(const GC* __restrict__ G, long ldg, long sG,
                                                    double2* __restrict__ Rm, long ldr, long sR, int nb,
                                                    double shift_rel, double dead_rel,
                                                    uint32_t* __restrict__ dead_out) {
  extern __shared__ __align__(16) double2 S[];  // packed upper triangle
  __shared__ double dg[128];
  __shared__ double red[16];
  __shared__ uint32_t dmask[4];
  __shared__ double rjj;
  __shared__ int isdead;
  const int b = blockIdx.x, tid = threadIdx.x;
  G += (long)b * sG;
  Rm += (long)b * sR;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e - i * nb;
    if (j >= i) S[pidx(i, j, nb)] = to_c64(G[(long)i * ldg + j]);
  }
  if (tid < nb) dg[tid] = (double)G[(long)tid * ldg + tid].x;
  if (tid < 4) dmask[tid] = 0;
  __syncthreads();
  const double trace = block_sum(tid < nb ? dg[tid] : 0.0, red);
  const double sft = (shift_rel > 0.0) ? shift_rel * trace : 0.0;
  if (tid < nb) S[pidx(tid, tid, nb)].x += sft;
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {
      const double d = S[pidx(j, j, nb)].x;
      const bool dead = (shift_rel > 0.0) ? !(d > 0.0) : !(d > dead_rel * dg[j]);
      isdead = dead;
      rjj = dead ? 1.0 : sqrt(d);
      if (dead) dmask[j >> 5] |= 1u << (j & 31);
    }
    __syncthreads();
    const double r = rjj;
    const bool dead = isdead;
    for (int k = j + 1 + tid; k < nb; k += blockDim.x) {
      const int p = pidx(j, k, nb);
      S[p] = dead ? make_double2(0, 0) : cscale(S[p], 1.0 / r);
    }
    if (tid == 0) S[pidx(j, j, nb)] = make_double2(r, 0);
    __syncthreads();
    // trailing update S(i, k) -= conj(S(j, i)) S(j, k) for j < i <= k, one warp per row i
    const int lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    const int offj = pidx(j, j, nb);
    for (int i = j + 1 + warp; i < nb; i += nwarp) {
      const double2 a = S[offj + (i - j)];
      const int offi = pidx(i, i, nb);
      for (int k = i + lane; k < nb; k += 32) {
        const double2 c = S[offj + (k - j)];
        double2 t = S[offi + (k - i)];
        t.x = fma(-a.x, c.x, t.x);
        t.x = fma(-a.y, c.y, t.x);
        t.y = fma(-a.x, c.y, t.y);
        t.y = fma(a.y, c.x, t.y);
        S[offi + (k - i)] = t;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, k = e - i * nb;
    Rm[(long)i * ldr + k] = (k >= i) ? S[pidx(i, k, nb)] : make_double2(0, 0);
  }
  if (tid < 4) dead_out[b * 4 + tid] = dmask[tid];
}

template <typename GC>
int chol_upper(const GC* G, long ldg, long sG, double2* Rm, long ldr, long sR, int nb, int batch, double shift_rel,
               double dead_rel, uint32_t* dead, cudaStream_t s) {
  if (nb <= 0 || batch <= 0) return TSVD_OK;
  if (nb > 128) return TSVD_ERR_UNSUPPORTED;
  const size_t smem = (size_t)nb * (nb + 1) / 2 * sizeof(double2);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_chol_upper<GC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_chol_upper<GC><<<batch, 256, smem, s>>>(G, ldg, sG, Rm, ldr, sR, nb, shift_rel, dead_rel, dead);
  TSVD_LAUNCHED();
  return TSVD_OK;
}
template int chol_upper<double2>(const double2*, long, long, double2*, long, long, int, int, double, double,
                                 uint32_t*, cudaStream_t);
template int chol_upper<float2>(const float2*, long, long, double2*, long, long, int, int, double, double, uint32_t*,
                                cudaStream_t);

// ---------------------------------------------------------------------------
// W <- W R^{-1}: each thread owns one row x of its CTA's tile and solves
// x R = w column by column in right-looking order (x_j = w_j / R_jj, then
// w_k -= x_j R_jk for every k > j: independent updates, so the FMA pipe stays
// busy).  R (packed, in W's precision) and the rows live in shared memory.
// ---------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(64) k_trsm_right_upper(C* __restrict__ W, long ldw, long sW,
                                                               const double2* __restrict__ Rm, long ldr, long sR,
                                                               int n1, int nb, const uint32_t* __restrict__ dead) {
  using R = decltype(C().x);
  extern __shared__ __align__(16) unsigned char smraw[];
  C* Rp = (C*)smraw;                       // packed upper, nb(nb+1)/2; diagonal holds 1/R_jj
  C* Ws = Rp + nb * (nb + 1) / 2;          // [rows][nb + 1], rows = blockDim.x
  const int b = blockIdx.y, tid = threadIdx.x, rows = blockDim.x;
  const int r0 = blockIdx.x * rows;
  W += (long)b * sW;
  Rm += (long)b * sR;
  uint32_t dm[4];
#pragma unroll
  for (int w = 0; w < 4; ++w) dm[w] = dead[b * 4 + w];
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
  const int ld = nb + 1;
  for (int e = tid; e < rows * nb; e += blockDim.x) {
    const int r = e / nb, j = e - r * nb;
    C v;
    v.x = R(0);
    v.y = R(0);
    if (r0 + r < n1) v = W[(long)(r0 + r) * ldw + j];
    Ws[r * ld + j] = v;
  }
  __syncthreads();
  C* x = Ws + tid * ld;
  for (int j = 0; j < nb; ++j) {
    const C xj = cscale(x[j], Rp[pidx(j, j, nb)].x);  // dead columns: scale 0
    x[j] = xj;
    for (int k = j + 1; k < nb; ++k) {
      const C rjk = Rp[pidx(j, k, nb)];
      C t = x[k];
      t.x -= xj.x * rjk.x - xj.y * rjk.y;
      t.y -= xj.x * rjk.y + xj.y * rjk.x;
      x[k] = t;
    }
  }
  __syncthreads();
  for (int e = tid; e < rows * nb; e += blockDim.x) {
    const int r = e / nb, j = e - r * nb;
    if (r0 + r < n1) W[(long)(r0 + r) * ldw + j] = Ws[r * ld + j];
  }
}

template <typename C>
int trsm_right_upper(C* W, long ldw, long sW, const double2* Rm, long ldr, long sR, int n1, int nb, int batch,
                     const uint32_t* dead, cudaStream_t s) {
  if (nb <= 0 || n1 <= 0 || batch <= 0) return TSVD_OK;
  if (nb > 128) return TSVD_ERR_UNSUPPORTED;
  int rows = 64;
  size_t smem = ((size_t)nb * (nb + 1) / 2 + (size_t)rows * (nb + 1)) * sizeof(C);
  if (smem > 200 * 1024) {
    rows = 32;
    smem = ((size_t)nb * (nb + 1) / 2 + (size_t)rows * (nb + 1)) * sizeof(C);
  }
  if (smem > 227 * 1024) return TSVD_ERR_UNSUPPORTED;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_trsm_right_upper<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid(cdiv(n1, rows), batch);
  k_trsm_right_upper<C><<<grid, rows, smem, s>>>(W, ldw, sW, Rm, ldr, sR, n1, nb, dead);
  TSVD_LAUNCHED();
  return TSVD_OK;
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
