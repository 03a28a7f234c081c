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

// ---------------------------------------------------------------------------
// Cholesky (upper, right-looking) R^H R = G + s I of one nb x nb Gram matrix
// per CTA, in the Gram's own precision, s = shift_rel * trace(G), followed by
// the inverse M of R-tilde, written dense (zeros below the diagonal):
//   pivot test: shifted pass -> dead iff d_j <= 0; plain pass -> dead iff
//   d_j <= dead_rel * G_jj;
//   R-tilde: R with every dead row and every dead column replaced by the unit
//   vector (so R-tilde = diag(R_live, I) up to a permutation);
//   M: R-tilde^{-1} with the dead columns set to zero, so that W M is
//   W_live R_live^{-1} on the live columns and zero on the dead ones.
// Warp w keeps the entries [32 EPT w, 32 EPT (w+1)) of the packed upper
// triangle (row-major; lane-strided) in registers, so each step is one round
// of independent register updates between two barriers, and a warp whose rows
// are all finished skips the step:
//   factorisation, step j: S(i,k) -= conj(S(j,i)) S(j,k) / d_j for
//   j < i <= k, with row j read from shared memory, where its owners
//   published it when it became final (end of step j-1); the published rows
//   are R unscaled (row j is divided by sqrt(d_j) when read);
//   inverse, step l = nb-1 .. 1 (backward substitution R X = I for all
//   columns at once, B = I initially): B(i,k) -= R(i,l) X(l,k) for
//   i < l <= k, where X(l,k) = B(l,k) / R_ll, final after step l+1, is
//   published in a double-buffered row.
// ---------------------------------------------------------------------------
template <typename GC, int EPT, int NTHR>  // NTHR threads, EPT >= nb (nb+1) / 2 / NTHR entries per thread
__global__ void __launch_bounds__(NTHR) k_chol_inv(const GC* __restrict__ G, long ldg, long sG,
                                                       GC* __restrict__ Mo, long ldm, long sM, int nb,
                                                       double shift_rel, double dead_rel,
                                                       uint32_t* __restrict__ dead_out) {
  using Rt = decltype(GC().x);
  extern __shared__ __align__(16) unsigned char chsm[];
  GC* S = (GC*)chsm;               // published rows of the packed triangle: S(i, k) = S[rb(i) + k]
  GC* Xr = S + nb * (nb + 1) / 2;  // [2][nb] published rows of X
  __shared__ Rt dg[128];           // diagonal of G (pivot test of the plain passes)
  __shared__ Rt dj[128];           // pivots d_j (0 for a dead column)
  __shared__ Rt pinv[128];         // 1 / d_j (0 for a dead column)
  __shared__ Rt ri[128];           // 1 / R-tilde_jj
  __shared__ double red[NTHR / 32];
  const int b = blockIdx.x, tid = threadIdx.x;
  const int np = nb * (nb + 1) / 2;
  auto rb = [nb](int i) { return i * nb - (i * (i + 1)) / 2; };  // packed offset of row i, minus i
  G += (long)b * sG;
  Mo += (long)b * sM;
  if (tid < nb) dg[tid] = G[(long)tid * ldg + tid].x;
  // row of packed index p: largest i with rb(i) + i <= p (closed form in FP32 -- GB300's FP64
  // unit is narrow -- then corrected exactly)
  auto row_of = [&](int p) {
    const float q = 2.0f * nb + 1.0f;
    int i = (int)((q - sqrtf(fmaxf(q * q - 8.0f * p, 0.0f))) * 0.5f);
    i = max(0, min(i, nb - 1));
    while (i > 0 && rb(i) + i > p) --i;
    while (i + 1 < nb && rb(i + 1) + i + 1 <= p) ++i;
    return i;
  };
  // warp w owns the packed range [32 EPT w, 32 EPT (w+1)), lane-strided; its first and last
  // rows decide when it has nothing left to do (rows <= j in the factorisation, >= l in the inverse)
  const int warp = tid >> 5, lane = tid & 31;
  const int pw0 = 32 * EPT * warp, pw1 = min(pw0 + 32 * EPT, np) - 1;
  const int wrow0 = (pw0 < np) ? row_of(pw0) : nb, wrow1 = (pw0 < np) ? row_of(pw1) : -1;
  // owned entries: (row, column) (-1 if none), packed offset and value
  int ei[EPT], ek[EPT];  // the packed offset of entry e is pw0 + 32 e + lane (a constant per e)
  GC v[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int p = pw0 + 32 * e + lane;
    int i = -1, k = -1;
    if (p < np) {
      i = row_of(p);
      k = p - rb(i);
    }
    ei[e] = i;
    ek[e] = k;
    v[e] = (p < np) ? G[(long)i * ldg + k] : GC{Rt(0), Rt(0)};
  }
  __syncthreads();
  const double trace = block_sum(tid < nb ? (double)dg[tid] : 0.0, red);
  const Rt sft = (shift_rel > 0.0) ? (Rt)(shift_rel * trace) : Rt(0);
  // a final diagonal entry d_i: pivot test, published with its row
  auto pivot = [&](int i, Rt d) {
    const bool dead = (shift_rel > 0.0) ? !(d > Rt(0)) : !(d > (Rt)dead_rel * dg[i]);
    dj[i] = dead ? Rt(0) : d;
    pinv[i] = dead ? Rt(0) : Rt(1) / d;
  };
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    if (ei[e] >= 0 && ei[e] == ek[e]) v[e].x += sft;
    if (ei[e] == 0) {  // row 0 is final
      S[pw0 + 32 * e + lane] = v[e];
      if (ek[e] == 0) pivot(0, v[e].x);
    }
  }
  __syncthreads();
  // every step is branch-free: the operands of each entry are loaded whether or not it is
  // active (in-range addresses), and the update is selected
  for (int j = 0; j < nb; ++j) {
    const GC* Sj = S + rb(j);
    const Rt inv = pinv[j];
    if (wrow1 > j) {
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int i = ei[e], k = ek[e];
        const GC a = Sj[max(i, 0)];
        const GC c = Sj[max(k, 0)];
        const Rt ax = a.x * inv, ay = a.y * inv;  // conj(a) / d times c
        GC t = v[e];
        t.x = fma(-ax, c.x, t.x);
        t.x = fma(-ay, c.y, t.x);
        t.y = fma(-ax, c.y, t.y);
        t.y = fma(ay, c.x, t.y);
        if (i > j) v[e] = t;
        if (i == j + 1) {  // row j+1 is final
          S[pw0 + 32 * e + lane] = v[e];
          if (k == i) pivot(i, v[e].x);
        }
      }
    }
    __syncthreads();
  }
  if (tid < nb) ri[tid] = (dj[tid] > Rt(0)) ? Rt(1) / sqrt(dj[tid]) : Rt(1);
  __syncthreads();
  // inverse: B in the registers (0 above the diagonal, 1 on it); R-tilde(i, l) = R(i, l) / sqrt(d_i)
  // read from the published rows (0 where row i or column l is dead)
  Rt er[EPT];  // 1 / R-tilde_ii of the entry's row, 0 for a dead row
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int i = max(ei[e], 0);
    er[e] = (dj[i] > Rt(0)) ? ri[i] : Rt(0);
    v[e] = GC{Rt(0), Rt(0)};
  }
  for (int l = nb - 1; l >= 1; --l) {
    const GC* xl = Xr + (l & 1) * nb;  // X(l, k), k > l
    const Rt rl = ri[l];
    const bool live_l = dj[l] > Rt(0);
    if (wrow0 < l) {
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const int i = ei[e], k = ek[e];
        const int ic = max(i, 0), kc = max(k, 0);
        const GC cr = S[rb(ic) + l];
        const GC xv = xl[kc];
        const Rt sc = live_l ? er[e] : Rt(0);
        const Rt cx = cr.x * sc, cy = cr.y * sc;
        const GC x = (k == l) ? GC{rl, Rt(0)} : xv;
        GC t = v[e];
        t.x = fma(-cx, x.x, t.x);
        t.x = fma(cy, x.y, t.x);
        t.y = fma(-cx, x.y, t.y);
        t.y = fma(-cy, x.x, t.y);
        if (i >= 0 && i < l && k >= l) v[e] = t;
        if (i == l - 1 && k > i) {  // row l-1 of B is final: publish X(l-1, k)
          const Rt s2 = ri[i];
          Xr[((l - 1) & 1) * nb + k] = GC{v[e].x * s2, v[e].y * s2};
        }
      }
    }
    __syncthreads();
  }
  // M(i, k) = B(i, k) / R_ii (M(i, i) = 1 / R_ii); dead columns and the lower triangle zero
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int i = ei[e], k = ek[e];
    if (i < 0) continue;
    GC mv = GC{Rt(0), Rt(0)};
    if (dj[k] > Rt(0)) {
      if (k == i) {
        mv.x = ri[i];
      } else {
        mv.x = v[e].x * ri[i];
        mv.y = v[e].y * ri[i];
      }
    }
    Mo[(long)i * ldm + k] = mv;
  }
  for (int e = tid; e < nb * nb; e += NTHR) {
    const int i = e / nb, k = e - i * nb;
    if (k < i) Mo[(long)i * ldm + k] = GC{Rt(0), Rt(0)};
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
int chol_inv(const GC* G, long ldg, long sG, GC* M, long ldm, long sM, int nb, int batch, double shift_rel,
             double dead_rel, uint32_t* dead, cudaStream_t s) {
  if (nb <= 0 || batch <= 0) return TSVD_OK;
  if (nb > 128) return TSVD_ERR_UNSUPPORTED;
  const int np = nb * (nb + 1) / 2;
  const size_t smem = ((size_t)np + 2 * (size_t)nb) * sizeof(GC);  // published rows + X rows
  auto go = [&](auto kern, int nthr) {
    // with the kernel's static arrays (about 4 KB) the total passes the 48 KB default earlier
    if (smem > 40 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return TSVD_ERR_CUDA;
    }
    kern<<<batch, nthr, smem, s>>>(G, ldg, sG, M, ldm, sM, nb, shift_rel, dead_rel, dead);
    TSVD_LAUNCHED();
    return TSVD_OK;
  };
  // 512 threads (16 warps: a step's latency is hidden across warps; 128 threads with 16 entries
  // each measured twice as slow at nb = 60)
  if (np <= 2 * 512) return go(k_chol_inv<GC, 2, 512>, 512);
  if (np <= 4 * 512) return go(k_chol_inv<GC, 4, 512>, 512);
  if (np <= 8 * 512) return go(k_chol_inv<GC, 8, 512>, 512);
  // larger Grams up to 8192 packed entries (90 < nb <= 127), FP32: 1024 threads with 8 entries
  // each rather than 17 on 512 (each warp's chain of a step halves and twice the warps hide it;
  // FP64 spills at 1024 x 8)
  if constexpr (std::is_same<GC, float2>::value)
    if (np <= 8 * 1024) return go(k_chol_inv<GC, 8, 1024>, 1024);
  static_assert(17 * 512 >= 128 * 129 / 2, "the last variant covers every nb <= 128");
  return go(k_chol_inv<GC, 17, 512>, 512);
}
template int chol_inv<double2>(const double2*, long, long, double2*, long, long, int, int, double, double, uint32_t*,
                               cudaStream_t);
template int chol_inv<float2>(const float2*, long, long, float2*, long, long, int, int, double, double, uint32_t*,
                              cudaStream_t);

// asynchronous global -> shared copy of one complex element (8 or 16 bytes)
template <typename C>
__device__ __forceinline__ void cp_async_elem(C* dst, const C* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(C) == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src));
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(src));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---------------------------------------------------------------------------
// O <- W M for the n1 x nb block of every slice (M nb x nb, upper
// triangular, dense): a CTA stages TM_ROWS full rows of W and, kchunk rows at
// a time, M in shared memory (all of M at once when it fits); thread
// (ty, tx) accumulates rows ty + 16a (a < 4) and columns tx + 16u in
// registers; column group u takes no terms from rows k >= 16 (u + 1).
// ---------------------------------------------------------------------------
constexpr int TM_ROWS = 64;
template <typename C, int NU>  // NU = ceil(nb / 16) column groups per thread
__global__ void __launch_bounds__(256) k_rmul_block(const C* W, long ldw, long sW, const C* __restrict__ M,
                                                  long ldm, long sM, int n1, int nb, int kchunk, C* O, long ldo,
                                                  long sO) {
  using R = decltype(C().x);
  extern __shared__ __align__(16) unsigned char rmsm[];
  constexpr int MC = 16 * NU;
  C* Ws = (C*)rmsm;                  // [TM_ROWS][nb + 1]
  const int lw = nb + 1;
  C* Ms = Ws + TM_ROWS * lw;         // [kchunk][MC]
  const int b = blockIdx.y, tid = threadIdx.x;
  const int r0 = blockIdx.x * TM_ROWS;
  W += (long)b * sW;
  M += (long)b * sM;
  O += (long)b * sO;
  // asynchronous copies: every element of the rows and of the chunk of M is in flight at once
  for (int r = tid >> 5; r < TM_ROWS; r += 8)
    for (int k = tid & 31; k < nb; k += 32) {
      if (r0 + r < n1) cp_async_elem(Ws + r * lw + k, W + (long)(r0 + r) * ldw + k);
      else Ws[r * lw + k] = C{R(0), R(0)};
    }
  const int ty = tid >> 4, tx = tid & 15;
  C acc[4][NU];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int u = 0; u < NU; ++u) acc[a][u] = C{R(0), R(0)};
  for (int k0 = 0; k0 < nb; k0 += kchunk) {
    const int kc = min(kchunk, nb - k0);
    if (k0 > 0) __syncthreads();  // the previous chunk of M consumed
    for (int e = tid; e < kc * MC; e += 256) {
      const int kk = e / MC, c = e - kk * MC;
      if (c < nb) cp_async_elem(Ms + e, M + (long)(k0 + kk) * ldm + c);
      else Ms[e] = C{R(0), R(0)};
    }
    cp_async_wait_all();
    __syncthreads();
    for (int kk = 0; kk < kc; ++kk) {
      const int k = k0 + kk;
      C a[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) a[q] = Ws[(ty + 16 * q) * lw + k];
      const int u0 = k >> 4;  // M(k, c) = 0 for c < k
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        if (u >= u0) {
          const C mv = Ms[kk * MC + tx + 16 * u];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            acc[q][u].x = fma(a[q].x, mv.x, acc[q][u].x);
            acc[q][u].x = fma(-a[q].y, mv.y, acc[q][u].x);
            acc[q][u].y = fma(a[q].x, mv.y, acc[q][u].y);
            acc[q][u].y = fma(a[q].y, mv.x, acc[q][u].y);
          }
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = r0 + ty + 16 * q;
    if (r < n1) {
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        const int c = tx + 16 * u;
        if (c < nb) O[(long)r * ldo + c] = acc[q][u];
      }
    }
  }
}

template <typename C>
int rmul_block(const C* W, long ldw, long sW, const C* M, long ldm, long sM, int n1, int nb, int batch, C* O, long ldo,
               long sO, cudaStream_t s) {
  if (nb <= 0 || n1 <= 0 || batch <= 0) return TSVD_OK;
  if (nb > 128) return TSVD_ERR_UNSUPPORTED;
  if (batch > 65535) return TSVD_ERR_UNSUPPORTED;
  const int nu = (nb + 15) / 16;
  const size_t wbytes = (size_t)TM_ROWS * (nb + 1) * sizeof(C), mrow = (size_t)16 * nu * sizeof(C);
  int kchunk = nb;
  while (wbytes + kchunk * mrow > 200 * 1024) kchunk = (kchunk + 1) / 2;
  const size_t smem = wbytes + kchunk * mrow;
  const dim3 grid(cdiv(n1, TM_ROWS), batch);
  auto go = [&](auto kern) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return TSVD_ERR_CUDA;
    }
    kern<<<grid, 256, smem, s>>>(W, ldw, sW, M, ldm, sM, n1, nb, kchunk, O, ldo, sO);
    TSVD_LAUNCHED();
    return TSVD_OK;
  };
  switch (nu) {
    case 1: return go(k_rmul_block<C, 1>);
    case 2: return go(k_rmul_block<C, 2>);
    case 3: return go(k_rmul_block<C, 3>);
    case 4: return go(k_rmul_block<C, 4>);
    case 5: return go(k_rmul_block<C, 5>);
    case 6: return go(k_rmul_block<C, 6>);
    case 7: return go(k_rmul_block<C, 7>);
    default: return go(k_rmul_block<C, 8>);
  }
}
template int rmul_block<double2>(const double2*, long, long, const double2*, long, long, int, int, int, double2*, long,
                                 long, cudaStream_t);
template int rmul_block<float2>(const float2*, long, long, const float2*, long, long, int, int, int, float2*, long, long,
                                cudaStream_t);

// ---------------------------------------------------------------------------
// Dependent Krylov columns (exact low rank, zero data): replace column c+j by
// a Philox Gaussian direction (stream 3) projected twice against every other
// live column of the basis, then normalised.  Any orthonormal completion of
// span(K) leaves the Rayleigh-Ritz result of Alg. 2 optimal (Sec. 4: Q (Q^T A)_k is the best rank-k approximation within range(Q)).
// ---------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(256) k_repair_dead(C* __restrict__ Q, long ldq, long sQ, int n1, int c, int nb,
                                                     const uint32_t* __restrict__ dead, uint64_t seed, int block_id,
                                                     int* __restrict__ dead_count, int k0, int nyq) {
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
  const int k = k0 + b;  // Fourier slice index of this problem
  const bool real_slice = (k == 0) || (k == nyq);
  if (tid == 0) atomicAdd(dead_count, ndead);
  uint32_t pending[4] = {dm[0], dm[1], dm[2], dm[3]};
  for (int j = 0; j < nb; ++j) {
    if (!((dm[j >> 5] >> (j & 31)) & 1u)) continue;
    const int col = c + j;
    for (int attempt = 0; attempt < 4; ++attempt) {
      for (int i = tid; i < n1; i += blockDim.x) {
        const uint4 x = philox10(make_uint4((uint32_t)i, (uint32_t)col | ((uint32_t)attempt << 24),
                                            (uint32_t)block_id, 3u + ((uint32_t)k << 8)),
                                 (uint32_t)seed, (uint32_t)(seed >> 32));
        const double u1 = ((double)x.x + 1.0) * (1.0 / 4294967296.0);
        const double u2 = ((double)x.y + 1.0) * (1.0 / 4294967296.0);
        const double r = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        // the DC slice (and the Nyquist slice of an even-length transform) of a real
        // tensor's spectrum is real: its replacement directions are real too
        C v;
        v.x = (R)(r * cs);
        v.y = real_slice ? (R)0 : (R)(r * sn);
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
                int block_id, int* dead_count, int k0, int nyq, cudaStream_t s) {
  if (nb <= 0 || batch <= 0) return TSVD_OK;
  k_repair_dead<C><<<batch, 256, 0, s>>>(Q, ldq, sQ, n1, c, nb, dead, seed, block_id, dead_count, k0, nyq);
  TSVD_LAUNCHED();
  return TSVD_OK;
}
template int repair_dead<double2>(double2*, long, long, int, int, int, const uint32_t*, int, uint64_t, int, int*,
                                  int, int, cudaStream_t);
template int repair_dead<float2>(float2*, long, long, int, int, int, const uint32_t*, int, uint64_t, int, int*, int,
                                 int, cudaStream_t);

// Orthonormalise the nb leading columns of W (n1 x b per slice) against the c
// finished columns of Q and write them to Q columns [c, c+nb), in the
// precision L: shifted CholeskyQR3 (the shift makes the first Cholesky
// succeed for any W; the next two passes restore orthogonality to rounding
// level), each pass preceded by a classical Gram-Schmidt projection against
// Q_{<i}; dependent columns are then replaced.
// The FP32 block step with every product on tcgen05 in split TF32 (FP32-level
// accuracy, tc_gemm.cu): the block Gram W^H W and the coefficients Q^H W as
// real products of de-interleaved columns (K = n1), the update W -= Q (Q^H W)
// and W R^-1 as real(X) E(Y)^T with the small expanded real form E of the
// thin factor.  Q's finished columns are split once per block (hi / lo
// interleaved and de-interleaved rows) and reused by all later projections;
// the update's epilogue writes W's split rows for W R^-1.
// X^H Y (rows x cols complex) from the real product P = X_d Y_d^T of the de-interleaved columns
// (row 2c of X_d the real parts of column c of X, row 2c+1 the imaginary parts; Y_d alike):
//   (X^H Y)_ij = P[2i][2j] + P[2i+1][2j+1] + i (P[2i][2j+1] - P[2i+1][2j])
__global__ void k_complex_from_real(const float* __restrict__ P, long ldp, long sp, int rows, int cols,
                                    float2* __restrict__ G, long ldg, long sG, int batch) {
  const long total = (long)batch * rows * cols;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int j = idx % cols;
    const long r = idx / cols;
    const int i = r % rows;
    const int b = r / rows;
    const float* p0 = P + (long)b * sp + (long)(2 * i) * ldp + 2 * j;
    const float* p1 = p0 + ldp;
    G[(long)b * sG + (long)i * ldg + j] = make_float2(p0[0] + p1[1], p0[1] - p1[0]);
  }
}

static int complex_from_real(const float* P, long ldp, long sp, int rows, int cols, float2* G, long ldg, long sG,
                             int batch, cudaStream_t s) {
  const long total = (long)batch * rows * cols;
  if (total <= 0) return TSVD_OK;
  k_complex_from_real<<<(unsigned)std::min<long>(cdiv(total, 256), 4096), 256, 0, s>>>(P, ldp, sp, rows, cols, G,
                                                                                      ldg, sG, batch);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

static int orth_block_tc(int n1, int b, int m, int h, const OrthWs& w, int c, int nb, int block_id, uint64_t seed,
                         cudaStream_t s) {
  const OrthTc& t = *w.tc;
  float2* Q = (float2*)w.Q;
  float2* W = (float2*)w.W;
  float2* P = (float2*)w.P;
  float2* Gs = (float2*)w.G;
  float2* Mi = (float2*)w.Minv;
  const long sQ = (long)n1 * m, sW = (long)n1 * b, sP = (long)m * b, sG = (long)b * b;
  const long sWT = (long)b * t.ldq2, sWr = (long)n1 * t.ldw2, sE = 2L * b * t.ldq2;
  const long ldd = t.ldq2 / 2;  // de-interleaved rows: >= n1, a multiple of 4 (16-byte rows)
  // which split copies of the current W exist: wd its de-interleaved rows (WThi / WTlo), wr its
  // rows (Whi / Wlo), written by the epilogue of the GEMM that produced W
  bool wd = false, wr = false;
  TcSplitOut both;
  both.Rhi = t.Whi;
  both.Rlo = t.Wlo;
  both.ldr = t.ldw2;
  both.sr = sWr;
  both.Thi = t.WThi;
  both.Tlo = t.WTlo;
  both.ldt = ldd;
  both.st = sWT;
  TcSplitOut rows_only = both;  // measured: the transposed copy costs the epilogue more than a
  rows_only.Thi = rows_only.Tlo = nullptr;  // separate de-interleaving pass
  for (int pass = 0; pass < 3; ++pass) {
    if (c > 0) {
      // the projection on tcgen05 against the cached split operands of Q's finished columns:
      // Q^H W from the real product Q_d W_d^T (K = n1), then W -= Q (Q^H W) with Q's
      // interleaved rows (K = 2c) against the expanded coefficients
      TSVD_STAGE("orth_cgs", s);
      if (!wd) TSVD_TRY(split_deinterleave(W, n1, nb, b, sW, h, t.WThi, t.WTlo, ldd, sWT, s));
      TSVD_TRY(tc_gemm_split(t.Qdhi, t.Qdlo, ldd, 2L * m * ldd, 2 * c, t.WThi, t.WTlo, ldd, sWT, 2 * nb, n1, t.Elo,
                             2L * b, 4L * m * b, h, t.err, s));
      TSVD_TRY(complex_from_real(t.Elo, 2L * b, 4L * m * b, c, nb, P, nb, sP, h, s));
      const long sEq = 2L * b * t.ldqi;
      TSVD_TRY(expand_thin_split(P, nb, sP, c, nb, t.Ehi, t.Elo, t.ldqi, sEq, h, 0, s));
      TSVD_TRY(tc_gemm_split(t.Qhi, t.Qlo, t.ldqi, (long)n1 * t.ldqi, n1, t.Ehi, t.Elo, t.ldqi, sEq, 2 * nb, 2 * c,
                             (float*)W, 2L * b, 2L * sW, h, t.err, s, -1.0f, 1.0f, &rows_only));
      wd = false;
      wr = true;
    }
    {
      // G = W^H W through the real Gram of W's de-interleaved columns (K = n1; 2 nb x 2 nb outputs,
      // kept in Elo until the Cholesky has read G)
      TSVD_STAGE("orth_gram", s);
      float* Pr = t.Elo;
      if (!wd) TSVD_TRY(split_deinterleave(W, n1, nb, b, sW, h, t.WThi, t.WTlo, ldd, sWT, s));
      TSVD_TRY(tc_gemm_split(t.WThi, t.WTlo, ldd, sWT, 2 * nb, t.WThi, t.WTlo, ldd, sWT, 2 * nb, n1, Pr, 2L * b,
                             4L * b * b, h, t.err, s));
      TSVD_TRY(complex_from_real(Pr, 2L * b, 4L * b * b, nb, nb, Gs, b, sG, h, s));
    }
    {
      TSVD_STAGE("orth_chol", s);
      TSVD_TRY(chol_inv<float2>(Gs, b, sG, Mi, b, sG, nb, h, pass == 0 ? 1e-5 : 0.0, 1e-7, w.dead, s));
    }
    {
      TSVD_STAGE("orth_trsm", s);  // W R^-1, the last pass straight into its columns of Q
      if (!wr) TSVD_TRY(split_rows((const float*)W, 2L * b, t.Whi, t.Wlo, t.ldw2, 2 * nb, (long)h * n1, s));
      TSVD_TRY(expand_thin_split(Mi, b, sG, nb, nb, t.Ehi, t.Elo, t.ldw2, sE, h, 0, s));
      float* out = (pass < 2) ? (float*)W : (float*)(Q + c);
      TSVD_TRY(tc_gemm_split(t.Whi, t.Wlo, t.ldw2, sWr, n1, t.Ehi, t.Elo, t.ldw2, sE, 2 * nb, 2 * nb, out,
                             pass < 2 ? 2L * b : 2L * m, pass < 2 ? 2L * sW : 2L * sQ, h, t.err, s));
      wd = wr = false;
    }
  }
  {
    TSVD_STAGE("orth_repair", s);
    TSVD_TRY(repair_dead<float2>(Q, m, sQ, n1, c, nb, w.dead, h, seed, block_id, w.dead_count, w.k0, w.nyq, s));
  }
  // the finished columns' split operands for the projections of the later blocks
  TSVD_STAGE("orth_cgs", s);
  TSVD_TRY(split_block((const float*)(Q + c), 2L * m, t.Qhi + 2L * c, t.Qlo + 2L * c, t.ldqi, 2 * nb, (long)h * n1,
                       s));
  return split_deinterleave(Q + c, n1, nb, m, sQ, h, t.Qdhi + 2L * c * ldd, t.Qdlo + 2L * c * ldd, ldd,
                            2L * m * ldd, s);
}

template <typename L>
int orth_block_cols(int n1, int b, int m, int h, const OrthWs& w, int c, int nb, int block_id, uint64_t seed,
                    cudaStream_t s) {
  using CL = cx_t<L>;
  if constexpr (std::is_same<L, float>::value) {
    if (w.tc) return orth_block_tc(n1, b, m, h, w, c, nb, block_id, seed, s);
  }
  const long sQ = (long)n1 * m, sW = (long)n1 * b, sP = (long)m * b, sG = (long)b * b;
  CL* Q = (CL*)w.Q;
  CL* W = (CL*)w.W;
  CL* P = (CL*)w.P;
  CL* Gs = (CL*)w.G;
  const size_t sk = std::is_same<L, double>::value ? w.splitk_elems : 2 * w.splitk_elems;
  // FP64: Fukaya et al.'s shift 11 (n nb + nb (nb+1)) u ||W||^2 (trace as the norm
  // bound); FP32: 1e-5 trace(G), above the FP32 Gram error ~ sqrt(n) u ||W||^2
  const double shift = std::is_same<L, double>::value
                           ? 11.0 * ((double)n1 * nb + (double)nb * (nb + 1)) * 1.1102230246251565e-16
                           : 1e-5;
  const double dead_rel = std::is_same<L, double>::value ? 1e-12 : 1e-7;
  for (int pass = 0; pass < 3; ++pass) {
    // a Gram-Schmidt projection before every pass: without the third, blocks
    // whose new directions are tiny next to the old ones (exact low rank in
    // FP32, the fast-decaying spectra of Sec. 5 Ex. 1 in FP64) lose accuracy
    if (c > 0) {
      TSVD_STAGE("orth_cgs", s);
      TSVD_TRY(cgemm<CL>(gemm('H', 'N', c, nb, n1, 1.0, Q, m, sQ, W, b, sW, 0.0, P, nb, sP, h), w.splitk, sk, s));
      TSVD_TRY(cgemm<CL>(gemm('N', 'N', n1, nb, c, -1.0, Q, m, sQ, P, nb, sP, 1.0, W, b, sW, h), w.splitk, sk, s));
    }
    {
      TSVD_STAGE("orth_gram", s);
      TSVD_TRY(cgemm<CL>(gemm('H', 'N', nb, nb, n1, 1.0, W, b, sW, W, b, sW, 0.0, Gs, b, sG, h), w.splitk, sk, s));
    }
    CL* Mi = (CL*)w.Minv;  // R-tilde^{-1}, nb x nb per slice (leading dimension b)
    {
      TSVD_STAGE("orth_chol", s);
      TSVD_TRY(chol_inv<CL>(Gs, b, sG, Mi, b, sG, nb, h, pass == 0 ? shift : 0.0, dead_rel, w.dead, s));
    }
    {
      TSVD_STAGE("orth_trsm", s);
      // the last pass writes the finished block straight into its columns of Q
      if (pass < 2) TSVD_TRY(rmul_block<CL>(W, b, sW, Mi, b, sG, n1, nb, h, W, b, sW, s));
      else TSVD_TRY(rmul_block<CL>(W, b, sW, Mi, b, sG, n1, nb, h, Q + c, m, sQ, s));
    }
  }
  {
    TSVD_STAGE("orth_repair", s);
    TSVD_TRY(repair_dead<CL>(Q, m, sQ, n1, c, nb, w.dead, h, seed, block_id, w.dead_count, w.k0, w.nyq, s));
  }
  if (w.Qt) {
    TSVD_STAGE("convert", s);
    TSVD_TRY(convert_c64_to_c32((const double2*)Q + c, m, sQ, (float2*)w.Qt + c, m, sQ, n1, nb, h, s));
  }
  return TSVD_OK;
}

template int orth_block_cols<double>(int, int, int, int, const OrthWs&, int, int, int, uint64_t, cudaStream_t);
template int orth_block_cols<float>(int, int, int, int, const OrthWs&, int, int, int, uint64_t, cudaStream_t);

}  // namespace tsvd
