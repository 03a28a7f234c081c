// eig.cu -- the Hermitian eigen-solve behind the small SVD of Alg. 2
// ([U_c, S_c, V_c] = T-SVD(C) with C = Q^H X per Fourier slice): with
// G = C C^H = U_c S_c^2 U_c^H, the R largest eigenpairs of the m x m G give
// sigma_i = sqrt(lambda_i) and U_c(:, 1:R).
//
//   1. Householder reduction to tridiagonal form, T' = H_{m-2}..H_0 G H_0..H_{m-2};
//      a cluster of CTAs shares each slice's rows (FP64 is the bound, so the
//      work of one slice is spread over several SMs).
//   2. T = D^H T' D real symmetric (D diagonal unitary); bisection on Sturm
//      counts (a division-free three-term recurrence) for the R largest
//      eigenvalues, inverse iteration with a partially pivoted LU for the
//      vectors, two classical Gram-Schmidt passes inside clusters of close
//      eigenvalues.
//   3. u_r = H_0 .. H_{m-2} D z_r.
#include <cooperative_groups.h>
#include <float.h>

#include "common.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace tsvd {

constexpr int HETRD_CLUSTER = 4;

struct EigScratch {
  double* d;       // [batch][m] diagonal of T
  double* f;       // [batch][m] off-diagonal |alpha_j|
  double2* alpha;  // [batch][m] complex off-diagonals of T'
  double2* delta;  // [batch][m] phases making T real
  double2* Hv;     // [batch][m][m] Householder vectors (row j, columns j+1..m-1)
  double2* pbuf;   // [batch][HETRD_CLUSTER][m] partial matrix-vector products of a cluster
  double* Z;       // [batch][R][m] real eigenvectors of T (vector-contiguous)
  double* lu;      // [batch][5][m][R] inverse-iteration LU factors
  double* tnorm;   // [batch]
  double2* Sg;     // packed own rows of the cluster reduction when they do not fit in shared memory
};

static bool hetrd_needs_global_rows(int m, int batch);

static EigScratch carve_eig(void* base, int m, int R, int batch, size_t* bytes) {
  Carver cv(base);
  EigScratch e;
  e.d = cv.take<double>((size_t)batch * m);
  e.f = cv.take<double>((size_t)batch * m);
  e.alpha = cv.take<double2>((size_t)batch * m);
  e.delta = cv.take<double2>((size_t)batch * m);
  e.Hv = cv.take<double2>((size_t)batch * m * m);
  e.pbuf = cv.take<double2>((size_t)batch * HETRD_CLUSTER * m);
  e.Z = cv.take<double>((size_t)batch * m * R);
  e.lu = cv.take<double>((size_t)batch * 5 * m * R);
  e.tnorm = cv.take<double>((size_t)batch);
  // CL CTAs of a slice own at most m(m+1)/2 + CL m packed elements together (CL <= 8)
  e.Sg = hetrd_needs_global_rows(m, batch) ? cv.take<double2>((size_t)batch * ((size_t)m * (m + 1) / 2 + 8 * (size_t)m))
                                           : nullptr;
  if (bytes) *bytes = cv.bytes();
  return e;
}

size_t eig_scratch_bytes(int m, int R, int batch) {
  size_t b = 0;
  carve_eig(nullptr, m, R, batch, &b);
  return b;
}

__device__ __forceinline__ double2 ldcg2(const double2* p) { return __ldcg(p); }

// ---------------------------------------------------------------------------
// Householder tridiagonalisation, one cluster of CL CTAs per slice; only the
// lower triangle of G is read and updated.  Rows of the trailing block are
// owned round-robin (global row g by CTA g mod CL).  Step j:
//   x = G(j+1:, j), alpha = -e^{i arg x_0} ||x||, v = (x - alpha e_1)/||.||
//   (every CTA forms the same v);
//   p = 2 A v from the lower triangle: each CTA adds, for its rows r, the row
//   part sum_{k<=r} A(r,k) v_k to p_r and the transposed part conj(A(r,k)) v_r
//   to p_k (k < r) into a shared partial, then the CL partials are summed
//   after a cluster barrier;
//   w = p - (v^H p) v;  A(r,k) -= v_r conj(w_k) + w_r conj(v_k) for k <= r.
// Data another CTA wrote is read with L2-coherent loads after the barrier
// (release / acquire at cluster scope).
// ---------------------------------------------------------------------------
template <int CL>
__global__ void __launch_bounds__(512) k_hetrd(double2* __restrict__ G, long ldg, long sG, int m, EigScratch e) {
  extern __shared__ __align__(16) double2 sh[];
  double2* v = sh;            // [m]
  double2* p = sh + m;        // [m] full product / w
  double2* pw = sh + 2 * m;   // [nwarp][m] per-warp partial products (fixed-order sum: deterministic)
  __shared__ double red[64];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (CL > 1) ? (int)cluster.block_rank() : 0;
  const int b = blockIdx.x / CL;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  G += (long)b * sG;
  double2* Hv = e.Hv + (long)b * m * m;
  double2* pb = e.pbuf + (long)b * CL * m;  // [CL][m] partial products of the cluster's CTAs
  double2* mine = pw + (long)warp * m;
  for (int j = 0; j < m - 1; ++j) {
    const int n = m - j - 1;
    double part = 0;
    for (int i = tid; i < n; i += blockDim.x) {
      const double2 x = ldcg2(G + (long)(j + 1 + i) * ldg + j);
      v[i] = x;
      part += cabs2(x);
    }
    for (int i = lane; i < n; i += 32) mine[i] = make_double2(0, 0);
    const double nrm2 = block_sum(part, red);  // synchronises: v visible
    const double2 x0 = v[0];
    const double djj = ldcg2(G + (long)j * ldg + j).x;
    __syncthreads();
    if (rank == 0 && tid == 0) e.d[(long)b * m + j] = djj;
    const bool skip = !(nrm2 > 0.0);  // identical in every CTA of the cluster
    const int r0 = ((rank - (j + 1)) % CL + CL) % CL;
    if (!skip) {
      const double nrm = sqrt(nrm2), ax0 = sqrt(cabs2(x0));
      const double2 ph = (ax0 > 0) ? cscale(x0, 1.0 / ax0) : make_double2(1, 0);
      const double2 alpha = cscale(ph, -nrm);
      const double vinv = 1.0 / sqrt(2.0 * nrm * (nrm + ax0));
      for (int i = tid; i < n; i += blockDim.x) {
        double2 vi = v[i];
        if (i == 0) vi = csub(vi, alpha);
        vi = cscale(vi, vinv);
        v[i] = vi;
        if (rank == 0) Hv[(long)j * m + j + 1 + i] = vi;
      }
      if (rank == 0 && tid == 0) e.alpha[(long)b * m + j] = alpha;
      __syncthreads();
      // this warp's rows: row part into mine[r], transposed part conj(A(r,k)) v_r into mine[k]
      for (int r = r0 + warp * CL; r < n; r += nwarp * CL) {
        const double2* row = G + (long)(j + 1 + r) * ldg + j + 1;
        const double2 vr = v[r];
        double2 acc = make_double2(0, 0);
        for (int k = lane; k <= r; k += 32) {
          const double2 a = row[k];
          cfma(acc, a, v[k]);
          if (k < r) {  // t += conj(a) v_r
            double2 t = mine[k];
            t.x = fma(a.x, vr.x, t.x);
            t.x = fma(a.y, vr.y, t.x);
            t.y = fma(a.x, vr.y, t.y);
            t.y = fma(-a.y, vr.x, t.y);
            mine[k] = t;
          }
        }
        acc = warp_sum(acc);
        __syncwarp();
        if (lane == 0) mine[r] = cadd(mine[r], acc);
        __syncwarp();
      }
      __syncthreads();
      for (int i = tid; i < n; i += blockDim.x) {
        double2 s = make_double2(0, 0);
        for (int w = 0; w < nwarp; ++w) s = cadd(s, pw[(long)w * m + i]);
        __stcg(pb + (long)rank * m + i, s);
      }
    } else {
      for (int i = tid; i < n; i += blockDim.x)
        if (rank == 0) Hv[(long)j * m + j + 1 + i] = make_double2(0, 0);
      if (rank == 0 && tid == 0) e.alpha[(long)b * m + j] = make_double2(0, 0);
    }
    if (CL > 1) cluster.sync();
    else __syncthreads();
    if (!skip) {
      double2 kp = make_double2(0, 0);
      for (int i = tid; i < n; i += blockDim.x) {
        double2 pi = make_double2(0, 0);
#pragma unroll
        for (int c = 0; c < CL; ++c) pi = cadd(pi, ldcg2(pb + (long)c * m + i));
        pi = cscale(pi, 2.0);
        p[i] = pi;
        cfmac(kp, v[i], pi);
      }
      const double K = block_sum2(kp, red).x;
      for (int i = tid; i < n; i += blockDim.x) p[i] = csub(p[i], cscale(v[i], K));  // p <- w
      __syncthreads();
      // lower-triangle update of this CTA's rows, one warp per row
      for (int r = r0 + warp * CL; r < n; r += nwarp * CL) {
        double2* row = G + (long)(j + 1 + r) * ldg + j + 1;
        const double2 vr = v[r], wr = p[r];
        for (int k = lane; k <= r; k += 32) {
          const double2 vk = v[k], wk = p[k];
          double2 t = row[k];
          // t -= v_r conj(w_k) + w_r conj(v_k), as four fused multiply-adds per component
          t.x = fma(-vr.x, wk.x, t.x);
          t.x = fma(-vr.y, wk.y, t.x);
          t.x = fma(-wr.x, vk.x, t.x);
          t.x = fma(-wr.y, vk.y, t.x);
          t.y = fma(-vr.y, wk.x, t.y);
          t.y = fma(vr.x, wk.y, t.y);
          t.y = fma(-wr.y, vk.x, t.y);
          t.y = fma(wr.x, vk.y, t.y);
          row[k] = t;
        }
      }
    }
    if (CL > 1) cluster.sync();
    else __syncthreads();
  }
  if (rank == 0 && tid == 0) {
    e.d[(long)b * m + m - 1] = ldcg2(G + (long)(m - 1) * ldg + m - 1).x;
    // phases: T = D^H T' D real with T(j+1, j) = |alpha_j|
    double2 dl = make_double2(1, 0);
    e.delta[(long)b * m] = dl;
    double tn = 0;
    for (int j = 0; j < m - 1; ++j) {
      const double2 a = e.alpha[(long)b * m + j];
      const double aa = sqrt(cabs2(a));
      e.f[(long)b * m + j] = aa;
      if (aa > 0) dl = cmul(dl, cscale(a, 1.0 / aa));
      e.delta[(long)b * m + j + 1] = dl;
    }
    for (int j = 0; j < m; ++j) {
      const double fl = (j > 0) ? e.f[(long)b * m + j - 1] : 0.0, fr = (j < m - 1) ? e.f[(long)b * m + j] : 0.0;
      tn = fmax(tn, fabs(e.d[(long)b * m + j]) + fl + fr);
    }
    e.tnorm[b] = tn;
  }
}

// ---------------------------------------------------------------------------
// Householder tridiagonalisation with the lower triangle resident in shared
// memory.  One cluster of CL CTAs per slice; CTA c owns global rows
// g = c + CL q, stored packed (row g holds columns 0..g).  GB300 issues FP64
// at 2 DFMA per clock per SM, so the kernel is organised to spend its FP64
// instructions on the 16 DFMA per trailing element and step that the method
// needs, on full warps:
//   * the rank-2 update of step j-1 is applied lazily inside step j's pass
//     over the trailing triangle (one visit per element and step);
//   * the work of a pass is cut into equal contiguous segments, one per
//     thread, of a row-major enumeration (row part sum_k A(g,k) v_k) and of
//     a column-major enumeration (transposed part sum_g conj(A(g,k)) v_g), so
//     every accumulation is private to a thread; rows or columns split
//     between threads are summed from per-thread slots in thread order
//     (deterministic);
//   * the column x_j and the partial products are exchanged through
//     distributed shared memory with two cluster barriers per step.
// Step j (A^{(j)} = the matrix after j reflectors; the stored S lags one
// update behind: S = A^{(j-1)} on the trailing block):
//   x_g = S(g,j) - v'_g conj(w'_j) - w'_g conj(v'_j)      (v', w' of step j-1)
//   alpha = -e^{i arg x_0} ||x||,  v = (x - alpha e_1) / ||x - alpha e_1||
//   S(g,k) <- S(g,k) - v'_g conj(w'_k) - w'_g conj(v'_k)   (k <= g, both > j)
//   p = 2 A^{(j)} v,  w = p - (v^H p) v
// ---------------------------------------------------------------------------
constexpr int HS_THREADS = 256;
constexpr int HS_U_GLOBAL = 4;  // row-store elements a thread loads before using them, rows in L2

__host__ __device__ __forceinline__ int hs_own_rows(int m, int c, int CL) { return (c < m) ? (m - 1 - c) / CL + 1 : 0; }
__host__ __device__ __forceinline__ int hs_rowbase(int q, int c, int CL) { return q * (c + 1) + CL * q * (q - 1) / 2; }
// first own row index q with c + CL q > j
__host__ __device__ __forceinline__ int hs_qfirst(int j, int c, int CL) { return (j < c) ? 0 : (j - c) / CL + 1; }

static size_t hetrd_smem_elems(int m, int CL) {
  int mx = 0;
  for (int c = 0; c < CL; ++c) mx = std::max(mx, hs_rowbase(hs_own_rows(m, c, CL), c, CL));
  return (size_t)mx;
}
static size_t hetrd_smem_bytes(int m, int CL, int nt = HS_THREADS, bool global_rows = false) {
  const size_t vown = (size_t)(m + CL - 1) / CL;  // v at the own rows, compacted
  const size_t rows = global_rows ? 0 : hetrd_smem_elems(m, CL);
  const size_t el = (rows + 5 * (size_t)m + 2 * (size_t)nt + vown) * sizeof(double2);
  return el + (size_t)(m + 1) * sizeof(int);
}

// A pass of E elements is cut into contiguous segments of L elements (the
// last one shorter), one per thread: L is odd and at least 5, so the
// addresses of neighbouring lanes inside a row differ by an odd multiple of
// 16 bytes and fall in different shared-memory bank groups.
template <int NT>
__device__ __forceinline__ int hs_seglen(int E) {
  int L = max(5, E / NT) | 1;
  while ((E + L - 1) / L > NT) L += 2;
  return L;
}
__device__ __forceinline__ int hs_seg(int t, int E, int L) { return min(t * L, E); }
// the segment holding element e
__device__ __forceinline__ int hs_owner(int e, int L) { return e / L; }

template <int CL, bool GS>
__global__ void __launch_bounds__(HS_THREADS, 1) k_hetrd_smem(const double2* __restrict__ G, long ldg, long sG, int m,
                                                           int s_elems, EigScratch e, int b0) {
  extern __shared__ __align__(16) double2 hsm[];
  // own rows, packed: in shared memory, or (GS) in this CTA's private part of a
  // global array, which stays L2-resident (only this CTA reads or writes it)
  double2* S = GS ? e.Sg + (long)blockIdx.x * s_elems : hsm;
  double2* bufV = GS ? hsm : S + s_elems;      // [2][m] v of this and of the previous step
  double2* bufW = bufV + 2 * m;                // [2][m] w
  double2* pv = bufW + 2 * m;                  // [m] this CTA's part of p
  double2* slotF = pv + m;                     // [T] partial of a thread's first (split) row / column
  double2* slotL = slotF + HS_THREADS;         // [T] partial of a thread's last (split) row / column
  double2* vown = slotL + HS_THREADS;          // [ceil(m/CL)] v at the own rows (odd lane stride in the column pass)
  int* CP = (int*)(vown + (m + CL - 1) / CL);  // [m+1] prefix of the per-column own-row counts
  __shared__ double red[2 * (HS_THREADS / 32)];
  cg::cluster_group cluster = cg::this_cluster();
  const int c = (CL > 1) ? (int)cluster.block_rank() : 0;
  const int b = b0 + (int)blockIdx.x / CL;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = HS_THREADS / 32;
  G += (long)b * sG;
  double2* Hv = e.Hv + (long)b * m * m;
  const int nq = hs_own_rows(m, c, CL);

  // load the own rows of the lower triangle; column prefix counts
  for (int q = warp; q < nq; q += NW) {
    const int g = c + CL * q;
    const double2* src = G + (long)g * ldg;
    double2* dst = S + hs_rowbase(q, c, CL);
    for (int k = lane; k <= g; k += 32) dst[k] = __ldcg(src + k);
  }
  if (tid == 0) {
    int acc = 0;
    for (int k = 0; k < m; ++k) {
      CP[k] = acc;
      acc += max(0, nq - hs_qfirst(k, c, CL));
    }
    CP[m] = acc;
  }
  for (int i = tid; i < 4 * m; i += HS_THREADS) bufV[i] = make_double2(0, 0);  // v', w' of "step -1"
  if (CL > 1) cluster.sync();
  else __syncthreads();

  for (int j = 0; j < m - 1; ++j) {
    const int cur = j & 1;
    double2* v = bufV + cur * m;
    double2* w = bufW + cur * m;
    const double2* vp = bufV + (cur ^ 1) * m;
    const double2* wp = bufW + (cur ^ 1) * m;
    const bool lag = j > 0;
    // (0) column j of A^{(j)} from the own rows, pushed to every CTA's v
    {
      const double2 vpj = vp[j], wpj = wp[j];
      for (int q = hs_qfirst(j, c, CL) + tid; q < nq; q += HS_THREADS) {
        const int g = c + CL * q;
        double2 a = S[hs_rowbase(q, c, CL) + j];
        if (lag) {
          const double2 vg = vp[g], wg = wp[g];
          a.x -= vg.x * wpj.x + vg.y * wpj.y + wg.x * vpj.x + wg.y * vpj.y;
          a.y -= vg.y * wpj.x - vg.x * wpj.y + wg.y * vpj.x - wg.x * vpj.y;
        }
#pragma unroll
        for (int rr = 0; rr < CL; ++rr) {
          double2* dst = (CL > 1) ? cluster.map_shared_rank(v, rr) : v;
          dst[g] = a;
        }
      }
      if (tid == 0 && (j % CL) == c) {
        const double2 s = S[hs_rowbase((j - c) / CL, c, CL) + j];
        e.d[(long)b * m + j] = s.x - 2.0 * (vpj.x * wpj.x + vpj.y * wpj.y);
      }
    }
    if (CL > 1) cluster.sync();
    else __syncthreads();
    // (1) the reflector (every CTA forms the same v)
    const int n = m - j - 1;
    const double2 x0 = v[j + 1];
    double part = 0;
    for (int i = tid; i < n; i += HS_THREADS) part += cabs2(v[j + 1 + i]);
    for (int i = tid; i < n; i += HS_THREADS) pv[j + 1 + i] = make_double2(0, 0);
    const double nrm2 = block_sum(part, red);
    const bool skip = !(nrm2 > 0.0);
    double2 alpha = make_double2(0, 0);
    double vinv = 0.0;
    if (!skip) {
      const double nrm = sqrt(nrm2), ax0 = sqrt(cabs2(x0));
      const double2 ph = (ax0 > 0) ? cscale(x0, 1.0 / ax0) : make_double2(1, 0);
      alpha = cscale(ph, -nrm);
      vinv = 1.0 / sqrt(2.0 * nrm * (nrm + ax0));
    }
    for (int i = tid; i < n; i += HS_THREADS) {
      double2 vi = v[j + 1 + i];
      if (i == 0) vi = csub(vi, alpha);
      vi = cscale(vi, vinv);
      v[j + 1 + i] = vi;
      if (c == 0) Hv[(long)j * m + j + 1 + i] = vi;
    }
    if (c == 0 && tid == 0) e.alpha[(long)b * m + j] = alpha;
    __syncthreads();

    // (2) row pass: lazy update of S and the row part of A v over own rows g > j, columns j+1..g
    const int q0 = hs_qfirst(j, c, CL);
    for (int q = q0 + tid; q < nq; q += HS_THREADS) vown[q] = v[c + CL * q];
    const int nr = max(0, nq - q0);
    const int g0 = c + CL * q0;
    const int E1 = nr * (g0 - j) + CL * nr * (nr - 1) / 2;  // sum of the row lengths g - j
    if (E1 > 0) {
      const int L1 = hs_seglen<HS_THREADS>(E1);
      const int e0 = hs_seg(tid, E1, L1), e1 = hs_seg(tid + 1, E1, L1);
      if (e0 < e1) {
        // row i holds elements [P(i), P(i+1)), P(i) = i (g0 - j) + CL i (i - 1) / 2
        int lo = 0, hi = nr - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (mid * (g0 - j) + CL * mid * (mid - 1) / 2 <= e0) lo = mid;
          else hi = mid - 1;
        }
        int i = lo;
        int Pi = i * (g0 - j) + CL * i * (i - 1) / 2;
        int g = g0 + CL * i;
        int k = j + 1 + (e0 - Pi);
        double2* row = S + hs_rowbase(q0 + i, c, CL);
        bool whole = (e0 == Pi), first = true;
        double2 vg = vp[g], wg = wp[g];
        double2 acc = make_double2(0, 0);
        for (int el = e0; el < e1; ++el) {
          double2 a = row[k];
          if (lag) {
            const double2 wk = wp[k], vk = vp[k];
            a.x = fma(-vg.x, wk.x, a.x);
            a.x = fma(-vg.y, wk.y, a.x);
            a.x = fma(-wg.x, vk.x, a.x);
            a.x = fma(-wg.y, vk.y, a.x);
            a.y = fma(-vg.y, wk.x, a.y);
            a.y = fma(vg.x, wk.y, a.y);
            a.y = fma(-wg.y, vk.x, a.y);
            a.y = fma(wg.x, vk.y, a.y);
            if (k == g) a.y = 0.0;  // the diagonal stays real
            row[k] = a;
          }
          cfma(acc, a, v[k]);
          if (++k > g) {  // row g done
            if (whole) pv[g] = acc;
            else slotF[tid] = acc;  // a row ending here but started earlier is this thread's first row
            first = false;
            whole = true;
            acc = make_double2(0, 0);
            row += g + 1;
            g += CL;
            k = j + 1;
            if (el + 1 < e1) {
              vg = vp[g];
              wg = wp[g];
            }
          }
        }
        if (k != j + 1) {  // the segment ends inside row g
          if (first) slotF[tid] = acc;
          else slotL[tid] = acc;
        }
      }
      __syncthreads();
      // rows split between threads: fixed-order sum of the slots
      for (int i = tid; i < nr; i += HS_THREADS) {
        const int Pi = i * (g0 - j) + CL * i * (i - 1) / 2;
        const int len = g0 + CL * i - j;
        const int ta = hs_owner(Pi, L1), tb = hs_owner(Pi + len - 1, L1);
        if (ta == tb) continue;
        double2 s = (hs_seg(ta, E1, L1) == Pi) ? slotF[ta] : slotL[ta];
        for (int t = ta + 1; t <= tb; ++t)
          if (hs_seg(t, E1, L1) < hs_seg(t + 1, E1, L1)) s = cadd(s, slotF[t]);
        pv[g0 + CL * i] = s;
      }
    }
    __syncthreads();

    // (3) column pass: transposed part sum_{g > k} conj(S(g,k)) v_g, columns k > j
    const int cb = CP[j + 1];
    const int E2 = CP[m] - cb;
    if (E2 > 0) {
      const int L2 = hs_seglen<HS_THREADS>(E2);
      const int e0 = hs_seg(tid, E2, L2), e1 = hs_seg(tid + 1, E2, L2);
      if (e0 < e1) {
        int lo = j + 1, hi = m - 1;  // last column k with CP[k] <= cb + e0
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (CP[mid] <= cb + e0) lo = mid;
          else hi = mid - 1;
        }
        int k = lo;
        int o = cb + e0 - CP[k];
        int cnt = CP[k + 1] - CP[k];
        int q = hs_qfirst(k, c, CL) + o;
        int g = c + CL * q, base = hs_rowbase(q, c, CL);
        bool whole = (o == 0), first = true;
        double2 acc = make_double2(0, 0);
        for (int el = e0; el < e1; ++el) {
          cfmac(acc, S[base + k], vown[q]);
          base += g + 1;  // next own row
          g += CL;
          ++q;
          if (++o == cnt) {  // column k done
            if (whole) pv[k] = cadd(pv[k], acc);
            else slotF[tid] = acc;
            first = false;
            whole = true;
            acc = make_double2(0, 0);
            if (el + 1 < e1) {
              do {
                ++k;
              } while (CP[k + 1] == CP[k]);
              cnt = CP[k + 1] - CP[k];
              q = hs_qfirst(k, c, CL);
              g = c + CL * q;
              base = hs_rowbase(q, c, CL);
              o = 0;
            }
          }
        }
        if (o != cnt && o != 0) {  // the segment ends inside column k
          if (first) slotF[tid] = acc;
          else slotL[tid] = acc;
        }
      }
      __syncthreads();
      for (int k = j + 1 + tid; k < m; k += HS_THREADS) {
        const int cnt = CP[k + 1] - CP[k];
        if (cnt == 0) continue;
        const int s0 = CP[k] - cb;
        const int ta = hs_owner(s0, L2), tb = hs_owner(s0 + cnt - 1, L2);
        if (ta == tb) continue;
        double2 s = (hs_seg(ta, E2, L2) == s0) ? slotF[ta] : slotL[ta];
        for (int t = ta + 1; t <= tb; ++t)
          if (hs_seg(t, E2, L2) < hs_seg(t + 1, E2, L2)) s = cadd(s, slotF[t]);
        pv[k] = cadd(pv[k], s);
      }
    }
    if (CL > 1) cluster.sync();
    else __syncthreads();

    // (4) p = 2 sum over the cluster's parts (fixed order), w = p - (v^H p) v
    double2 kp = make_double2(0, 0);
    for (int i = j + 1 + tid; i < m; i += HS_THREADS) {
      double2 pi = make_double2(0, 0);
#pragma unroll
      for (int rr = 0; rr < CL; ++rr) {
        const double2* src = (CL > 1) ? cluster.map_shared_rank(pv, rr) : pv;
        pi = cadd(pi, src[i]);
      }
      pi = cscale(pi, 2.0);
      w[i] = pi;
      cfmac(kp, v[i], pi);
    }
    const double K = block_sum2(kp, red).x;
    for (int i = j + 1 + tid; i < m; i += HS_THREADS) w[i] = csub(w[i], cscale(v[i], K));
    __syncthreads();
  }
  // last diagonal entry: apply the pending update of step m-2
  if (tid == 0 && ((m - 1) % CL) == c) {
    const double2 s = S[hs_rowbase((m - 1 - c) / CL, c, CL) + m - 1];
    const double2 vq = bufV[((m - 2) & 1) * m + m - 1], wq = bufW[((m - 2) & 1) * m + m - 1];
    e.d[(long)b * m + m - 1] = (m > 1) ? s.x - 2.0 * (vq.x * wq.x + vq.y * wq.y) : s.x;
  }
  __threadfence();
  if (CL > 1) cluster.sync();
  else __syncthreads();
  if (c == 0 && tid == 0) {
    double2 dl = make_double2(1, 0);
    e.delta[(long)b * m] = dl;
    double tn = 0;
    for (int jj = 0; jj < m - 1; ++jj) {
      const double2 a = __ldcg(e.alpha + (long)b * m + jj);
      const double aa = sqrt(cabs2(a));
      e.f[(long)b * m + jj] = aa;
      if (aa > 0) dl = cmul(dl, cscale(a, 1.0 / aa));
      e.delta[(long)b * m + jj + 1] = dl;
    }
    for (int jj = 0; jj < m; ++jj) {
      const double fl = (jj > 0) ? e.f[(long)b * m + jj - 1] : 0.0, fr = (jj < m - 1) ? e.f[(long)b * m + jj] : 0.0;
      tn = fmax(tn, fabs(__ldcg(e.d + (long)b * m + jj)) + fl + fr);
    }
    e.tnorm[b] = tn;
  }
}

// ---------------------------------------------------------------------------
// Double-float variant of k_hetrd_smem for the FP32 path.  GB300 issues FP32
// at 64x its FP64 rate, so the same reduction is carried in unevaluated pairs
// (hi, lo) of floats (about 48 significant bits) built from the error-free
// transformations TwoSum (Knuth) and TwoProduct via FMA (Dekker): a
// multiply-add costs about 15 FP32 instructions instead of one DFMA at 1/64
// of the rate.  G is first scaled by a power of two so its entries stay far
// inside the FP32 exponent range; the per-step scalars (norm, alpha, the
// scale of v, v^H p) are formed in FP64 by one thread.  The rounding level
// (about 2^-47 ||G|| per operation) is far below what the FP32 path's
// accuracy needs; the FP64 path keeps k_hetrd_smem.
// ---------------------------------------------------------------------------
struct __align__(8) dfl {
  float hi, lo;
};
struct __align__(16) cdf {  // complex double-float, 16 bytes like double2 (one 16-byte access)
  float rh, rl, ih, il;
};

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return dfl{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = a + b;
  return dfl{s, b - (s - a)};
}
// a + x y
__device__ __forceinline__ dfl df_fma(dfl a, dfl x, dfl y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
  const dfl s = df_two_sum(a.hi, p);
  return df_fast_two_sum(s.hi, s.lo + (a.lo + e));
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  const dfl s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return df_fast_two_sum(p, e);
}
// square root: correctly rounded FP32 root, then one correction with the
// exactly computed residual a - x^2 (about 46 correct bits)
__device__ __forceinline__ dfl df_sqrt(dfl a) {
  if (!(a.hi > 0.f)) return dfl{0.f, 0.f};
  const float x = sqrtf(a.hi);
  const float p = x * x, pe = fmaf(x, x, -p);
  const float r = ((a.hi - p) - pe) + a.lo;
  return df_fast_two_sum(x, r / (2.f * x));
}
// quotient: FP32 quotient, then one correction with the residual a - q b
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
  const float q = a.hi / b.hi;
  const float p = q * b.hi, pe = fmaf(q, b.hi, -p);
  const float r = (((a.hi - p) - pe) + a.lo) - q * b.lo;
  return df_fast_two_sum(q, r / b.hi);
}
// Reciprocal square root and square root without a division: the correctly
// rounded FP32 reciprocal square root y, then one Newton correction with the
// residual formed in double-float (y (1 + e/2), e = 1 - a y^2; for the root,
// x = a_hi y and x + y (a - x^2) / 2 with a - x^2 exact by FMA).  About 46
// correct bits from a 24-bit start.  a > 0.
__device__ __forceinline__ dfl df_rsqrt(dfl a) {
  const float y = __frsqrt_rn(a.hi);
  const float p = y * y, pe = fmaf(y, y, -p);  // y^2 = p + pe exactly
  const dfl ay2 = df_mul(a, dfl{p, pe});
  const float e = (1.0f - ay2.hi) - ay2.lo;    // 1 - a y^2 (1 - ay2.hi exact: ay2.hi is within 2^-22 of 1)
  return df_fast_two_sum(y, 0.5f * y * e);
}
__device__ __forceinline__ dfl df_sqrt_nodiv(dfl a) {
  if (!(a.hi > 0.f)) return dfl{0.f, 0.f};
  const float y = __frsqrt_rn(a.hi);
  const float x = a.hi * y;
  const float r = (fmaf(-x, x, a.hi)) + a.lo;  // a - x^2 (the high part exact by FMA)
  return df_fast_two_sum(x, 0.5f * y * r);
}
__device__ __forceinline__ dfl df_from(double x) {
  const float h = (float)x;
  return dfl{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to(dfl a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dfl cre(cdf a) { return dfl{a.rh, a.rl}; }
__device__ __forceinline__ dfl cim(cdf a) { return dfl{a.ih, a.il}; }
__device__ __forceinline__ cdf cdf_make(dfl r, dfl i) { return cdf{r.hi, r.lo, i.hi, i.lo}; }
__device__ __forceinline__ cdf cdf_from(double2 x) { return cdf_make(df_from(x.x), df_from(x.y)); }
__device__ __forceinline__ double2 cdf_to(cdf a) { return make_double2(df_to(cre(a)), df_to(cim(a))); }
__device__ __forceinline__ cdf cdf_zero() { return cdf{0.f, 0.f, 0.f, 0.f}; }
__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) { return cdf_make(df_add(cre(a), cre(b)), df_add(cim(a), cim(b))); }
// acc += a b
// a + sum_i x_i y_i with one renormalisation at the end: each exact product
// (TwoProduct by FMA plus the two cross terms) is added to the running high
// part by TwoSum and every rounding error goes to one low accumulator (the
// compensated dot product of Ogita, Rump and Oishi in double-float form).
template <int N>
__device__ __forceinline__ dfl df_dot(dfl a, const dfl (&x)[N], const dfl (&y)[N]) {
  float s = a.hi, e = a.lo;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float p = x[i].hi * y[i].hi;
    float pe = fmaf(x[i].hi, y[i].hi, -p);
    pe = fmaf(x[i].hi, y[i].lo, fmaf(x[i].lo, y[i].hi, pe));
    const float t = s + p, bb = t - s;
    e += ((s - (t - bb)) + (p - bb)) + pe;
    s = t;
  }
  return df_fast_two_sum(s, e);
}
// acc += a b
__device__ __forceinline__ void cdf_fma(cdf& acc, cdf a, cdf b) {
  const dfl xr[2] = {cre(a), df_neg(cim(a))}, yr[2] = {cre(b), cim(b)};
  const dfl xi[2] = {cre(a), cim(a)}, yi[2] = {cim(b), cre(b)};
  acc = cdf_make(df_dot<2>(cre(acc), xr, yr), df_dot<2>(cim(acc), xi, yi));
}
// acc += conj(a) b
__device__ __forceinline__ void cdf_fmac(cdf& acc, cdf a, cdf b) {
  const dfl xr[2] = {cre(a), cim(a)}, yr[2] = {cre(b), cim(b)};
  const dfl xi[2] = {cre(a), df_neg(cim(a))}, yi[2] = {cim(b), cre(b)};
  acc = cdf_make(df_dot<2>(cre(acc), xr, yr), df_dot<2>(cim(acc), xi, yi));
}
// acc += a b and acc += conj(a) b with acc kept unnormalised: the high words
// carry the running sums, the low words every rounding error (the loop of
// df_dot without its final renormalisation, which cdf_add does later)
__device__ __forceinline__ void df_acc(float& s, float& e, float xh, float xl, float yh, float yl) {
  const float p = xh * yh;
  float pe = fmaf(xh, yh, -p);
  pe = fmaf(xh, yl, fmaf(xl, yh, pe));
  const float t = s + p, bb = t - s;
  e += ((s - (t - bb)) + (p - bb)) + pe;
  s = t;
}
__device__ __forceinline__ void cdf_fma_acc(cdf& acc, cdf a, cdf b) {
  df_acc(acc.rh, acc.rl, a.rh, a.rl, b.rh, b.rl);
  df_acc(acc.rh, acc.rl, -a.ih, -a.il, b.ih, b.il);
  df_acc(acc.ih, acc.il, a.rh, a.rl, b.ih, b.il);
  df_acc(acc.ih, acc.il, a.ih, a.il, b.rh, b.rl);
}
__device__ __forceinline__ void cdf_fmac_acc(cdf& acc, cdf a, cdf b) {
  df_acc(acc.rh, acc.rl, a.rh, a.rl, b.rh, b.rl);
  df_acc(acc.rh, acc.rl, a.ih, a.il, b.ih, b.il);
  df_acc(acc.ih, acc.il, a.rh, a.rl, b.ih, b.il);
  df_acc(acc.ih, acc.il, -a.ih, -a.il, b.rh, b.rl);
}
// a - vg conj(wk) - wg conj(vk)
__device__ __forceinline__ cdf cdf_lag(cdf a, cdf vg, cdf wg, cdf vk, cdf wk) {
  const dfl xr[4] = {df_neg(cre(vg)), df_neg(cim(vg)), df_neg(cre(wg)), df_neg(cim(wg))};
  const dfl yr[4] = {cre(wk), cim(wk), cre(vk), cim(vk)};
  const dfl xi[4] = {df_neg(cim(vg)), cre(vg), df_neg(cim(wg)), cre(wg)};
  const dfl yi[4] = {cre(wk), cim(wk), cre(vk), cim(vk)};
  return cdf_make(df_dot<4>(cre(a), xr, yr), df_dot<4>(cim(a), xi, yi));
}
// x * s for a real double-float s
__device__ __forceinline__ cdf cdf_scale(cdf x, dfl s) {
  const dfl z{0.f, 0.f};
  return cdf_make(df_fma(z, cre(x), s), df_fma(z, cim(x), s));
}
__device__ __forceinline__ dfl df_shfl_xor(dfl a, int o) {
  return dfl{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ cdf cdf_shfl_xor(cdf a, int o) {
  return cdf{__shfl_xor_sync(0xffffffffu, a.rh, o), __shfl_xor_sync(0xffffffffu, a.rl, o),
             __shfl_xor_sync(0xffffffffu, a.ih, o), __shfl_xor_sync(0xffffffffu, a.il, o)};
}
// block-wide sum in a fixed order, result on every thread (two barriers)
__device__ __forceinline__ dfl df_block_sum(dfl v, dfl* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  dfl t = (lane < nw) ? red[lane] : dfl{0.f, 0.f};
  for (int o = 16; o > 0; o >>= 1) t = df_add(t, df_shfl_xor(t, o));
  return t;
}

template <int CL, int NT, bool GS>
__global__ void __launch_bounds__(NT, 1) k_hetrd_df(const double2* __restrict__ G, long ldg, long sG, int m,
                                                            int s_elems, EigScratch e, int b0) {
  extern __shared__ __align__(16) cdf dsm[];
  // own rows, packed: in shared memory, or (GS) in this CTA's private part of a
  // global array, which stays L2-resident (only this CTA reads or writes it)
  cdf* S = GS ? (cdf*)e.Sg + (long)blockIdx.x * s_elems : dsm;
  cdf* bufV = GS ? dsm : S + s_elems;
  constexpr int HS_U = HS_U_GLOBAL;
  cdf* bufW = bufV + 2 * m;
  cdf* pv = bufW + 2 * m;
  cdf* slotF = pv + m;
  cdf* slotL = slotF + NT;
  cdf* vown = slotL + NT;
  int* CP = (int*)(vown + (m + CL - 1) / CL);
  __shared__ dfl red[NT / 32];
  __shared__ int s_exp;
  __shared__ cdf s_am;   // -alpha of the current reflector
  __shared__ dfl s_vinv; // its normalisation
  cg::cluster_group cluster = cg::this_cluster();
  const int c = (CL > 1) ? (int)cluster.block_rank() : 0;
  const int b = b0 + (int)blockIdx.x / CL;  // slice (launches may cover a range of slices from b0)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NT / 32;
  G += (long)b * sG;
  float2* Hv32 = (float2*)e.Hv + (long)b * m * m;
  const int nq = hs_own_rows(m, c, CL);

  // power-of-two scale from the largest diagonal entry (identical in every CTA)
  {
    double mx = 0;
    for (int i = tid; i < m; i += NT) mx = fmax(mx, fabs(__ldcg(G + (long)i * ldg + i).x));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ double wmx[NW];
    if (lane == 0) wmx[warp] = mx;
    __syncthreads();
    if (tid == 0) {
      double t = 0;
      for (int w = 0; w < NW; ++w) t = fmax(t, wmx[w]);
      int ex = 0;
      if (t > 0 && isfinite(t)) frexp(t, &ex);
      s_exp = ex;
    }
    __syncthreads();
  }
  const int ex = s_exp;
  for (int q = warp; q < nq; q += NW) {
    const int g = c + CL * q;
    const double2* src = G + (long)g * ldg;
    cdf* dst = S + hs_rowbase(q, c, CL);
    for (int k = lane; k <= g; k += 32) {
      const double2 x = __ldcg(src + k);
      dst[k] = cdf_from(make_double2(ldexp(x.x, -ex), ldexp(x.y, -ex)));
    }
  }
  if (tid == 0) {
    int acc = 0;
    for (int k = 0; k < m; ++k) {
      CP[k] = acc;
      acc += max(0, nq - hs_qfirst(k, c, CL));
    }
    CP[m] = acc;
  }
  for (int i = tid; i < 4 * m; i += NT) bufV[i] = cdf_zero();
  if (CL > 1) cluster.sync();
  else __syncthreads();

  for (int j = 0; j < m - 1; ++j) {
    const int cur = j & 1;
    cdf* v = bufV + cur * m;
    cdf* w = bufW + cur * m;
    const cdf* vp = bufV + (cur ^ 1) * m;
    const cdf* wp = bufW + (cur ^ 1) * m;
    const bool lag = j > 0;
    {
      const cdf vpj = vp[j], wpj = wp[j];
      for (int q = hs_qfirst(j, c, CL) + tid; q < nq; q += NT) {
        const int g = c + CL * q;
        cdf a = S[hs_rowbase(q, c, CL) + j];
        if (lag) a = cdf_lag(a, vp[g], wp[g], vpj, wpj);
#pragma unroll
        for (int rr = 0; rr < CL; ++rr) {
          cdf* dst = (CL > 1) ? cluster.map_shared_rank(v, rr) : v;
          dst[g] = a;
        }
      }
      if (tid == 0 && (j % CL) == c) {
        const cdf sj = S[hs_rowbase((j - c) / CL, c, CL) + j];
        dfl t = cre(sj);
        t = df_fma(t, df_neg(cre(vpj)), cre(wpj));
        t = df_fma(t, df_neg(cim(vpj)), cim(wpj));
        t = df_fma(t, df_neg(cre(vpj)), cre(wpj));
        t = df_fma(t, df_neg(cim(vpj)), cim(wpj));
        e.d[(long)b * m + j] = ldexp(df_to(t), ex);
      }
    }
    if (CL > 1) cluster.sync();
    else __syncthreads();
    const int n = m - j - 1;
    {
      // |x|^2 and the reflector scalars by warp 0 alone (the other warps clear the partial
      // products meanwhile), handed over through shared memory: lanes take entries
      // lane + 32 u + 128 k in four independent chains, then a butterfly of double-float sums;
      // -alpha = e^{i arg x0} |x|, v = (x - alpha e1) / sqrt(2 |x| (|x| + |x0|))
      for (int i = tid; i < n; i += NT) pv[j + 1 + i] = cdf_zero();
      if (warp > 0 && lag) {
        // meanwhile the other warps apply the pending rank-2 update of step j-1 to the own rows'
        // entries k in [j+1, g] (contiguous segments over NT - 32 threads), so that the
        // matrix-vector passes below read updated values and need only v_j
        const int q0 = hs_qfirst(j, c, CL);
        const int nr = max(0, nq - q0);
        const int g0 = c + CL * q0;
        const int E1 = nr * (g0 - j) + CL * nr * (nr - 1) / 2;
        if (E1 > 0) {
          const int lt = tid - 32;
          const int L = hs_seglen<NT - 32>(E1);
          const int e0 = hs_seg(lt, E1, L), e1 = hs_seg(lt + 1, E1, L);
          if (e0 < e1) {
            int lo = 0, hi = nr - 1;
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (mid * (g0 - j) + CL * mid * (mid - 1) / 2 <= e0) lo = mid;
              else hi = mid - 1;
            }
            const int i = lo;
            const int Pi = i * (g0 - j) + CL * i * (i - 1) / 2;
            int g = g0 + CL * i;
            int k = j + 1 + (e0 - Pi);
            cdf* row = S + hs_rowbase(q0 + i, c, CL);
            if constexpr (GS) {
              // HS_U elements at a time: their addresses first, then independent loads
              // (several row-store accesses in flight per thread), then the updates
              for (int el = e0; el < e1; el += HS_U) {
                cdf* p[HS_U];
                int kk[HS_U], gg[HS_U];
  #pragma unroll
                for (int u = 0; u < HS_U; ++u) {
                  p[u] = row + k;
                  kk[u] = k;
                  gg[u] = g;
                  if (++k > g) {
                    row += g + 1;
                    g += CL;
                    k = j + 1;
                  }
                }
                cdf a[HS_U];
  #pragma unroll
                for (int u = 0; u < HS_U; ++u)
                  if (el + u < e1) a[u] = *p[u];
  #pragma unroll
                for (int u = 0; u < HS_U; ++u)
                  if (el + u < e1) {
                    cdf x = cdf_lag(a[u], vp[gg[u]], wp[gg[u]], vp[kk[u]], wp[kk[u]]);
                    if (kk[u] == gg[u]) {
                      x.ih = 0.f;
                      x.il = 0.f;
                    }
                    *p[u] = x;
                  }
              }
            } else {
              cdf vg = vp[g], wg = wp[g];
              for (int el = e0; el < e1; ++el) {
                cdf a = cdf_lag(row[k], vg, wg, vp[k], wp[k]);
                if (k == g) {
                  a.ih = 0.f;
                  a.il = 0.f;
                }
                row[k] = a;
                if (++k > g) {
                  row += g + 1;
                  g += CL;
                  k = j + 1;
                  if (el + 1 < e1) {
                    vg = vp[g];
                    wg = wp[g];
                  }
                }
              }
            }
          }
        }
      }
      if (warp == 0) {
        dfl pa[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        for (int i0 = 0; i0 < n; i0 += 128) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = i0 + 32 * u + lane;
            if (i < n) {
              const cdf x = v[j + 1 + i];
              pa[u] = df_fma(pa[u], cre(x), cre(x));
              pa[u] = df_fma(pa[u], cim(x), cim(x));
            }
          }
        }
        dfl nrm2d = df_add(df_add(pa[0], pa[1]), df_add(pa[2], pa[3]));
        for (int o = 16; o > 0; o >>= 1) nrm2d = df_add(nrm2d, df_shfl_xor(nrm2d, o));
        cdf am = cdf_zero();  // -alpha
        dfl vinv{0.f, 0.f};
        if (nrm2d.hi > 0.f) {
          const cdf x0 = v[j + 1];
          const dfl nrm = df_sqrt_nodiv(nrm2d);
          const dfl ax2 = df_fma(df_fma(dfl{0.f, 0.f}, cre(x0), cre(x0)), cim(x0), cim(x0));
          dfl phr{1.f, 0.f}, phi{0.f, 0.f}, ax0{0.f, 0.f};
          if (ax2.hi > 0.f) {
            const dfl iax = df_rsqrt(ax2);  // 1 / |x0|
            ax0 = df_mul(ax2, iax);
            phr = df_mul(cre(x0), iax);
            phi = df_mul(cim(x0), iax);
          }
          am = cdf_make(df_mul(phr, nrm), df_mul(phi, nrm));
          vinv = df_rsqrt(df_mul(df_add(nrm, nrm), df_add(nrm, ax0)));
        }
        if (lane == 0) {
          s_am = am;
          s_vinv = vinv;
          if (c == 0) {
            const double2 al = cdf_to(am);
            e.alpha[(long)b * m + j] = make_double2(-ldexp(al.x, ex), -ldexp(al.y, ex));
          }
        }
      }
      __syncthreads();
      const cdf am = s_am;
      const dfl vinv = s_vinv;
      for (int i = tid; i < n; i += NT) {
        cdf vi = v[j + 1 + i];
        if (i == 0) vi = cdf_add(vi, am);
        vi = cdf_scale(vi, vinv);
        v[j + 1 + i] = vi;
        // read by the FP32 back-transform after this kernel: evict-first, so the
        // row store keeps the L2
        if (c == 0) __stcs(Hv32 + (long)j * m + j + 1 + i, make_float2(vi.rh, vi.ih));
      }
    }
    __syncthreads();

    // row pass (as in k_hetrd_smem, the pending update already applied)
    const int q0 = hs_qfirst(j, c, CL);
    for (int q = q0 + tid; q < nq; q += NT) vown[q] = v[c + CL * q];
    const int nr = max(0, nq - q0);
    const int g0 = c + CL * q0;
    const int E1 = nr * (g0 - j) + CL * nr * (nr - 1) / 2;
    if (E1 > 0) {
      const int L1 = hs_seglen<NT>(E1);
      const int e0 = hs_seg(tid, E1, L1), e1 = hs_seg(tid + 1, E1, L1);
      if (e0 < e1) {
        int lo = 0, hi = nr - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (mid * (g0 - j) + CL * mid * (mid - 1) / 2 <= e0) lo = mid;
          else hi = mid - 1;
        }
        int i = lo;
        const int Pi = i * (g0 - j) + CL * i * (i - 1) / 2;
        int g = g0 + CL * i;
        int k = j + 1 + (e0 - Pi);
        const cdf* row = S + hs_rowbase(q0 + i, c, CL);
        if constexpr (GS) {
          bool whole = (e0 == Pi), first = true, pending = false;
          cdf acc = cdf_zero();
          for (int el = e0; el < e1; el += HS_U) {
            const cdf* p[HS_U];
            int kk[HS_U], gend[HS_U];  // gend: the row an element ends, else -1
  #pragma unroll
            for (int u = 0; u < HS_U; ++u) {
              p[u] = row + k;
              kk[u] = k;
              gend[u] = -1;
              if (++k > g) {
                gend[u] = g;
                row += g + 1;
                g += CL;
                k = j + 1;
              }
            }
            cdf a[HS_U];
  #pragma unroll
            for (int u = 0; u < HS_U; ++u)
              if (el + u < e1) a[u] = *p[u];
  #pragma unroll
            for (int u = 0; u < HS_U; ++u)
              if (el + u < e1) {
                cdf_fma(acc, a[u], v[kk[u]]);
                pending = gend[u] < 0;
                if (!pending) {
                  if (whole) pv[gend[u]] = acc;
                  else slotF[tid] = acc;
                  first = false;
                  whole = true;
                  acc = cdf_zero();
                }
              }
          }
          if (pending) {
            if (first) slotF[tid] = acc;
            else slotL[tid] = acc;
          }
        } else {
          bool whole = (e0 == Pi), first = true;
          cdf acc = cdf_zero();
          for (int el = e0; el < e1; ++el) {
            cdf_fma(acc, row[k], v[k]);
            if (++k > g) {
              if (whole) pv[g] = acc;
              else slotF[tid] = acc;
              first = false;
              whole = true;
              acc = cdf_zero();
              row += g + 1;
              g += CL;
              k = j + 1;
            }
          }
          if (k != j + 1) {
            if (first) slotF[tid] = acc;
            else slotL[tid] = acc;
          }
        }
      }
      __syncthreads();
      // rows split between threads: 8 lanes per row sum every 8th slot, then a 3-level butterfly
      for (int base = 0; base < nr; base += NT / 8) {
        const int i = base + (tid >> 3), q = tid & 7;
        cdf sacc = cdf_zero();
        bool split = false;
        if (i < nr) {
          const int Pi = i * (g0 - j) + CL * i * (i - 1) / 2;
          const int len = g0 + CL * i - j;
          const int ta = hs_owner(Pi, L1), tb = hs_owner(Pi + len - 1, L1);
          split = ta != tb;
          if (split) {
            if (q == 0) sacc = (hs_seg(ta, E1, L1) == Pi) ? slotF[ta] : slotL[ta];
            for (int t = ta + 1 + q; t <= tb; t += 8)
              if (hs_seg(t, E1, L1) < hs_seg(t + 1, E1, L1)) sacc = cdf_add(sacc, slotF[t]);
          }
        }
        for (int o = 1; o < 8; o <<= 1) sacc = cdf_add(sacc, cdf_shfl_xor(sacc, o));
        if (split && q == 0) pv[g0 + CL * i] = sacc;
      }
    }
    __syncthreads();

    // column pass
    const int cb = CP[j + 1];
    const int E2 = CP[m] - cb;
    if (E2 > 0) {
      const int L2 = hs_seglen<NT>(E2);
      const int e0 = hs_seg(tid, E2, L2), e1 = hs_seg(tid + 1, E2, L2);
      if (e0 < e1) {
        int lo = j + 1, hi = m - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (CP[mid] <= cb + e0) lo = mid;
          else hi = mid - 1;
        }
        int k = lo;
        int o = cb + e0 - CP[k];
        int cnt = CP[k + 1] - CP[k];
        int q = hs_qfirst(k, c, CL) + o;
        int g = c + CL * q, base = hs_rowbase(q, c, CL);
        if constexpr (GS) {
          bool whole = (o == 0), first = true, pending = false;
          cdf acc = cdf_zero();
          for (int el = e0; el < e1; el += HS_U) {
            int addr[HS_U], qq[HS_U], kend[HS_U];  // kend: the column an element ends, else -1
  #pragma unroll
            for (int u = 0; u < HS_U; ++u) {
              addr[u] = base + k;
              qq[u] = q;
              kend[u] = -1;
              base += g + 1;
              g += CL;
              ++q;
              if (++o == cnt) {
                kend[u] = k;
                if (el + u + 1 < e1) {
                  do {
                    ++k;
                  } while (CP[k + 1] == CP[k]);
                  cnt = CP[k + 1] - CP[k];
                  q = hs_qfirst(k, c, CL);
                  g = c + CL * q;
                  base = hs_rowbase(q, c, CL);
                  o = 0;
                }
              }
            }
            cdf a[HS_U];
  #pragma unroll
            for (int u = 0; u < HS_U; ++u)
              if (el + u < e1) a[u] = S[addr[u]];
  #pragma unroll
            for (int u = 0; u < HS_U; ++u)
              if (el + u < e1) {
                cdf_fmac(acc, a[u], vown[qq[u]]);
                pending = kend[u] < 0;
                if (!pending) {
                  if (whole) pv[kend[u]] = cdf_add(pv[kend[u]], acc);
                  else slotF[tid] = acc;
                  first = false;
                  whole = true;
                  acc = cdf_zero();
                }
              }
          }
          if (pending) {
            if (first) slotF[tid] = acc;
            else slotL[tid] = acc;
          }
        } else {
          bool whole = (o == 0), first = true;
          cdf acc = cdf_zero();
          for (int el = e0; el < e1; ++el) {
            cdf_fmac(acc, S[base + k], vown[q]);
            base += g + 1;
            g += CL;
            ++q;
            if (++o == cnt) {
              if (whole) pv[k] = cdf_add(pv[k], acc);
              else slotF[tid] = acc;
              first = false;
              whole = true;
              acc = cdf_zero();
              if (el + 1 < e1) {
                do {
                  ++k;
                } while (CP[k + 1] == CP[k]);
                cnt = CP[k + 1] - CP[k];
                q = hs_qfirst(k, c, CL);
                g = c + CL * q;
                base = hs_rowbase(q, c, CL);
                o = 0;
              }
            }
          }
          if (o != cnt && o != 0) {
            if (first) slotF[tid] = acc;
            else slotL[tid] = acc;
          }
        }
      }
      __syncthreads();
      for (int k = j + 1 + tid; k < m; k += NT) {
        const int cnt = CP[k + 1] - CP[k];
        if (cnt == 0) continue;
        const int s0 = CP[k] - cb;
        const int ta = hs_owner(s0, L2), tb = hs_owner(s0 + cnt - 1, L2);
        if (ta == tb) continue;
        cdf sacc = (hs_seg(ta, E2, L2) == s0) ? slotF[ta] : slotL[ta];
        for (int t = ta + 1; t <= tb; ++t)
          if (hs_seg(t, E2, L2) < hs_seg(t + 1, E2, L2)) sacc = cdf_add(sacc, slotF[t]);
        pv[k] = cdf_add(pv[k], sacc);
      }
    }
    if (CL > 1) cluster.sync();
    else __syncthreads();

    // p = 2 sum of the parts; K = Re(v^H p); w = p - K v
    dfl kp{0.f, 0.f};
    for (int i = j + 1 + tid; i < m; i += NT) {
      cdf pi = cdf_zero();
#pragma unroll
      for (int rr = 0; rr < CL; ++rr) {
        const cdf* src = (CL > 1) ? cluster.map_shared_rank(pv, rr) : pv;
        pi = cdf_add(pi, src[i]);
      }
      pi = cdf_make(dfl{2.f * pi.rh, 2.f * pi.rl}, dfl{2.f * pi.ih, 2.f * pi.il});
      w[i] = pi;
      const cdf vi = v[i];
      kp = df_fma(kp, cre(vi), cre(pi));
      kp = df_fma(kp, cim(vi), cim(pi));
    }
    const dfl K = df_block_sum(kp, red);
    const dfl nK = df_neg(K);
    for (int i = j + 1 + tid; i < m; i += NT) {
      const cdf vi = v[i];
      cdf wi = w[i];
      wi = cdf_make(df_fma(cre(wi), cre(vi), nK), df_fma(cim(wi), cim(vi), nK));
      w[i] = wi;
    }
    __syncthreads();
  }
  if (tid == 0 && ((m - 1) % CL) == c) {
    const cdf sl = S[hs_rowbase((m - 1 - c) / CL, c, CL) + m - 1];
    dfl t = cre(sl);
    if (m > 1) {
      const cdf vq = bufV[((m - 2) & 1) * m + m - 1], wq = bufW[((m - 2) & 1) * m + m - 1];
      t = df_fma(t, df_neg(cre(vq)), cre(wq));
      t = df_fma(t, df_neg(cim(vq)), cim(wq));
      t = df_fma(t, df_neg(cre(vq)), cre(wq));
      t = df_fma(t, df_neg(cim(vq)), cim(wq));
    }
    e.d[(long)b * m + m - 1] = ldexp(df_to(t), ex);
  }
  __threadfence();
  if (CL > 1) cluster.sync();
  else __syncthreads();
  if (c == 0 && tid == 0) {
    double2 dl = make_double2(1, 0);
    e.delta[(long)b * m] = dl;
    double tn = 0;
    for (int jj = 0; jj < m - 1; ++jj) {
      const double2 a = __ldcg(e.alpha + (long)b * m + jj);
      const double aa = sqrt(cabs2(a));
      e.f[(long)b * m + jj] = aa;
      if (aa > 0) dl = cmul(dl, cscale(a, 1.0 / aa));
      e.delta[(long)b * m + jj + 1] = dl;
    }
    for (int jj = 0; jj < m; ++jj) {
      const double fl = (jj > 0) ? e.f[(long)b * m + jj - 1] : 0.0, fr = (jj < m - 1) ? e.f[(long)b * m + jj] : 0.0;
      tn = fmax(tn, fabs(__ldcg(e.d + (long)b * m + jj)) + fl + fr);
    }
    e.tnorm[b] = tn;
  }
}

// ---------------------------------------------------------------------------
// One-pass double-float reduction with the rows in global memory (L2): the
// same steps as k_hetrd_df (the update of step j-1 applied lazily in step j),
// but its three sweeps of the trailing triangle (the pending rank-2 update,
// the row and the column matrix-vector passes) become one.  Warps take strips
// of HF_SR consecutive own rows and walk them 32 columns at a time, lane l on
// column k0 + l (512-byte coalesced loads); each element is updated, stored
// once and used twice:
//   row part     p_g += a_gk v_k              (k <= g; lane-local over the
//                                              strip, reduced across lanes once
//                                              per strip)
//   column part  p_k += conj(a_gk) v_g        (k < g; the lane's column, summed
//                                              over the strip's rows, added to a
//                                              warp-private partial of p)
// The warp partials are summed per column after the sweep.  The strips go to
// the warps by a schedule fixed for every step in the prologue: longest first
// to the least loaded warp, which balances the sweep to about one short strip
// and keeps every sum in a fixed order.
// ---------------------------------------------------------------------------
constexpr int HF_SR = 4;  // own rows per strip

// strips of the sweep of one CTA (the most of any CTA of a cluster of CL)
static int hetrd_df1_strips(int m, int CL) { return (hs_own_rows(m, 0, CL) + HF_SR - 1) / HF_SR; }
// v[2], w[2], p, the warp partials [NW]; with `sched`, the strip schedule [m-1][strips] after them
static size_t hetrd_df1_smem_bytes(int m, int nt, int CL = 1, bool sched = false) {
  const size_t base = (size_t)(5 + nt / 32) * (size_t)m * sizeof(double2);
  return sched ? base + (((size_t)(m - 1) * hetrd_df1_strips(m, CL) + 15) & ~(size_t)15) : base;
}

template <int CL, int NT>
__global__ void __launch_bounds__(NT, 1) k_hetrd_df1(const double2* __restrict__ G, long ldg, long sG, int m,
                                                     int s_elems, EigScratch e, int use_sched) {
  extern __shared__ __align__(16) cdf dsm[];
  constexpr int NW = NT / 32;
  static_assert(HF_SR == 4, "the row-sum reduction below is written for strips of four rows");
  cdf* S = (cdf*)e.Sg + (long)blockIdx.x * s_elems;  // own rows, packed, private to this CTA
  cdf* bufV = dsm;                                   // [2][m] v of this and of the previous step
  cdf* bufW = bufV + 2 * m;                          // [2][m] w
  cdf* pv = bufW + 2 * m;                            // [m] this CTA's part of p
  cdf* cpart = pv + m;                               // [NW][m] column parts of p, one per warp
  uint8_t* sched = (uint8_t*)(cpart + NW * m);       // [m-1][NSM] the warp of every strip of every step
  __shared__ dfl red[NW];
  __shared__ int s_exp;
  cg::cluster_group cluster = cg::this_cluster();
  const int c = (CL > 1) ? (int)cluster.block_rank() : 0;
  const int b = (int)blockIdx.x / CL;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  G += (long)b * sG;
  float2* Hv32 = (float2*)e.Hv + (long)b * m * m;
  const int nq = hs_own_rows(m, c, CL);
  const int NSM = (hs_own_rows(m, 0, CL) + HF_SR - 1) / HF_SR;

  // The strip schedule of every step, fixed before the first (so the column parts are
  // summed in the same order on every run): longest strip first to the least loaded
  // warp (lowest index on ties), a strip costing its 32-column chunks x 4 rows plus one
  // for its row-sum reduction.  Without room for it, the warps take the strips in snake
  // order (w, 2 NW - 1 - w, 2 NW + w, ...).
  if (use_sched) {
    for (int jj = tid; jj < m - 1; jj += NT) {
      const int q0j = hs_qfirst(jj, c, CL);
      const int nsj = (max(0, nq - q0j) + HF_SR - 1) / HF_SR;
      int load[NW];
#pragma unroll
      for (int w2 = 0; w2 < NW; ++w2) load[w2] = 0;
      for (int t = 0; t < nsj; ++t) {
        const int sj = nsj - 1 - t;
        const int glast = c + CL * min(q0j + sj * HF_SR + HF_SR - 1, nq - 1);
        const int cost = ((glast - jj) + 31) / 32 * HF_SR + 1;
        int wb = 0, lb = load[0];
#pragma unroll
        for (int w2 = 1; w2 < NW; ++w2)
          if (load[w2] < lb) {
            lb = load[w2];
            wb = w2;
          }
#pragma unroll
        for (int w2 = 0; w2 < NW; ++w2)
          if (w2 == wb) load[w2] += cost;
        sched[jj * NSM + sj] = (uint8_t)wb;
      }
    }
  }

  // power-of-two scale from the largest diagonal entry (identical in every CTA)
  {
    double mx = 0;
    for (int i = tid; i < m; i += NT) mx = fmax(mx, fabs(__ldcg(G + (long)i * ldg + i).x));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ double wmx[NW];
    if (lane == 0) wmx[warp] = mx;
    __syncthreads();
    if (tid == 0) {
      double t = 0;
      for (int w = 0; w < NW; ++w) t = fmax(t, wmx[w]);
      int ex = 0;
      if (t > 0 && isfinite(t)) frexp(t, &ex);
      s_exp = ex;
    }
    __syncthreads();
  }
  const int ex = s_exp;
  for (int q = warp; q < nq; q += NW) {
    const int g = c + CL * q;
    const double2* src = G + (long)g * ldg;
    cdf* dst = S + hs_rowbase(q, c, CL);
    for (int k = lane; k <= g; k += 32) {
      const double2 x = __ldcg(src + k);
      dst[k] = cdf_from(make_double2(ldexp(x.x, -ex), ldexp(x.y, -ex)));
    }
  }
  for (int i = tid; i < (5 + NW) * m; i += NT) bufV[i] = cdf_zero();
  if (CL > 1) cluster.sync();
  else __syncthreads();

  for (int j = 0; j < m - 1; ++j) {
    const int cur = j & 1;
    cdf* v = bufV + cur * m;
    cdf* w = bufW + cur * m;
    const cdf* vp = bufV + (cur ^ 1) * m;
    const cdf* wp = bufW + (cur ^ 1) * m;
    const bool lag = j > 0;
    // column j of A^(j) (the pending update applied) to every CTA's v; the diagonal d_j
    {
      const cdf vpj = vp[j], wpj = wp[j];
      for (int q = hs_qfirst(j, c, CL) + tid; q < nq; q += NT) {
        const int g = c + CL * q;
        cdf a = S[hs_rowbase(q, c, CL) + j];
        if (lag) a = cdf_lag(a, vp[g], wp[g], vpj, wpj);
#pragma unroll
        for (int rr = 0; rr < CL; ++rr) {
          cdf* dst = (CL > 1) ? cluster.map_shared_rank(v, rr) : v;
          dst[g] = a;
        }
      }
      if (tid == 0 && (j % CL) == c) {
        const cdf sj = S[hs_rowbase((j - c) / CL, c, CL) + j];
        dfl t = cre(sj);
        t = df_fma(t, df_neg(cre(vpj)), cre(wpj));
        t = df_fma(t, df_neg(cim(vpj)), cim(wpj));
        t = df_fma(t, df_neg(cre(vpj)), cre(wpj));
        t = df_fma(t, df_neg(cim(vpj)), cim(wpj));
        e.d[(long)b * m + j] = ldexp(df_to(t), ex);
      }
    }
    if (CL > 1) cluster.sync();
    else __syncthreads();
    const int n = m - j - 1;
    // the reflector: |x|^2 by the whole block (fixed order, so both CTAs agree), then every
    // thread forms -alpha = e^{i arg x0} |x| and 1 / sqrt(2 |x| (|x| + |x0|)) itself
    {
      const cdf x0 = v[j + 1];
      dfl t{0.f, 0.f};
      for (int i = tid; i < n; i += NT) {
        const cdf x = v[j + 1 + i];
        t = df_fma(t, cre(x), cre(x));
        t = df_fma(t, cim(x), cim(x));
      }
      const dfl nrm2d = df_block_sum(t, red);
      cdf am = cdf_zero();  // -alpha
      dfl vinv{0.f, 0.f};
      if (nrm2d.hi > 0.f) {
        const dfl nrm = df_sqrt_nodiv(nrm2d);
        const dfl ax2 = df_fma(df_fma(dfl{0.f, 0.f}, cre(x0), cre(x0)), cim(x0), cim(x0));
        dfl phr{1.f, 0.f}, phi{0.f, 0.f}, ax0{0.f, 0.f};
        if (ax2.hi > 0.f) {
          const dfl iax = df_rsqrt(ax2);  // 1 / |x0|
          ax0 = df_mul(ax2, iax);
          phr = df_mul(cre(x0), iax);
          phi = df_mul(cim(x0), iax);
        }
        am = cdf_make(df_mul(phr, nrm), df_mul(phi, nrm));
        vinv = df_rsqrt(df_mul(df_add(nrm, nrm), df_add(nrm, ax0)));
      }
      if (tid == 0 && c == 0) {
        const double2 al = cdf_to(am);
        e.alpha[(long)b * m + j] = make_double2(-ldexp(al.x, ex), -ldexp(al.y, ex));
      }
      for (int i = tid; i < n; i += NT) {
        cdf vi = v[j + 1 + i];
        if (i == 0) vi = cdf_add(vi, am);
        vi = cdf_scale(vi, vinv);
        v[j + 1 + i] = vi;
        // read by the FP32 back-transform after this kernel: evict-first, so the
        // row store keeps the L2
        if (c == 0) __stcs(Hv32 + (long)j * m + j + 1 + i, make_float2(vi.rh, vi.ih));
      }
    }
    __syncthreads();

    // the sweep: pending update, store, row and column parts of p = A^(j) v
    const int q0 = hs_qfirst(j, c, CL);
    const int nstrip = (max(0, nq - q0) + HF_SR - 1) / HF_SR;
    cdf* cp = cpart + warp * m;
    const uint8_t* own = sched + j * NSM;
    unsigned mine = 0;  // this warp's strips among s0 .. s0 + 31 (with the schedule)
    for (int s0 = 0, it = 0; s0 < nstrip;) {
      int s;
      if (use_sched) {
        if (it == 0) {
          const int sl = s0 + lane;
          mine = __ballot_sync(0xffffffffu, sl < nstrip && own[sl] == warp);
        }
        if (mine == 0) {  // the next group of 32 strips
          s0 += 32;
          it = 0;
          continue;
        }
        const int bit = 31 - __clz(mine);
        mine &= ~(1u << bit);
        s = s0 + bit;
        it = 1;
      } else {
        s = s0 + (((s0 / NW) & 1) ? NW - 1 - warp : warp);  // snake order
        s0 += NW;
        if (s >= nstrip) continue;
      }
      const int qs = q0 + s * HF_SR;
      int gr[HF_SR];
      cdf* rowp[HF_SR];
#pragma unroll
      for (int r = 0; r < HF_SR; ++r) {
        const int q = min(qs + r, nq - 1);
        gr[r] = (qs + r < nq) ? c + CL * q : -1;  // -1: no row (past the last own row)
        rowp[r] = S + hs_rowbase(q, c, CL);
      }
      const int glast = c + CL * min(qs + HF_SR - 1, nq - 1);
      cdf racc[HF_SR];
#pragma unroll
      for (int r = 0; r < HF_SR; ++r) racc[r] = cdf_zero();
      for (int k0 = j + 1; k0 <= glast; k0 += 32) {
        const int k = k0 + lane;
        cdf a[HF_SR];
#pragma unroll
        for (int r = 0; r < HF_SR; ++r)
          if (k <= gr[r]) a[r] = rowp[r][k];
        if (k <= glast) {
          const cdf vk = v[k];
          cdf vpk = cdf_zero(), wpk = cdf_zero();
          if (lag) {
            vpk = vp[k];
            wpk = wp[k];
          }
          cdf cacc = cdf_zero();
#pragma unroll
          for (int r = 0; r < HF_SR; ++r) {
            if (k <= gr[r]) {
              const int g = gr[r];
              cdf x = a[r];
              if (lag) {
                x = cdf_lag(x, vp[g], wp[g], vpk, wpk);
                if (k == g) {
                  x.ih = 0.f;
                  x.il = 0.f;
                }
                rowp[r][k] = x;
              }
              cdf_fma_acc(racc[r], x, vk);
              if (k < g) cdf_fmac_acc(cacc, x, v[g]);
            }
          }
          if (k < glast) cp[k] = cdf_add(cp[k], cacc);
        }
      }
      // row sums across the lanes: halve the rows twice (lanes 16-31 keep rows 2, 3; then
      // lanes with bit 3 set keep the odd row), then a 3-level butterfly; lane l ends with
      // row l / 8
      {
        const bool u16 = (lane & 16) != 0, u8 = (lane & 8) != 0;
        cdf k0v = u16 ? racc[2] : racc[0], k1v = u16 ? racc[3] : racc[1];
        const cdf s0v = u16 ? racc[0] : racc[2], s1v = u16 ? racc[1] : racc[3];
        k0v = cdf_add(k0v, cdf_shfl_xor(s0v, 16));
        k1v = cdf_add(k1v, cdf_shfl_xor(s1v, 16));
        cdf kk = u8 ? k1v : k0v;
        const cdf ss = u8 ? k0v : k1v;
        kk = cdf_add(kk, cdf_shfl_xor(ss, 8));
        for (int o = 4; o > 0; o >>= 1) kk = cdf_add(kk, cdf_shfl_xor(kk, o));
        const int r = lane >> 3;
        int gsel = gr[0];
#pragma unroll
        for (int rr = 1; rr < HF_SR; ++rr)
          if (r == rr) gsel = gr[rr];
        if ((lane & 7) == 0 && gsel >= 0) pv[gsel] = kk;
      }
    }
    __syncthreads();
    // p of this CTA: its rows' row parts plus every warp's column parts; the partials are
    // cleared for the next step as they are read
    for (int k = j + 1 + tid; k < m; k += NT) {
      cdf part[NW];  // all loads first, then a pairwise sum (fixed order), then the clearing
#pragma unroll
      for (int w2 = 0; w2 < NW; ++w2) part[w2] = cpart[w2 * m + k];
#pragma unroll
      for (int h = NW / 2; h > 0; h >>= 1)
#pragma unroll
        for (int w2 = 0; w2 < h; ++w2) part[w2] = cdf_add(part[w2], part[w2 + h]);
#pragma unroll
      for (int w2 = 0; w2 < NW; ++w2) cpart[w2 * m + k] = cdf_zero();
      pv[k] = (k % CL == c) ? cdf_add(pv[k], part[0]) : part[0];
    }
    if (CL > 1) cluster.sync();
    else __syncthreads();
    // p = 2 sum of the parts; K = Re(v^H p); w = p - K v
    dfl kp{0.f, 0.f};
    for (int i = j + 1 + tid; i < m; i += NT) {
      cdf pi = cdf_zero();
#pragma unroll
      for (int rr = 0; rr < CL; ++rr) {
        const cdf* src = (CL > 1) ? cluster.map_shared_rank(pv, rr) : pv;
        pi = cdf_add(pi, src[i]);
      }
      pi = cdf_make(dfl{2.f * pi.rh, 2.f * pi.rl}, dfl{2.f * pi.ih, 2.f * pi.il});
      w[i] = pi;
      const cdf vi = v[i];
      kp = df_fma(kp, cre(vi), cre(pi));
      kp = df_fma(kp, cim(vi), cim(pi));
    }
    const dfl K = df_block_sum(kp, red);
    const dfl nK = df_neg(K);
    for (int i = j + 1 + tid; i < m; i += NT) {
      const cdf vi = v[i];
      cdf wi = w[i];
      wi = cdf_make(df_fma(cre(wi), cre(vi), nK), df_fma(cim(wi), cim(vi), nK));
      w[i] = wi;
    }
    __syncthreads();
  }
  if (tid == 0 && ((m - 1) % CL) == c) {
    const cdf sl = S[hs_rowbase((m - 1 - c) / CL, c, CL) + m - 1];
    dfl t = cre(sl);
    if (m > 1) {
      const cdf vq = bufV[((m - 2) & 1) * m + m - 1], wq = bufW[((m - 2) & 1) * m + m - 1];
      t = df_fma(t, df_neg(cre(vq)), cre(wq));
      t = df_fma(t, df_neg(cim(vq)), cim(wq));
      t = df_fma(t, df_neg(cre(vq)), cre(wq));
      t = df_fma(t, df_neg(cim(vq)), cim(wq));
    }
    e.d[(long)b * m + m - 1] = ldexp(df_to(t), ex);
  }
  __threadfence();
  if (CL > 1) cluster.sync();
  else __syncthreads();
  if (c == 0 && tid == 0) {
    double2 dl = make_double2(1, 0);
    e.delta[(long)b * m] = dl;
    double tn = 0;
    for (int jj = 0; jj < m - 1; ++jj) {
      const double2 a = __ldcg(e.alpha + (long)b * m + jj);
      const double aa = sqrt(cabs2(a));
      e.f[(long)b * m + jj] = aa;
      if (aa > 0) dl = cmul(dl, cscale(a, 1.0 / aa));
      e.delta[(long)b * m + jj + 1] = dl;
    }
    for (int jj = 0; jj < m; ++jj) {
      const double fl = (jj > 0) ? e.f[(long)b * m + jj - 1] : 0.0, fr = (jj < m - 1) ? e.f[(long)b * m + jj] : 0.0;
      tn = fmax(tn, fabs(__ldcg(e.d + (long)b * m + jj)) + fl + fr);
    }
    e.tnorm[b] = tn;
  }
}

// Number of eigenvalues below x of the symmetric tridiagonal (d, f) (scaled
// to norm ~1): sign changes of the Sturm sequence P_0 = 1, P_1 = d_0 - x,
// P_i = (d_{i-1} - x) P_{i-1} - f_{i-2}^2 P_{i-2}, i.e. negative ratios
// q_i = P_i / P_{i-1}; a zero ratio is replaced by -pivmin.  The pair
// (P_i, P_{i-1}) is rescaled by powers of two to stay in range.
__device__ __forceinline__ int sturm_count(const double* d, const double* f2, int m, double x, double pivmin) {
  double pm = 1.0, p = d[0] - x;
  if (p == 0.0) p = -pivmin;
  int cnt = (int)((unsigned long long)__double_as_longlong(p) >> 63);
  for (int i = 1; i < m; ++i) {
    double pn = fma(d[i] - x, p, -f2[i - 1] * pm);
    long long bn = __double_as_longlong(pn);
    if ((bn << 1) == 0) {  // zero ratio
      pn = -pivmin * p;
      bn = __double_as_longlong(pn);
    }
    cnt += (int)((unsigned long long)(bn ^ __double_as_longlong(p)) >> 63);
    pm = p;
    p = pn;
    // keep the pair in range: rescale both by a power of two when the exponent of p leaves +-600
    const int ex = (int)((bn >> 52) & 0x7ff) - 1023;
    if (ex > 600 || ex < -600) {
      const double sc = __longlong_as_double((long long)(1023 - ex) << 52);
      p *= sc;
      pm *= sc;
    }
  }
  return cnt;
}

// The reduced-precision counts below clamp every ratio q_i of magnitude
// below 2^-64 to -2^-64 (a perturbation of d_{i-1} by at most 2^-63 ||T||)
// and rescale the pair by a power of two whenever |P_i| leaves
// [2^-32, 2^32].  The clamp bounds |P_{i-1} / P_i| by 2^64, so neither member
// of the pair can overflow or become subnormal.
constexpr float kSturmPiv = 0x1p-64f;

// FP32 count.  df[i] = (d_i, f_{i-1}^2) with f_{-1} = 0.  A computed count is
// the exact count of a tridiagonal whose d_i - x and f^2 moved by a few units
// in the last place (the recurrence is backward stable), i.e. of one within
// about 5e-7 ||T|| of the given one, so a bracket from FP32 counts holds the
// eigenvalue once widened by a margin above that.
__device__ __forceinline__ int sturm_count_f32(const float2* __restrict__ df, int m, float x) {
  float p = 1.0f, pm = 0.0f;
  int cnt = 0;
#pragma unroll 4
  for (int i = 0; i < m; ++i) {
    const float2 v = df[i];
    float pn = fmaf(v.x - x, p, -v.y * pm);
    if (fabsf(pn) < kSturmPiv * fabsf(p)) pn = -kSturmPiv * p;
    cnt += (int)((__float_as_uint(pn) ^ __float_as_uint(p)) >> 31);
    pm = p;
    p = pn;
    const float an = fabsf(pn);
    if (an > 0x1p32f || an < 0x1p-32f) {
      const int ex = (int)((__float_as_uint(pn) >> 23) & 0xffu) - 127;
      const float sc = __uint_as_float((unsigned)(127 - ex) << 23);
      p *= sc;
      pm *= sc;
    }
  }
  return cnt;
}

// The same count in double-float arithmetic (each value hi + lo, two FP32
// numbers, about 48 significant bits) on the FP32 pipe, which on GB300 issues
// 64 times the FP64 rate.  v[i] = (d_i hi, d_i lo, f_{i-1}^2 hi, f_{i-1}^2 lo).
// Per step: d_i - x by TwoSum of the high parts plus the low parts; the two
// products by TwoProduct (FMA) of the high parts plus the cross terms; their
// difference by TwoSum and one renormalisation.  Every operation is exact up
// to about 2^-47 of its operands, so a computed count is the exact count of a
// tridiagonal within about 1e-14 ||T|| of the given one.
__device__ __forceinline__ int sturm_count_df(const float4* __restrict__ v, int m, dfl x) {
  float ph = 1.0f, pl = 0.0f, qh = 0.0f, ql = 0.0f;  // P_i, P_{i-1}
  int cnt = 0;
#pragma unroll 2
  for (int i = 0; i < m; ++i) {
    const float4 c = v[i];
    const float th = c.x - x.hi;  // t = d_i - x, not renormalised
    const float tb = th - c.x;
    const float tl = ((c.x - (th - tb)) + (-x.hi - tb)) + (c.y - x.lo);
    const float a = th * ph;  // t P_i
    const float ae = fmaf(tl, ph, fmaf(th, pl, fmaf(th, ph, -a)));
    const float b = c.z * qh;  // f^2 P_{i-1}
    const float be = fmaf(c.w, qh, fmaf(c.z, ql, fmaf(c.z, qh, -b)));
    const float sh = a - b;
    const float sb = sh - a;
    const float sl = ((a - (sh - sb)) + (-b - sb)) + (ae - be);
    float nh = sh + sl;
    float nl = sl - (nh - sh);
    if (fabsf(nh) < kSturmPiv * fabsf(ph)) {
      nh = -kSturmPiv * ph;
      nl = -kSturmPiv * pl;
    }
    cnt += (int)((__float_as_uint(nh) ^ __float_as_uint(ph)) >> 31);
    qh = ph;
    ql = pl;
    ph = nh;
    pl = nl;
    const float an = fabsf(nh);
    if (an > 0x1p32f || an < 0x1p-32f) {
      const int ex = (int)((__float_as_uint(nh) >> 23) & 0xffu) - 127;
      const float sc = __uint_as_float((unsigned)(127 - ex) << 23);
      ph *= sc;
      pl *= sc;
      qh *= sc;
      ql *= sc;
    }
  }
  return cnt;
}

// Multisection: one warp per wanted eigenvalue (the (r+1)-th largest of the
// slice's scaled T); per step the 32 lanes count at 32 interior points of the
// bracket, so the bracket shrinks 33-fold per step.
//
// abs_tol = 0 (FP64 path): FP64 counts until the bracket is within two units
// in the last place of the eigenvalue.  abs_tol > 0 (FP32 path): BIS_F32_ROUNDS
// rounds of FP32 counts, the bracket widened by BIS_F32_MARGIN on both sides
// (about seven times the FP32 count's backward error bound), then
// double-float counts until the bracket is at most abs_tol wide.  Each round
// moves an end only to a point whose count was taken, at that point's value
// in the precision of the count.
constexpr int BIS_WARPS = 4;
constexpr int BIS_F32_ROUNDS = 4;
constexpr double BIS_F32_MARGIN = 0x1p-18;
__global__ void __launch_bounds__(BIS_WARPS * 32) k_bisect(int m, int R, EigScratch e, double* __restrict__ lam_out,
                                                          double abs_tol) {
  extern __shared__ __align__(16) double bsm[];
  double* d = bsm;                        // [m] scaled diagonal
  double* f2 = bsm + m;                   // [m] scaled squared off-diagonal
  float4* v4 = (float4*)(bsm + 2 * m);    // [m] double-float (d_i, f_{i-1}^2)
  float2* v2 = (float2*)(v4 + m);         // [m] FP32 (d_i, f_{i-1}^2)
  __shared__ double s_scale, s_lo[BIS_WARPS], s_hi[BIS_WARPS];
  const int b = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.x * BIS_WARPS + warp;
  if (threadIdx.x == 0) {
    const double tn = e.tnorm[b];
    s_scale = (tn > 0.0 && isfinite(tn)) ? 1.0 / tn : 1.0;
  }
  __syncthreads();
  const double sc = s_scale;
  const double* ed = e.d + (long)b * m;
  const double* ef = e.f + (long)b * m;
  double glo = DBL_MAX, ghi = -DBL_MAX;  // Gershgorin bracket of the scaled T
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double di = ed[i] * sc;
    const double fr = (i < m - 1) ? ef[i] * sc : 0.0;
    const double fl = (i > 0) ? ef[i - 1] * sc : 0.0;
    d[i] = di;
    f2[i] = fr * fr;
    const double fl2 = fl * fl;
    const dfl dh = df_from(di), fh = df_from(fl2);
    v4[i] = make_float4(dh.hi, dh.lo, fh.hi, fh.lo);
    v2[i] = make_float2((float)di, (float)fl2);
    glo = fmin(glo, di - fabs(fl) - fabs(fr));
    ghi = fmax(ghi, di + fabs(fl) + fabs(fr));
  }
  for (int o = 16; o > 0; o >>= 1) {
    glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, o));
    ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
  }
  if (lane == 0) {
    s_lo[warp] = glo;
    s_hi[warp] = ghi;
  }
  __syncthreads();
  if (r >= R) return;
  if (!(e.tnorm[b] > 0.0)) {  // T = 0 (zero data): every eigenvalue is 0
    if (lane == 0) lam_out[(long)b * R + r] = 0.0;
    return;
  }
  double g_lo = s_lo[0], g_hi = s_hi[0];
  for (int w = 1; w < BIS_WARPS; ++w) {
    g_lo = fmin(g_lo, s_lo[w]);
    g_hi = fmax(g_hi, s_hi[w]);
  }
  const double tn = fmax(fabs(g_lo), fabs(g_hi));
  const double pivmin = DBL_MIN * 0x1p+64;
  double lo = g_lo - (4.0 * DBL_EPSILON * tn + pivmin);
  double hi = g_hi + (4.0 * DBL_EPSILON * tn + pivmin);
  const int idx = m - 1 - r;  // ascending index of the wanted eigenvalue
  if (abs_tol > 0.0) {
    for (int it = 0; it < BIS_F32_ROUNDS; ++it) {
      const double w = hi - lo;
      const float x = (float)(lo + w * ((double)(lane + 1) / 33.0));
      const unsigned above = __ballot_sync(0xffffffffu, sturm_count_f32(v2, m, x) > idx);
      const int first = above ? __ffs(above) - 1 : 32;
      const double nlo = (first == 0) ? lo : (double)(float)(lo + w * ((double)first / 33.0));
      const double nhi = (first == 32) ? hi : (double)(float)(lo + w * ((double)(first + 1) / 33.0));
      lo = nlo;
      hi = nhi;
    }
    lo = fmax(lo - BIS_F32_MARGIN * tn, g_lo - (4.0 * DBL_EPSILON * tn + pivmin));
    hi = fmin(hi + BIS_F32_MARGIN * tn, g_hi + (4.0 * DBL_EPSILON * tn + pivmin));
    for (int it = 0; it < 16; ++it) {
      const double w = hi - lo;
      if (w <= abs_tol) break;
      const dfl x = df_from(lo + w * ((double)(lane + 1) / 33.0));
      const unsigned above = __ballot_sync(0xffffffffu, sturm_count_df(v4, m, x) > idx);
      const int first = above ? __ffs(above) - 1 : 32;
      const double nlo = (first == 0) ? lo : df_to(df_from(lo + w * ((double)first / 33.0)));
      const double nhi = (first == 32) ? hi : df_to(df_from(lo + w * ((double)(first + 1) / 33.0)));
      if (nlo == lo && nhi == hi) break;
      lo = nlo;
      hi = nhi;
    }
  } else {
    for (int it = 0; it < 64; ++it) {
      const double w = hi - lo;
      // relative to the eigenvalue
      if (w <= 2.0 * DBL_EPSILON * (fabs(lo) + fabs(hi)) + pivmin) break;
      const double x = lo + w * ((double)(lane + 1) / 33.0);
      const unsigned above = __ballot_sync(0xffffffffu, sturm_count(d, f2, m, x, pivmin) > idx);
      const int first = above ? __ffs(above) - 1 : 32;  // lowest point with more than idx values below it
      const double nlo = (first == 0) ? lo : lo + w * ((double)first / 33.0);
      const double nhi = (first == 32) ? hi : lo + w * ((double)(first + 1) / 33.0);
      if (nlo == lo && nhi == hi) break;
      lo = nlo;
      hi = nhi;
    }
  }
  if (lane == 0) lam_out[(long)b * R + r] = 0.5 * (lo + hi) / sc;
}

// One thread per wanted eigenpair r (the (r+1)-th largest), TP_THREADS pairs
// per CTA: inverse iteration (three solves, two on the FP32 path) with a partially pivoted LU of
// T - lam I for the eigenvalue found by k_bisect.  The LU factors stream
// from global memory (coalesced across the CTA's threads); the iterate lives
// in shared memory, so the dependent chain of each solve never waits on L2.
constexpr int TP_THREADS = 32;

__global__ void __launch_bounds__(TP_THREADS) k_tridiag_pairs(int m, int R, EigScratch e,
                                                              const double* __restrict__ lam_out, int iters) {
  extern __shared__ __align__(16) double tsm[];
  double* d = tsm;      // [m] scaled diagonal
  double* f = tsm + m;  // [m] scaled off-diagonal
  double* f2 = f + m;   // [m] squares
  double* xs = f2 + m;  // [m][TP_THREADS] iterates
  __shared__ double s_scale;
  const int b = blockIdx.y, t = threadIdx.x, r = blockIdx.x * TP_THREADS + t;
  if (t == 0) {
    const double tn = e.tnorm[b];
    s_scale = (tn > 0.0 && isfinite(tn)) ? 1.0 / tn : 1.0;
  }
  __syncthreads();
  const double sc = s_scale;
  for (int i = t; i < m; i += blockDim.x) {
    d[i] = e.d[(long)b * m + i] * sc;
    const double fi = (i < m - 1) ? e.f[(long)b * m + i] * sc : 0.0;
    f[i] = fi;
    f2[i] = fi * fi;
  }
  __syncthreads();
  if (r >= R) return;
  double* Z = e.Z + ((long)b * R + r) * m;  // vector r, contiguous
  if (!(e.tnorm[b] > 0.0)) {  // T = 0 (zero data): vectors e_r
    for (int i = 0; i < m; ++i) Z[i] = (i == r) ? 1.0 : 0.0;
    return;
  }
  double tn = 0;
  for (int i = 0; i < m; ++i) tn = fmax(tn, fabs(d[i]) + ((i > 0) ? f[i - 1] : 0.0) + f[i]);
  const double lam = lam_out[(long)b * R + r] * sc;

  // factor element i of array a at lu[((b*5 + a)*m + i)*R + r] (coalesced over r)
  // a: 0 multiplier, 1 reciprocal U diagonal, 2 U first super, 3 U second super, 4 row swap (0 / 1)
  double* base = e.lu + (long)b * 5 * m * R + r;
#define LU(a, i) base[((long)(a) * m + (i)) * R]
  double* x = xs + t;
#define X(i) x[(long)(i) * TP_THREADS]
  const double tiny = DBL_EPSILON * fmax(tn, 1e-200);
  double dcur = d[0] - lam, ucur = f[0];
  for (int i = 0; i < m - 1; ++i) {
    const double sub = f[i];
    const double dn = d[i + 1] - lam, un = (i < m - 2) ? f[i + 1] : 0.0;
    if (fabs(dcur) >= fabs(sub)) {
      const double piv = (fabs(dcur) < tiny) ? copysign(tiny, dcur) : dcur;
      const double rp = 1.0 / piv;  // one division per step
      const double l = sub * rp;
      LU(0, i) = l;
      LU(1, i) = rp;
      LU(2, i) = ucur;
      LU(3, i) = 0.0;
      LU(4, i) = 0.0;
      dcur = dn - l * ucur;
      ucur = un;
    } else {
      // swap rows i and i+1: the new row i is (sub, dn, un); the old row i is eliminated
      const double sb = (fabs(sub) < tiny) ? copysign(tiny, sub) : sub;
      const double rs = 1.0 / sb;
      const double l = dcur * rs;
      LU(0, i) = l;
      LU(1, i) = rs;
      LU(2, i) = dn;
      LU(3, i) = un;
      LU(4, i) = 1.0;
      const double nd = ucur - l * dn;
      ucur = -l * un;
      dcur = nd;
    }
  }
  LU(1, m - 1) = 1.0 / ((fabs(dcur) < tiny) ? copysign(tiny, dcur) : dcur);
  LU(2, m - 1) = 0.0;
  LU(3, m - 1) = 0.0;
  for (int i = 0; i < m; ++i) {  // starting vector: Philox uniforms in (-1, 1)
    const uint4 w = philox10(make_uint4((uint32_t)i, (uint32_t)r, (uint32_t)b, 0x1e16u), 0x2504u, 0x4989u);
    X(i) = ((double)w.x + 0.5) * (2.0 / 4294967296.0) - 1.0;
  }
  for (int iter = 0; iter < iters; ++iter) {
    double xi = X(0);
    for (int i = 0; i < m - 1; ++i) {  // row interchanges and multipliers: L^{-1} P
      double xn = X(i + 1);
      if (LU(4, i) != 0.0) {
        const double tmp = xi;
        xi = xn;
        xn = tmp;
      }
      X(i) = xi;
      xi = xn - LU(0, i) * xi;
    }
    X(m - 1) = xi;
    double mx = 0, x1 = 0, x2 = 0;
    for (int i = m - 1; i >= 0; --i) {  // back substitution with U
      const double s = (X(i) - LU(2, i) * x1 - LU(3, i) * x2) * LU(1, i);
      X(i) = s;
      x2 = x1;
      x1 = s;
      mx = fmax(mx, fabs(s));
    }
    if (!(mx > 0) || !isfinite(mx)) mx = 1.0;
    const double imx = 1.0 / mx;
    double nrm2 = 0;
    for (int i = 0; i < m; ++i) {
      const double v = X(i) * imx;
      X(i) = v;
      nrm2 += v * v;
    }
    const double inv = 1.0 / sqrt(nrm2);
    for (int i = 0; i < m; ++i) X(i) *= inv;
  }
  for (int i = 0; i < m; ++i) Z[i] = X(i);
#undef X
#undef LU
}

// Reciprocal: correctly rounded FP32 reciprocal, then one Newton correction
// with the residual 1 - b r formed exactly (FMA) plus the low part's term.
__device__ __forceinline__ dfl df_rcp(dfl b) {
  const float r = __frcp_rn(b.hi);
  const float p = b.hi * r, pe = fmaf(b.hi, r, -p);
  const float res = ((1.0f - p) - pe) - b.lo * r;
  return df_fast_two_sum(r, r * res);
}

// The inverse iteration of k_tridiag_pairs in double-float arithmetic (FP32
// path): the LU of T - lam I, the solves and the normalisation carry hi + lo
// pairs (about 48 significant bits, far below the FP32 accuracy this path
// returns) on the FP32 pipe, so each step's dependent chain is a few FP32
// operations rather than FP64 ones at 1/64 of the rate.  Pivots below 2^-47
// ||T|| are raised to that size.  Factors per step (coalesced over r):
// multiplier, reciprocal pivot and the two U super-diagonals as (hi, lo)
// pairs, the row swaps as bits of one word per 32 steps.  NTH pairs per CTA;
// SMF: the factors of all NTH pairs stay in shared memory (16 pairs at
// m = 300: 197 KB), so the solves never wait on L2; otherwise they live in
// global memory and the solves fetch them TP_CHUNK steps at a time, ahead of
// the dependent chain.
constexpr int TP_CHUNK = 8;
template <bool SMF>
__device__ __forceinline__ float2 tp_ld(const float2* p) {
  if constexpr (SMF) return *p;
  else return __ldcg(p);
}
template <bool SMF>
__device__ __forceinline__ unsigned tp_ld(const unsigned* p) {
  if constexpr (SMF) return *p;
  else return __ldcg(p);
}
static size_t tp_df_smem(int m, int nth, bool smf) {
  size_t bytes = (size_t)m * (sizeof(float4) + nth * sizeof(float2));
  if (smf) bytes += (size_t)m * nth * 4 * sizeof(float2) + (size_t)cdiv(m, 32) * nth * sizeof(unsigned);
  return bytes;
}
template <int NTH, bool SMF>
__global__ void __launch_bounds__(NTH) k_tridiag_pairs_df(int m, int R, EigScratch e,
                                                          const double* __restrict__ lam_out, int iters) {
  extern __shared__ __align__(16) double tsm[];
  float4* T4 = (float4*)tsm;         // [m] (d_i hi, lo, f_i hi, lo), f_{m-1} = 0
  float2* xs = (float2*)(T4 + m);    // [m][NTH] iterates
  __shared__ double s_scale;
  const int b = blockIdx.y, t = threadIdx.x, r = blockIdx.x * NTH + t;
  if (t == 0) {
    const double tn = e.tnorm[b];
    s_scale = (tn > 0.0 && isfinite(tn)) ? 1.0 / tn : 1.0;
  }
  __syncthreads();
  const double sc = s_scale;
  for (int i = t; i < m; i += blockDim.x) {
    const dfl dd = df_from(e.d[(long)b * m + i] * sc);
    const dfl ff = df_from((i < m - 1) ? e.f[(long)b * m + i] * sc : 0.0);
    T4[i] = make_float4(dd.hi, dd.lo, ff.hi, ff.lo);
  }
  __syncthreads();
  if (r >= R) return;
  double* Z = e.Z + ((long)b * R + r) * m;  // vector r, contiguous
  if (!(e.tnorm[b] > 0.0)) {  // T = 0 (zero data): vectors e_r
    for (int i = 0; i < m; ++i) Z[i] = (i == r) ? 1.0 : 0.0;
    return;
  }
  const dfl nlam = df_neg(df_from(lam_out[(long)b * R + r] * sc));
  // factor arrays, element i of this pair at [i * ls + lo]: shared memory [m][NTH] (SMF), else
  // this slice's part of e.lu, [m][R]
  const long ls = SMF ? NTH : R;
  float2* L0 = SMF ? (float2*)(xs + (long)m * NTH) : (float2*)(e.lu + (long)b * 5 * m * R);  // multiplier
  float2* L1 = L0 + (long)m * ls;                      // reciprocal pivot
  float2* L2 = L1 + (long)m * ls;                      // U first super-diagonal
  float2* L3 = L2 + (long)m * ls;                      // U second super-diagonal
  unsigned* FL = (unsigned*)(L3 + (long)m * ls);       // row swaps, [cdiv(m, 32)][ls]
  L0 += SMF ? t : r;
  L1 += SMF ? t : r;
  L2 += SMF ? t : r;
  L3 += SMF ? t : r;
  FL += SMF ? t : r;
  float2* x = xs + t;
#define X(i) x[(long)(i) * NTH]
  const float tiny = 0x1p-47f;
  dfl dcur = df_add(dfl{T4[0].x, T4[0].y}, nlam), ucur = dfl{T4[0].z, T4[0].w};
  unsigned flags = 0;
  for (int i = 0; i < m - 1; ++i) {
    const float4 c0 = T4[i], c1 = T4[i + 1];
    const dfl sub = dfl{c0.z, c0.w};
    const dfl dn = df_add(dfl{c1.x, c1.y}, nlam), un = dfl{c1.z, c1.w};
    // partial pivoting without a branch (lanes would diverge on the swaps): with a swap the new
    // row i is (sub, dn, un) and the old one is eliminated; both cases are one reciprocal, one
    // multiply and one multiply-add on selected operands
    const bool sw = !(fabsf(dcur.hi) >= fabsf(sub.hi));
    const dfl pv = sw ? sub : dcur, nm = sw ? dcur : sub;
    const dfl rp = df_rcp((fabsf(pv.hi) < tiny) ? dfl{copysignf(tiny, pv.hi), 0.0f} : pv);
    const dfl l = df_mul(nm, rp);
    const dfl u1 = sw ? dn : ucur, u2 = sw ? un : dfl{0.0f, 0.0f};
    const dfl ua = sw ? ucur : dn, ub = sw ? dn : ucur;
    const dfl lu = df_mul(df_neg(l), un);
    dcur = df_fma(ua, df_neg(l), ub);  // dn - l ucur, or ucur - l dn after a swap
    ucur = sw ? lu : un;
    flags |= (sw ? 1u : 0u) << (i & 31);
    const long o = (long)i * ls;
    L0[o] = make_float2(l.hi, l.lo);
    L1[o] = make_float2(rp.hi, rp.lo);
    L2[o] = make_float2(u1.hi, u1.lo);
    L3[o] = make_float2(u2.hi, u2.lo);
    if ((i & 31) == 31 || i == m - 2) {
      FL[(long)(i >> 5) * ls] = flags;
      flags = 0;
    }
  }
  {
    const dfl rp = df_rcp((fabsf(dcur.hi) < tiny) ? dfl{copysignf(tiny, dcur.hi), 0.0f} : dcur);
    const long o = (long)(m - 1) * ls;
    L1[o] = make_float2(rp.hi, rp.lo);
    L2[o] = make_float2(0.0f, 0.0f);
    L3[o] = make_float2(0.0f, 0.0f);
  }
  for (int i = 0; i < m; ++i) {  // starting vector: Philox uniforms in (-1, 1)
    const uint4 w = philox10(make_uint4((uint32_t)i, (uint32_t)r, (uint32_t)b, 0x1e16u), 0x2504u, 0x4989u);
    const dfl v = df_from(((double)w.x + 0.5) * (2.0 / 4294967296.0) - 1.0);
    X(i) = make_float2(v.hi, v.lo);
  }
  for (int iter = 0; iter < iters; ++iter) {
    // row interchanges and multipliers: L^{-1} P
    dfl xi = dfl{X(0).x, X(0).y};
    unsigned fw = 0;
    for (int i0 = 0; i0 < m - 1; i0 += TP_CHUNK) {
      float2 lc[TP_CHUNK];
#pragma unroll
      for (int k = 0; k < TP_CHUNK; ++k)
        lc[k] = (i0 + k < m - 1) ? tp_ld<SMF>(L0 + (long)(i0 + k) * ls) : make_float2(0.0f, 0.0f);
      if ((i0 & 31) == 0) fw = tp_ld<SMF>(FL + (long)(i0 >> 5) * ls);
#pragma unroll
      for (int k = 0; k < TP_CHUNK; ++k) {
        const int i = i0 + k;
        if (i < m - 1) {
          const float2 xv = X(i + 1);
          dfl xn = dfl{xv.x, xv.y};
          if ((fw >> (i & 31)) & 1u) {
            const dfl tmp = xi;
            xi = xn;
            xn = tmp;
          }
          X(i) = make_float2(xi.hi, xi.lo);
          xi = df_fma(xn, dfl{-lc[k].x, -lc[k].y}, xi);
        }
      }
    }
    X(m - 1) = make_float2(xi.hi, xi.lo);
    // back substitution with U
    dfl x1 = dfl{0.0f, 0.0f}, x2 = dfl{0.0f, 0.0f};
    float mx = 0.0f;
    for (int i0 = m - 1; i0 >= 0; i0 -= TP_CHUNK) {
      float2 pc[TP_CHUNK], ac[TP_CHUNK], bc[TP_CHUNK];
#pragma unroll
      for (int k = 0; k < TP_CHUNK; ++k) {
        const int i = i0 - k;
        const bool ok = i >= 0;
        const long o = (long)(ok ? i : 0) * ls;
        pc[k] = ok ? tp_ld<SMF>(L1 + o) : make_float2(0.0f, 0.0f);
        ac[k] = ok ? tp_ld<SMF>(L2 + o) : make_float2(0.0f, 0.0f);
        bc[k] = ok ? tp_ld<SMF>(L3 + o) : make_float2(0.0f, 0.0f);
      }
#pragma unroll
      for (int k = 0; k < TP_CHUNK; ++k) {
        const int i = i0 - k;
        if (i >= 0) {
          const float2 xv = X(i);
          dfl s = df_fma(dfl{xv.x, xv.y}, dfl{-ac[k].x, -ac[k].y}, x1);
          s = df_fma(s, dfl{-bc[k].x, -bc[k].y}, x2);
          s = df_mul(s, dfl{pc[k].x, pc[k].y});
          X(i) = make_float2(s.hi, s.lo);
          x2 = x1;
          x1 = s;
          mx = fmaxf(mx, fabsf(s.hi));
        }
      }
    }
    // rescale by a power of two (exact) so that the largest component is in [1, 2)
    if (mx > 0.0f && mx <= FLT_MAX) {
      const int ex = (int)((__float_as_uint(mx) >> 23) & 0xffu) - 127;
      const float s2 = ldexpf(1.0f, -ex);
      for (int i = 0; i < m; ++i) {
        const float2 v = X(i);
        X(i) = make_float2(v.x * s2, v.y * s2);
      }
    }
  }
  dfl nrm2 = dfl{0.0f, 0.0f};
  for (int i = 0; i < m; ++i) {
    const dfl v = dfl{X(i).x, X(i).y};
    nrm2 = df_fma(nrm2, v, v);
  }
  const dfl inv = df_rcp(df_sqrt(nrm2));
  for (int i = 0; i < m; ++i) Z[i] = df_to(df_mul(dfl{X(i).x, X(i).y}, inv));
#undef X
}

// Inside clusters of close eigenvalues (gap < 1e-3 ||T||) the vectors are
// made orthonormal.  On the FP32 path (CT = float) a cluster of at most
// CO_BLOCK vectors is orthonormalised as a block by CholeskyQR2: G = Z_c^T Z_c,
// G = R^T R (CTA-wide right-looking factorisation, one barrier per column),
// Z_c <- Z_c R^{-1}, twice -- the basis Gram-Schmidt in eigenvalue order gives,
// in exact arithmetic.  The inverse-iteration vectors of a cluster are close
// to orthonormal already; a pivot below 1e-5 (condition number above about
// 300, beyond what two FP32 passes restore) sends the cluster to two classical
// Gram-Schmidt passes per vector against its earlier members, then
// normalisation, which also serves larger clusters and the FP64 path.
// CT: storage and arithmetic (FP32 on the FP32 path, whose vectors are
// rounded to FP32 right after; FP64 otherwise).  The slice's R vectors are
// staged in shared memory for the whole kernel when they fit.
constexpr int CO_THREADS = 1024;
constexpr int CO_BLOCK = 64;
template <typename CT, bool STAGED>  // !STAGED (vectors too large for shared memory): CT = double, in place in Z
__global__ void __launch_bounds__(CO_THREADS) k_cluster_orth(int m, int R, EigScratch e, const double* __restrict__ lam) {
  extern __shared__ __align__(16) unsigned char cosm[];
  __shared__ double red[32];
  __shared__ CT dots[128];
  constexpr bool kBlock = std::is_same<CT, float>::value;
  __shared__ float Gs[kBlock ? CO_BLOCK * CO_BLOCK : 1];  // Gram, then R (upper, row-major)
  __shared__ float Rd[kBlock ? CO_BLOCK : 1];             // 1 / R_jj
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  double* Z = e.Z + (long)b * R * m;  // vector r at Z + r*m
  const double* l = lam + (long)b * R;
  const double tol = 1e-3 * e.tnorm[b];
  // only vectors inside a cluster change; find whether there is any
  bool any = false;
  for (int r = 1; r < R; ++r) any |= !(l[r - 1] - l[r] > tol);
  if (!any) return;
  CT* zsm = STAGED ? (CT*)cosm : (CT*)Z;  // [R][m]
  if (STAGED) {
    for (int q = tid; q < R * m; q += blockDim.x) zsm[q] = (CT)Z[q];
    __syncthreads();
  }
  // CholeskyQR2 of vectors [c0, c0 + nc) (FP32); false on a small pivot (vectors as after the
  // last completed pass)
  auto block_qr = [&](int c0, int nc) -> bool {
    float* zc = (float*)zsm + (long)c0 * m;
    for (int pass = 0; pass < 2; ++pass) {
      for (int a = 0; a < nc; ++a)
        for (int bb = a + warp; bb < nc; bb += nwarp) {
          float acc = 0.f;
          for (int i = lane; i < m; i += 32) acc = fmaf(zc[(long)a * m + i], zc[(long)bb * m + i], acc);
          acc = warp_sum(acc);
          if (lane == 0) Gs[a * CO_BLOCK + bb] = acc;
        }
      __syncthreads();
      // G(a, k) -= G(j, a) G(j, k) / d_j for j < a <= k; row j scaled by 1/sqrt(d_j) afterwards
      for (int j = 0; j < nc; ++j) {
        const float d = Gs[j * CO_BLOCK + j];
        if (!(d > 1e-5f)) return false;  // uniform: every thread reads the same pivot
        const float id = 1.0f / d;
        const int k = j + 1 + (tid & 63);
        for (int a = j + 1 + (tid >> 6); a <= k && k < nc; a += CO_THREADS / 64)
          Gs[a * CO_BLOCK + k] -= Gs[j * CO_BLOCK + a] * Gs[j * CO_BLOCK + k] * id;
        __syncthreads();
      }
      if (tid < nc) Rd[tid] = 1.0f / sqrtf(Gs[tid * CO_BLOCK + tid]);
      __syncthreads();
      for (int i = tid; i < m; i += blockDim.x) {  // row i of Z_c: x R = z by forward substitution, in place
        for (int bb = 0; bb < nc; ++bb) {
          float acc = zc[(long)bb * m + i];
          for (int a = 0; a < bb; ++a) acc = fmaf(-zc[(long)a * m + i], Gs[a * CO_BLOCK + bb] * Rd[a], acc);
          zc[(long)bb * m + i] = acc * Rd[bb];
        }
      }
      __syncthreads();
    }
    return true;
  };
  auto cgs2 = [&](int c0, int c1) {
    for (int r = c0 + 1; r < c1; ++r) {
      CT* zr = zsm + (long)r * m;
      for (int pass = 0; pass < 2; ++pass) {
        for (int s2 = c0 + warp; s2 < r; s2 += nwarp) {
          const CT* zs = zsm + (long)s2 * m;
          CT acc = 0;
          for (int i = lane; i < m; i += 32) acc += zs[i] * zr[i];
          acc = warp_sum(acc);
          if (lane == 0) dots[s2 - c0] = acc;
        }
        __syncthreads();
        for (int i = tid; i < m; i += blockDim.x) {
          CT acc = zr[i];
          for (int s2 = c0; s2 < r; ++s2) acc -= dots[s2 - c0] * zsm[(long)s2 * m + i];
          zr[i] = acc;
        }
        __syncthreads();
      }
      double part = 0;
      for (int i = tid; i < m; i += blockDim.x) part += (double)zr[i] * (double)zr[i];
      const CT inv = (CT)(1.0 / sqrt(block_sum(part, red)));
      for (int i = tid; i < m; i += blockDim.x) zr[i] *= inv;
      __syncthreads();
    }
  };
  int c0 = 0;
  for (int r = 1; r <= R; ++r) {
    if (r < R && !(l[r - 1] - l[r] > tol)) continue;  // r extends the cluster starting at c0
    const int nc = r - c0;
    bool done = nc < 2;
    if constexpr (kBlock) done = done || (nc <= CO_BLOCK && block_qr(c0, nc));
    if (!done) cgs2(c0, r);
    c0 = r;
  }
  if (STAGED)
    for (int q = tid; q < R * m; q += blockDim.x) Z[q] = (double)zsm[q];
}

// u_r = H_0 H_1 .. H_{m-2} D z_r in the precision of the output (the FP32
// path rounds U_c to FP32 for its GEMMs anyway): BT_VPC eigenvectors per CTA,
// one warp each, the vector in the warp's registers (entry i in lane i % 32,
// slot i / 32).  The reflectors (VT: float2 copies from the double-float
// reduction, else double2) are staged in shared memory by asynchronous copies
// one reflector ahead, three buffers deep (one barrier per reflector), and
// read by all the CTA's warps; slots wholly at or above row j are skipped.
constexpr int BT_VPC = 16;
__device__ __forceinline__ void bt_copy(float2* dst, const float2* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src));
}
__device__ __forceinline__ void bt_copy(double2* dst, const double2* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src));
}
template <typename C, typename VT, int NPL>  // NPL >= ceil(m / 32)
__global__ void __launch_bounds__(BT_VPC * 32) k_backtransform(int m, int R, EigScratch e, C* __restrict__ U,
                                                               long ldu, long sU) {
  using Rt = decltype(C().x);
  extern __shared__ __align__(16) unsigned char bts[];
  VT* vb = (VT*)bts;  // [3][m]
  const int b = blockIdx.y, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = blockIdx.x * BT_VPC + warp;
  const bool active = r < R;
  const VT* Hs = (const VT*)e.Hv + (long)b * m * m;  // reflector j at Hs + j m + j + 1
  C u[NPL];
#pragma unroll
  for (int t = 0; t < NPL; ++t) {
    const int i = lane + 32 * t;
    u[t] = C{Rt(0), Rt(0)};
    if (active && i < m) u[t] = from_c64<C>(cscale(e.delta[(long)b * m + i], e.Z[((long)b * R + r) * m + i]));
  }
  auto stage = [&](int j) {
    const VT* src = Hs + (long)j * m + j + 1;
    VT* dst = vb + (j % 3) * m + j + 1;
    for (int i = tid; i < m - j - 1; i += blockDim.x) bt_copy(dst + i, src + i);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  if (m >= 2) stage(m - 2);
  for (int j = m - 2; j >= 0; --j) {
    if (j > 0) {
      stage(j - 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();  // reflector j visible; the buffer staged next was last read two reflectors ago
    if (active) {
      const VT* v = vb + (j % 3) * m;
      Rt ax = Rt(0), ay = Rt(0);
#pragma unroll
      for (int t = 0; t < NPL; ++t) {
        if (32 * t + 31 > j) {
          const int i = lane + 32 * t;
          if (i > j && i < m) {
            const VT vv = v[i];
            const Rt vx = (Rt)vv.x, vy = (Rt)vv.y;
            ax = fma(vx, u[t].x, ax);  // conj(v_i) u_i
            ax = fma(vy, u[t].y, ax);
            ay = fma(vx, u[t].y, ay);
            ay = fma(-vy, u[t].x, ay);
          }
        }
      }
      ax = Rt(2) * warp_sum(ax);
      ay = Rt(2) * warp_sum(ay);
#pragma unroll
      for (int t = 0; t < NPL; ++t) {
        if (32 * t + 31 > j) {
          const int i = lane + 32 * t;
          if (i > j && i < m) {
            const VT vv = v[i];
            const Rt vx = (Rt)vv.x, vy = (Rt)vv.y;
            u[t].x -= vx * ax - vy * ay;
            u[t].y -= vx * ay + vy * ax;
          }
        }
      }
    }
  }
  if (!active) return;
  C* Ub = U + (long)b * sU;
#pragma unroll
  for (int t = 0; t < NPL; ++t) {
    const int i = lane + 32 * t;
    if (i < m) Ub[(long)i * ldu + r] = u[t];
  }
}

template <typename C, typename VT>
static int launch_backtransform(int m, int R, int batch, const EigScratch& e, C* U, long ldu, long sU,
                                cudaStream_t s) {
  const size_t smem = 3 * (size_t)m * sizeof(VT);
  const dim3 grid(cdiv(R, BT_VPC), batch);
  auto go = [&](auto kern) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return TSVD_ERR_CUDA;
    }
    kern<<<grid, BT_VPC * 32, smem, s>>>(m, R, e, U, ldu, sU);
    TSVD_LAUNCHED();
    return TSVD_OK;
  };
  const int npl = cdiv(m, 32);
  if (npl <= 4) return go(k_backtransform<C, VT, 4>);
  if (npl <= 8) return go(k_backtransform<C, VT, 8>);
  if (npl <= 12) return go(k_backtransform<C, VT, 12>);
  if (npl <= 16) return go(k_backtransform<C, VT, 16>);
  if (npl <= 24) return go(k_backtransform<C, VT, 24>);
  return TSVD_ERR_UNSUPPORTED;
}

static int device_attr(cudaDeviceAttr a, int fallback) {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, a, dev) != cudaSuccess || v <= 0) {
    cudaGetLastError();
    return fallback;
  }
  return v;
}

// Cluster size of the shared-memory tridiagonalisation, or 0 when the slice's
// rows do not fit: the largest CL in {8,4,2,1} with batch * CL CTAs resident
// at once (one per SM), at least 48 rows per CTA (else the per-step barriers
// dominate) and the packed rows within the opt-in shared memory.
static int hetrd_smem_cluster(int m, int batch, int nt, bool global_rows = false) {
  if (m < 2) return 0;
  const int sms = device_attr(cudaDevAttrMultiProcessorCount, 148);
  // the kernels' static arrays (up to about 1.3 KB) share the per-block limit with the dynamic part
  const size_t smax = (size_t)device_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin, 232448) - 2048;
  for (int CL = 8; CL >= 1; CL >>= 1) {
    if (CL > 1 && ((long)batch * CL > sms || m / CL < 48)) continue;
    if (hetrd_smem_bytes(m, CL, nt, global_rows) <= smax) return CL;
  }
  return 0;
}

// the packed rows do not fit in shared memory for the double-float reduction
// (the larger of the two): they go to a global array (EigScratch::Sg)
static bool hetrd_needs_global_rows(int m, int batch) {
  return m >= 2 && hetrd_smem_cluster(m, batch, 2 * HS_THREADS) == 0;
}

template <int CL, bool DF, bool GS>
static int launch_hetrd_smem_t(const double2* G, long ldg, long sG, int m, int batch, const EigScratch& e,
                               cudaStream_t s, int b0 = 0) {
  constexpr int NT = DF ? 2 * HS_THREADS : HS_THREADS;
  const size_t smem = hetrd_smem_bytes(m, CL, NT, GS);
  auto kern = DF ? k_hetrd_df<CL, NT, GS> : k_hetrd_smem<CL, GS>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return TSVD_ERR_CUDA;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(batch * CL);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, kern, G, ldg, sG, m, (int)hetrd_smem_elems(m, CL), e, b0) != cudaSuccess) {
    cudaGetLastError();
    return TSVD_ERR_CUDA;
  }
  TSVD_LAUNCHED();
  return TSVD_OK;
}

template <bool DF, bool GS>
static int launch_hetrd_smem(int CL, const double2* G, long ldg, long sG, int m, int batch, const EigScratch& e,
                             cudaStream_t s, int b0 = 0) {
  switch (CL) {
    case 8: return launch_hetrd_smem_t<8, DF, GS>(G, ldg, sG, m, batch, e, s, b0);
    case 4: return launch_hetrd_smem_t<4, DF, GS>(G, ldg, sG, m, batch, e, s, b0);
    case 2: return launch_hetrd_smem_t<2, DF, GS>(G, ldg, sG, m, batch, e, s, b0);
    default: return launch_hetrd_smem_t<1, DF, GS>(G, ldg, sG, m, batch, e, s, b0);
  }
}

// the one-pass reduction with rows in L2 (k_hetrd_df1): same cluster sizes as the
// sweep kernels; 0 when its per-warp partials of p do not fit in shared memory
constexpr int HF_THREADS = 2 * HS_THREADS;
static int hetrd_df1_cluster(int m, int batch) {
  if (m < 2) return 0;
  const size_t smax = (size_t)device_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin, 232448) - 2048;
  if (hetrd_df1_smem_bytes(m, HF_THREADS) > smax) return 0;
  const int sms = device_attr(cudaDevAttrMultiProcessorCount, 148);
  for (int CL = 8; CL >= 2; CL >>= 1)
    if ((long)batch * CL <= sms && m / CL >= 48) return CL;
  return 1;
}

template <int CL>
static int launch_hetrd_df1_t(const double2* G, long ldg, long sG, int m, int batch, const EigScratch& e,
                              cudaStream_t s) {
  const size_t smax = (size_t)device_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin, 232448) - 2048;
  const int use_sched = hetrd_df1_smem_bytes(m, HF_THREADS, CL, true) <= smax ? 1 : 0;
  const size_t smem = hetrd_df1_smem_bytes(m, HF_THREADS, CL, use_sched != 0);
  auto kern = k_hetrd_df1<CL, HF_THREADS>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return TSVD_ERR_CUDA;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(batch * CL);
  cfg.blockDim = dim3(HF_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, kern, G, ldg, sG, m, (int)hetrd_smem_elems(m, CL), e, use_sched) != cudaSuccess) {
    cudaGetLastError();
    return TSVD_ERR_CUDA;
  }
  TSVD_LAUNCHED();
  return TSVD_OK;
}

static int launch_hetrd_df1(int CL, const double2* G, long ldg, long sG, int m, int batch, const EigScratch& e,
                            cudaStream_t s) {
  switch (CL) {
    case 8: return launch_hetrd_df1_t<8>(G, ldg, sG, m, batch, e, s);
    case 4: return launch_hetrd_df1_t<4>(G, ldg, sG, m, batch, e, s);
    case 2: return launch_hetrd_df1_t<2>(G, ldg, sG, m, batch, e, s);
    default: return launch_hetrd_df1_t<1>(G, ldg, sG, m, batch, e, s);
  }
}

template <typename C>
int herm_eig_topR(double2* G, long ldg, long sG, int m, int R, int batch, double* lam, C* U, long ldu, long sU,
                  void* scratch, int* status, cudaStream_t s) {
  (void)status;
  if (m <= 0 || R <= 0 || batch <= 0) return TSVD_OK;
  if (R > m || R > 128 || m > 768) return TSVD_ERR_UNSUPPORTED;  // shared memory of k_hetrd
  EigScratch e = carve_eig(scratch, m, R, batch, nullptr);
  // FP32 path (C = float2): double-float reduction (twice the threads); FP64 path: FP64
  constexpr bool kDoubleFloat = std::is_same<C, float2>::value;
  const int NTh = kDoubleFloat ? 2 * HS_THREADS : HS_THREADS;
  const int CLs = hetrd_smem_cluster(m, batch, NTh);
  // rows too large for shared memory: the same double-float cluster reduction on
  // rows kept in L2 (the FP64 path keeps its FP64 L2 kernel below)
  const int CLg = (kDoubleFloat && CLs == 0 && e.Sg) ? hetrd_smem_cluster(m, batch, NTh, true) : 0;
  const int hv32 = (kDoubleFloat && (CLs > 0 || CLg > 0)) ? 1 : 0;  // Householder vectors stored as float2
  if (CLs > 0) {
    TSVD_STAGE("eig_hetrd", s);
    TSVD_TRY((launch_hetrd_smem<kDoubleFloat, false>(CLs, G, ldg, sG, m, batch, e, s)));
  } else if (CLg > 0) {
    // one launch over all slices: measured faster than waves sized to keep each
    // wave's rows in L2 (the pass is bound by its instructions, not by L2 misses)
    TSVD_STAGE("eig_hetrd", s);
    const int CL1 = hetrd_df1_cluster(m, batch);
    if (CL1 > 0) TSVD_TRY(launch_hetrd_df1(CL1, G, ldg, sG, m, batch, e, s));
    else TSVD_TRY((launch_hetrd_smem<kDoubleFloat, true>(CLg, G, ldg, sG, m, batch, e, s)));
  } else {
    TSVD_STAGE("eig_hetrd", s);
    const size_t smem = (2 + 16) * (size_t)m * sizeof(double2);  // v, p and 16 warps' partials
    if (smem > 40 * 1024) {  // with the static reduction arrays
      cudaFuncSetAttribute(k_hetrd<HETRD_CLUSTER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(batch * HETRD_CLUSTER);
    cfg.blockDim = dim3(512);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = HETRD_CLUSTER;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_hetrd<HETRD_CLUSTER>, G, ldg, sG, m, e) != cudaSuccess) {
      cudaGetLastError();
      return TSVD_ERR_CUDA;
    }
    TSVD_LAUNCHED();
  }
  {
    TSVD_STAGE("eig_bisect", s);
    const size_t smem_b = (size_t)m * (2 * sizeof(double) + sizeof(float4) + sizeof(float2));
    // FP32 path: eigenvalues to 3e-13 of ||T|| (the vectors and the outputs are FP32; the
    // smallest kept sigma^2 is far above that); FP64 path: to the eigenvalue's own precision
    const double abs_tol = kDoubleFloat ? 3e-13 : 0.0;
    k_bisect<<<dim3(cdiv(R, BIS_WARPS), batch), BIS_WARPS * 32, smem_b, s>>>(m, R, e, lam, abs_tol);
    TSVD_LAUNCHED();
  }
  {
    TSVD_STAGE("eig_invit", s);
    const size_t smem_tp = (3 + (size_t)TP_THREADS) * m * sizeof(double);
    if (smem_tp > 48 * 1024)
      cudaFuncSetAttribute(k_tridiag_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_tp);
    // solves: 3 (FP64 path), 2 on the FP32 path (eigenvalues to 3e-13 ||T|| already make one solve
    // amplify the wanted direction by gap / 3e-13; the vectors end in FP32)
    if (kDoubleFloat) {
      auto go = [&](auto kern, int nth, bool smf) {
        const size_t smem_df = tp_df_smem(m, nth, smf);
        if (smem_df > 40 * 1024 &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_df) != cudaSuccess) {
          cudaGetLastError();
          return TSVD_ERR_CUDA;
        }
        kern<<<dim3(cdiv(R, nth), batch), nth, smem_df, s>>>(m, R, e, lam, 2);
        return TSVD_OK;
      };
      if (tp_df_smem(m, 16, true) <= 200 * 1024) TSVD_TRY(go(k_tridiag_pairs_df<16, true>, 16, true));
      else TSVD_TRY(go(k_tridiag_pairs_df<TP_THREADS, false>, TP_THREADS, false));
    } else {
      k_tridiag_pairs<<<dim3(cdiv(R, TP_THREADS), batch), TP_THREADS, smem_tp, s>>>(m, R, e, lam, 3);
    }
    TSVD_LAUNCHED();
  }
  {
    TSVD_STAGE("eig_cluster", s);
    size_t smem_co = (size_t)R * m * (kDoubleFloat ? sizeof(float) : sizeof(double));
    using CoKernel = void (*)(int, int, EigScratch, const double*);
    CoKernel co = kDoubleFloat ? (CoKernel)k_cluster_orth<float, true> : (CoKernel)k_cluster_orth<double, true>;
    // the kernel's static arrays (the cluster Gram and its reductions) take about 17 KB of the
    // per-block limit
    const size_t smax_co = (size_t)device_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin, 232448) - 20 * 1024;
    if (smem_co > smax_co) {  // vectors stay in global memory
      co = k_cluster_orth<double, false>;
      smem_co = 0;
    }
    // the kernel's static shared memory (the cluster Gram, 16 KB) counts against the same 48 KB default
    if (smem_co > 0 && cudaFuncSetAttribute(co, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_co) !=
                           cudaSuccess) {
      cudaGetLastError();
      return TSVD_ERR_CUDA;
    }
    co<<<batch, CO_THREADS, smem_co, s>>>(m, R, e, lam);
    TSVD_LAUNCHED();
  }
  TSVD_STAGE("eig_backtransform", s);
  if constexpr (kDoubleFloat) {
    if (hv32) return launch_backtransform<C, float2>(m, R, batch, e, U, ldu, sU, s);
  }
  return launch_backtransform<C, double2>(m, R, batch, e, U, ldu, sU, s);
}
template int herm_eig_topR<double2>(double2*, long, long, int, int, int, double*, double2*, long, long, void*, int*,
                                    cudaStream_t);
template int herm_eig_topR<float2>(double2*, long, long, int, int, int, double*, float2*, long, long, void*, int*,
                                   cudaStream_t);

// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_sigma(const double* __restrict__ lam, int n, double* __restrict__ sig, cx_t<T>* __restrict__ Sh,
                        int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double l = lam[i];
  if (!isfinite(l)) atomicExch(status, TSVD_ERR_NOT_CONVERGED);
  const double sg = sqrt(fmax(l, 0.0));
  if (sig) sig[i] = sg;
  Sh[i] = mkc((T)sg, T(0));
}

template <typename T>
int sigma_from_lambda(const double* lam, int R, int batch, double* sig, cx_t<T>* Sh, cudaStream_t s, int* status) {
  const int n = R * batch;
  if (n <= 0) return TSVD_OK;
  k_sigma<T><<<cdiv(n, 256), 256, 0, s>>>(lam, n, sig, Sh, status);
  TSVD_LAUNCHED();
  return TSVD_OK;
}
template int sigma_from_lambda<double>(const double*, int, int, double*, double2*, cudaStream_t, int*);
template int sigma_from_lambda<float>(const double*, int, int, double*, float2*, cudaStream_t, int*);

template <typename T>
__global__ void k_scale_cols(cx_t<T>* __restrict__ V, long ldv, long sV, int rows, int R,
                             const double* __restrict__ lam, int batch) {
  const long total = (long)batch * rows * R;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int r = idx % R;
    const long t = idx / R;
    const int i = t % rows;
    const int b = t / rows;
    const double sg = sqrt(fmax(lam[(long)b * R + r], 0.0));
    const T inv = (sg > 0.0) ? (T)(1.0 / sg) : T(0);
    cx_t<T>* p = V + (long)b * sV + (long)i * ldv + r;
    *p = cscale(*p, inv);
  }
}

template <typename T>
int scale_columns_inv(cx_t<T>* V, long ldv, long sV, int rows, int R, const double* lam, int batch, cudaStream_t s) {
  const long total = (long)batch * rows * R;
  if (total <= 0) return TSVD_OK;
  k_scale_cols<T><<<std::min<long>(cdiv(total, 256), 8192), 256, 0, s>>>(V, ldv, sV, rows, R, lam, batch);
  TSVD_LAUNCHED();
  return TSVD_OK;
}
template int scale_columns_inv<double>(double2*, long, long, int, int, const double*, int, cudaStream_t);
template int scale_columns_inv<float>(float2*, long, long, int, int, const double*, int, cudaStream_t);

}  // namespace tsvd
