// tc_gemm.cu -- batched real GEMM on the 5th-generation tensor cores:
//   C_b (M x N, FP32) = A_b (M x K) * B_b^T,   B_b stored N x K,
// A and B K-major (K contiguous), TF32 (FP32 storage) or BF16 operands, FP32
// accumulation in tensor memory.
//
// One CTA computes a 128 x BN tile, BN = 128, or (TF32 and BF16) 256 when
// N > 128 (a product with N in (128, 256], as the Krylov products' 2b real
// columns, then reads each row panel of A once).  Operand tiles of 128 (A) and BN (B) rows x 128
// bytes of K are staged by TMA (128-byte swizzle) through a ring of shared
// buffers guarded by mbarriers; one thread issues tcgen05.mma (4 per stage,
// 32 bytes of K each) into a BN-column TMEM accumulator and commits each
// stage back to the producer; all four warps then read the accumulator with
// tcgen05.ld and store it (thread = row, 16 columns at a time as four 16-byte
// accesses where aligned; C = alpha A B^T + beta C, the old values loaded
// before any store).  Every wait is bounded: on a timeout the kernel records
// an error flag instead of hanging.  Options: `upper` skips the tiles wholly
// below the diagonal of a symmetric product (B = A); the split-TF32 epilogue
// can also write hi / lo copies of C and of C^T for a following product.
//
// A third mode keeps FP32 accuracy on the TF32 units ("split TF32"): each
// operand is split as x = hi + lo with hi = x rounded to TF32 and lo = x - hi
// (exact in FP32), and the tile product is hi*hi + hi*lo + lo*hi accumulated
// in the same TMEM tile (about 22 significant bits per product; lo*lo, below
// FP32 rounding, is dropped).  Four operand tiles per stage, three stages.
//
// Complex products use it without moving the big operand: an interleaved
// complex matrix X (rows x cols) is the real matrix [Re Im Re Im ...] of
// rows x 2cols, so X * Y = real(X) * E(Y)^T with a small expanded real form
// E(Y) of the thin factor (see expand_* below).  X^H Y with both factors tall
// takes their de-interleaved columns instead (split_deinterleave): one real
// product of the rows Re x_c, Im x_c against those of Y, combined 2 x 2.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace tsvd {

constexpr int TC_BM = 128;
constexpr int TC_A_BYTES = TC_BM * 128;  // 128 rows x 128 bytes of K
// MODE 0: TF32, 1: BF16, 2: split TF32; BN: 128 or 256 columns per tile
template <int BN>
constexpr int tc_b_bytes() { return BN * 128; }
template <int MODE, int BN>
constexpr int tc_stage_bytes() { return (MODE == 2 ? 2 : 1) * (TC_A_BYTES + tc_b_bytes<BN>()); }  // A, B[, A lo, B lo]
template <int MODE, int BN>
constexpr int tc_stages() { return MODE == 2 ? 3 : 4; }
template <int MODE, int BN>
constexpr int tc_smem() { return tc_stages<MODE, BN>() * tc_stage_bytes<MODE, BN>() + 1024 + 256; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// hi = x rounded to the nearest TF32 (lo = x - hi is exact in FP32)
__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// true once the phase of the given parity has completed; false after ~1 s
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (2LL << 30)) return false;
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(dst),
      "l"((unsigned long long)tm), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// shared-memory matrix descriptor: K-major operand tile, 128-byte swizzle,
// 8-row groups 1024 bytes apart (SBO), descriptor version 1
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;            // version
  d |= (uint64_t)2 << 61;            // swizzle 128B
  return d;
}

// instruction descriptor: D FP32, A/B TF32 (kind::tf32) or BF16 (kind::f16),
// both K-major, M = 128, N = BN
template <bool BF16, int BN>
__device__ __forceinline__ uint32_t instr_desc() {
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "M = 128 takes N in [16, 256], a multiple of 16");
  const uint32_t fmt = BF16 ? 1u : 2u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

template <bool BF16>
__device__ __forceinline__ void mma_issue(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  if (BF16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

template <int MODE, int BN>
__global__ void __launch_bounds__(128, 1) k_tc_gemm(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB,
                                                    const __grid_constant__ CUtensorMap tmA2,
                                                    const __grid_constant__ CUtensorMap tmB2, float* __restrict__ C,
                                                    long ldc, long sC, int M, int N, int nk, int* __restrict__ err,
                                                    float alpha, float beta, int upper, TcSplitOut o2) {
  constexpr bool BF16 = MODE == 1, SPLIT = MODE == 2;
  constexpr int STAGES = tc_stages<MODE, BN>(), SB = tc_stage_bytes<MODE, BN>();
  static_assert(tc_smem<MODE, BN>() <= 227 * 1024, "the stages must fit the opt-in shared memory of a CTA");
  constexpr int BB = tc_b_bytes<BN>();
  extern __shared__ unsigned char tc_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
  // o: A, B, A lo, B lo (every offset a multiple of 1024 bytes)
  auto tile = [&](int s, int o) {
    return base + s * SB + (o & 1) * TC_A_BYTES + (o >> 1) * (TC_A_BYTES + BB);
  };
  uint64_t* bars = (uint64_t*)(base + STAGES * SB);  // full[S], empty[S], done
  uint32_t* tslot = (uint32_t*)(bars + 2 * STAGES + 1);
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * TC_BM, bz = blockIdx.z;
  // upper: a symmetric product (B = A) needs only the tiles not wholly below the diagonal
  if (upper && n0 + BN <= m0) return;
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), done = smem_u32(bars + 2 * STAGES);
  constexpr int KE = BF16 ? 64 : 32;  // elements per 128 bytes of K

  if (tid == 0) {
    s_fail = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;

  int issued = 0;  // stages the producer loaded
  if (tid == 0) {  // TMA producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES, round = kb / STAGES;
      if (round > 0 && !mbar_wait(empty0 + 8 * s, (round - 1) & 1)) {
        s_fail = 1;
        break;
      }
      mbar_expect_tx(full0 + 8 * s, SB);
      tma_load_3d(smem_u32(tile(s, 0)), &tmA, kb * KE, m0, bz, full0 + 8 * s);
      tma_load_3d(smem_u32(tile(s, 1)), &tmB, kb * KE, n0, bz, full0 + 8 * s);
      if (SPLIT) {
        tma_load_3d(smem_u32(tile(s, 2)), &tmA2, kb * KE, m0, bz, full0 + 8 * s);
        tma_load_3d(smem_u32(tile(s, 3)), &tmB2, kb * KE, n0, bz, full0 + 8 * s);
      }
      issued = kb + 1;
    }
  } else if (tid == 32) {  // MMA issuer
    const uint32_t idesc = instr_desc<BF16, BN>();
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES, round = kb / STAGES;
      if (!mbar_wait(full0 + 8 * s, round & 1)) {
        s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint64_t ad = smem_desc_sw128(smem_u32(tile(s, 0)));
      const uint64_t bd = smem_desc_sw128(smem_u32(tile(s, 1)));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {  // 32 bytes of K per instruction: advance the start address by 2 x 16 B
        mma_issue<BF16>(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (kb | kk) != 0);
        if (SPLIT) {
          const uint64_t ad2 = smem_desc_sw128(smem_u32(tile(s, 2)));
          const uint64_t bd2 = smem_desc_sw128(smem_u32(tile(s, 3)));
          mma_issue<BF16>(tmem, ad + 2 * kk, bd2 + 2 * kk, idesc, 1);
          mma_issue<BF16>(tmem, ad2 + 2 * kk, bd + 2 * kk, idesc, 1);
        }
      }
      mma_commit(empty0 + 8 * s);
    }
    mma_commit(done);
  }
  __syncwarp();
  const bool ok = mbar_wait(done, 0);
  __syncwarp();
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();
  const bool good = ok && (s_fail == 0);
  if (good) {
    const int row = m0 + warp * 32 + lane;
    float* crow = C + (long)bz * sC + (long)row * ldc;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {
        float* dst = crow + n0 + c0;
        const bool full = n0 + c0 + 16 <= N;
        float o[16];  // the chunk's final values (C = alpha A B^T + beta C)
        if (full && ((uintptr_t)dst & 15) == 0) {
          // the thread's 16 columns as four 16-byte accesses (the old values all loaded first)
          float4 old4[4];
          if (beta != 0.0f) {
#pragma unroll
            for (int q = 0; q < 4; ++q) old4[q] = reinterpret_cast<const float4*>(dst)[q];
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float4 v = make_float4(alpha * __uint_as_float(r[4 * q]), alpha * __uint_as_float(r[4 * q + 1]),
                                   alpha * __uint_as_float(r[4 * q + 2]), alpha * __uint_as_float(r[4 * q + 3]));
            if (beta != 0.0f) {
              v.x = fmaf(beta, old4[q].x, v.x);
              v.y = fmaf(beta, old4[q].y, v.y);
              v.z = fmaf(beta, old4[q].z, v.z);
              v.w = fmaf(beta, old4[q].w, v.w);
            }
            reinterpret_cast<float4*>(dst)[q] = v;
            o[4 * q] = v.x;
            o[4 * q + 1] = v.y;
            o[4 * q + 2] = v.z;
            o[4 * q + 3] = v.w;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = n0 + c0 + j;
            o[j] = 0.0f;
            if (col < N) {
              const float v = alpha * __uint_as_float(r[j]);
              o[j] = (beta != 0.0f) ? fmaf(beta, crow[col], v) : v;
              crow[col] = o[j];
            }
          }
        }
        if (o2.Rhi) {  // split copy in C's layout
          float* rh = o2.Rhi + (long)bz * o2.sr + (long)row * o2.ldr + n0 + c0;
          float* rl = o2.Rlo + (long)bz * o2.sr + (long)row * o2.ldr + n0 + c0;
          if (full && (((uintptr_t)rh | (uintptr_t)rl) & 15) == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              float h4[4], l4[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                h4[u] = tf32_hi(o[4 * q + u]);
                l4[u] = o[4 * q + u] - h4[u];
              }
              reinterpret_cast<float4*>(rh)[q] = make_float4(h4[0], h4[1], h4[2], h4[3]);
              reinterpret_cast<float4*>(rl)[q] = make_float4(l4[0], l4[1], l4[2], l4[3]);
            }
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (n0 + c0 + j < N) {
                const float hv = tf32_hi(o[j]);
                rh[j] = hv;
                rl[j] = o[j] - hv;
              }
          }
        }
        if (o2.Thi) {  // split copy of C^T: lanes are consecutive rows, so each store is coalesced
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = n0 + c0 + j;
            if (col < N) {
              const long off = (long)bz * o2.st + (long)col * o2.ldt + row;
              const float hv = tf32_hi(o[j]);
              o2.Thi[off] = hv;
              o2.Tlo[off] = o[j] - hv;
            }
          }
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  if (tid == 0) {  // make sure no copy of this CTA is still landing in shared memory
    for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
      mbar_wait(full0 + 8 * (kb % STAGES), (kb / STAGES) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// rows x K (elements) per batch, row stride ld, batch stride sb (elements); boxes of
// box_rows rows x 128 bytes of K
static int make_map(CUtensorMap* tm, const void* ptr, int rows, int K, long ld, long sb, int batch, bool bf16,
                    int box_rows = TC_BM) {
  auto enc = get_encode();
  if (!enc) return TSVD_ERR_CUDA;
  const size_t es = bf16 ? 2 : 4;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * es), (cuuint64_t)(sb * es)};
  cuuint32_t box[3] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(tm, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)ptr, dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? TSVD_OK : TSVD_ERR_UNSUPPORTED;
}

bool tc_gemm_supported(const void* A, long lda, long sA, const void* B, long ldb, long sB, int batch, bool bf16) {
  const long es = bf16 ? 2 : 4;
  auto al = [](long bytes) { return bytes % 16 == 0; };
  if (((uintptr_t)A & 15) || ((uintptr_t)B & 15)) return false;
  if (!al(lda * es) || !al(ldb * es)) return false;
  if (batch > 1 && (!al(sA * es) || !al(sB * es))) return false;
  return batch <= 65535;
}

template <int MODE, int BN>
static int tc_launch(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& ta2, const CUtensorMap& tb2,
                     float* C, long ldc, long sC, int M, int N, int nk, int batch, int* err, cudaStream_t s,
                     float alpha = 1.0f, float beta = 0.0f, int upper = 0, const TcSplitOut& o2 = TcSplitOut()) {
  dim3 grid(cdiv(N, BN), cdiv(M, TC_BM), batch);
  if (cudaFuncSetAttribute(k_tc_gemm<MODE, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem<MODE, BN>()) !=
      cudaSuccess) {
    cudaGetLastError();
    return TSVD_ERR_CUDA;
  }
  k_tc_gemm<MODE, BN><<<grid, 128, tc_smem<MODE, BN>(), s>>>(ta, tb, ta2, tb2, C, ldc, sC, M, N, nk, err, alpha,
                                                               beta, upper, o2);
  TSVD_LAUNCHED();
  return TSVD_OK;
}
// tile width: 256 columns when N > 128 (one tile row covers the whole of N <= 256)
static int tc_bn(int N) { return N > 128 ? 256 : 128; }
int tc_gemm_tile_n(int N, bool bf16) { (void)bf16; return tc_bn(N); }

int tc_gemm(const void* A, long lda, long sA, int M, const void* B, long ldb, long sB, int N, int K, float* C, long ldc,
            long sC, int batch, bool bf16, int* err, cudaStream_t s, bool upper) {
  if (M <= 0 || N <= 0 || batch <= 0) return TSVD_OK;
  if (!tc_gemm_supported(A, lda, sA, B, ldb, sB, batch, bf16)) return TSVD_ERR_UNSUPPORTED;
  CUtensorMap ta, tb;
  const int bn = tc_bn(N);
  TSVD_TRY(make_map(&ta, A, M, K, lda, sA, batch, bf16));
  TSVD_TRY(make_map(&tb, B, N, K, ldb, sB, batch, bf16, bn));
  const int kelem = bf16 ? 64 : 32;
  const int nk = (K + kelem - 1) / kelem;
  const int up = upper ? 1 : 0;
  if (bf16)
    return bn == 256 ? tc_launch<1, 256>(ta, tb, ta, tb, C, ldc, sC, M, N, nk, batch, err, s, 1.f, 0.f, up)
                     : tc_launch<1, 128>(ta, tb, ta, tb, C, ldc, sC, M, N, nk, batch, err, s, 1.f, 0.f, up);
  return bn == 256 ? tc_launch<0, 256>(ta, tb, ta, tb, C, ldc, sC, M, N, nk, batch, err, s, 1.f, 0.f, up)
                   : tc_launch<0, 128>(ta, tb, ta, tb, C, ldc, sC, M, N, nk, batch, err, s, 1.f, 0.f, up);
}

int tc_gemm_split(const float* Ahi, const float* Alo, long lda, long sA, int M, const float* Bhi, const float* Blo,
                  long ldb, long sB, int N, int K, float* C, long ldc, long sC, int batch, int* err, cudaStream_t s,
                  float alpha, float beta, const TcSplitOut* out2) {
  if (M <= 0 || N <= 0 || batch <= 0) return TSVD_OK;
  if (!tc_gemm_supported(Ahi, lda, sA, Bhi, ldb, sB, batch, false) ||
      !tc_gemm_supported(Alo, lda, sA, Blo, ldb, sB, batch, false))
    return TSVD_ERR_UNSUPPORTED;
  // split TF32 keeps 128-column tiles: with four operand tiles per stage a 256-column tile
  // leaves room for two stages only, which measured slower
  CUtensorMap ta, tb, ta2, tb2;
  TSVD_TRY(make_map(&ta, Ahi, M, K, lda, sA, batch, false));
  TSVD_TRY(make_map(&tb, Bhi, N, K, ldb, sB, batch, false));
  TSVD_TRY(make_map(&ta2, Alo, M, K, lda, sA, batch, false));
  TSVD_TRY(make_map(&tb2, Blo, N, K, ldb, sB, batch, false));
  return tc_launch<2, 128>(ta, tb, ta2, tb2, C, ldc, sC, M, N, (K + 31) / 32, batch, err, s, alpha, beta, 0,
                           out2 ? *out2 : TcSplitOut());
}

// ---------------------------------------------------------------------------
// Expanded real forms of a thin complex factor Y (K x N per batch, interleaved,
// leading dim ldy), as E (2N x 2K per batch, leading dim lde), so that for an
// interleaved complex X (rows x K) seen as a real rows x 2K matrix,
// real(X) * E^T is the interleaved complex product:
//   mode 0 (X Y):       E[2n][2k] = Yr, E[2n][2k+1] = -Yi, E[2n+1][2k] = Yi, E[2n+1][2k+1] = Yr
//   mode 1 (conj(X) Y): E[2n][2k] = Yr, E[2n][2k+1] =  Yi, E[2n+1][2k] = Yi, E[2n+1][2k+1] = -Yr
// ---------------------------------------------------------------------------
template <typename O>
__device__ __forceinline__ O cvt_out(float v);
template <>
__device__ __forceinline__ float cvt_out<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_out<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

// 32 x 32 tiles of Y (k rows x n columns) through shared memory: reads
// coalesced along n (Y's rows), writes coalesced along k (E's rows).
template <typename O>
__global__ void __launch_bounds__(256) k_expand(const float2* __restrict__ Y, long ldy, long sy, int K, int N,
                                                O* __restrict__ E, long lde, long se, int mode) {
  __shared__ float2 t[32][33];
  const int b = blockIdx.z, k0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  const float2* Yb = Y + (long)b * sy;
  for (int kk = threadIdx.y; kk < 32; kk += blockDim.y) {
    const int k = k0 + kk, n = n0 + threadIdx.x;
    t[kk][threadIdx.x] = (k < K && n < N) ? Yb[(long)k * ldy + n] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  O* Eb = E + (long)b * se;
  for (int nn = threadIdx.y; nn < 32; nn += blockDim.y) {
    const int n = n0 + nn, k = k0 + threadIdx.x;
    if (n >= N || k >= K) continue;
    const float2 y = t[threadIdx.x][nn];
    O* e0 = Eb + (long)(2 * n) * lde + 2 * k;
    O* e1 = e0 + lde;
    if (mode == 0) {
      e0[0] = cvt_out<O>(y.x);
      e0[1] = cvt_out<O>(-y.y);
      e1[0] = cvt_out<O>(y.y);
      e1[1] = cvt_out<O>(y.x);
    } else {
      e0[0] = cvt_out<O>(y.x);
      e0[1] = cvt_out<O>(y.y);
      e1[0] = cvt_out<O>(y.y);
      e1[1] = cvt_out<O>(-y.x);
    }
  }
}

int expand_thin(const float2* Y, long ldy, long sy, int K, int N, void* E, long lde, long se, int batch, int mode,
                bool bf16, cudaStream_t s) {
  if ((long)batch * K * N <= 0) return TSVD_OK;
  if (batch > 65535 || cdiv(K, 32) > 65535) return TSVD_ERR_UNSUPPORTED;
  dim3 grid(cdiv(N, 32), cdiv(K, 32), batch), block(32, 8);
  if (bf16)
    k_expand<__nv_bfloat16><<<grid, block, 0, s>>>(Y, ldy, sy, K, N, (__nv_bfloat16*)E, lde, se, mode);
  else
    k_expand<float><<<grid, block, 0, s>>>(Y, ldy, sy, K, N, (float*)E, lde, se, mode);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

// rows x cols FP32 (leading dim ldx) to BF16 (round to nearest even) or FP32
// with leading dim ldy; the padding columns are zeroed
template <typename O>
__global__ void k_copy_rows(const float* __restrict__ x, long ldx, O* __restrict__ y, long ldy, int cols, long rows) {
  const long total = rows * ldy;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long r = i / ldy;
    const long c = i % ldy;
    y[i] = cvt_out<O>(c < cols ? x[r * ldx + c] : 0.0f);
  }
}

int copy_rows(const float* x, long ldx, void* y, long ldy, int cols, long rows, bool bf16, cudaStream_t s) {
  const long total = rows * ldy;
  if (total <= 0) return TSVD_OK;
  const unsigned grid = std::min<long>(cdiv(total, 256), 8192);
  if (bf16) k_copy_rows<__nv_bfloat16><<<grid, 256, 0, s>>>(x, ldx, (__nv_bfloat16*)y, ldy, cols, rows);
  else k_copy_rows<float><<<grid, 256, 0, s>>>(x, ldx, (float*)y, ldy, cols, rows);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

// ---------------------------------------------------------------------------
// Split operands for the split-TF32 mode: hi = x rounded to the nearest TF32
// (cvt.rna.tf32.f32), lo = x - hi (exact in FP32).
// ---------------------------------------------------------------------------

// rows x cols FP32 (leading dim ldx) to hi / lo rows of leading dim ldy (padding zeroed)
__global__ void k_split_rows(const float* __restrict__ x, long ldx, float* __restrict__ hi, float* __restrict__ lo,
                             long ldy, int cols, long rows) {
  const long total = rows * ldy;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long r = i / ldy;
    const long c = i % ldy;
    const float v = c < cols ? x[r * ldx + c] : 0.0f;
    const float h = tf32_hi(v);
    hi[i] = h;
    lo[i] = v - h;
  }
}

int split_rows(const float* x, long ldx, float* hi, float* lo, long ldy, int cols, long rows, cudaStream_t s) {
  const long total = rows * ldy;
  if (total <= 0) return TSVD_OK;
  k_split_rows<<<(unsigned)std::min<long>(cdiv(total, 256), 8192), 256, 0, s>>>(x, ldx, hi, lo, ldy, cols, rows);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

// per slice: complex X (rows x cols, interleaved, leading dim cols) transposed
// to XT (cols x rows complex = real rows of 2 rows floats, leading dim ldt),
// split into hi / lo; 32 x 32 complex tiles through shared memory
// columns [0, cols) of FP32 rows (leading dim ldx) -> hi (nearest TF32) / lo rows of leading dim ldy;
// the other columns of the destination rows are left as they are
__global__ void k_split_block(const float* __restrict__ x, long ldx, float* __restrict__ hi, float* __restrict__ lo,
                              long ldy, int cols, long rows) {
  const long total = rows * cols;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long r = i / cols;
    const long c = i % cols;
    const float v = x[r * ldx + c];
    const float h = tf32_hi(v);
    hi[r * ldy + c] = h;
    lo[r * ldy + c] = v - h;
  }
}

int split_block(const float* x, long ldx, float* hi, float* lo, long ldy, int cols, long rows, cudaStream_t s) {
  const long total = rows * cols;
  if (total <= 0) return TSVD_OK;
  k_split_block<<<(unsigned)std::min<long>(cdiv(total, 256), 8192), 256, 0, s>>>(x, ldx, hi, lo, ldy, cols, rows);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

__global__ void k_split_transpose(const float2* __restrict__ X, int rows, int cols, long ldx, long sx,
                                  float* __restrict__ hi, float* __restrict__ lo, long ldt, long st) {
  __shared__ float2 t[32][33];
  const int b = blockIdx.z;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const float2* Xb = X + (long)b * sx;
  for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
    const int r = r0 + rr, c = c0 + threadIdx.x;
    t[rr][threadIdx.x] = (r < rows && c < cols) ? Xb[(long)r * ldx + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float* hb = hi + (long)b * st;
  float* lb = lo + (long)b * st;
  for (int cc = threadIdx.y; cc < 32; cc += blockDim.y) {
    const int c = c0 + cc, r = r0 + threadIdx.x;
    if (c < cols && r < rows) {
      const float2 v = t[threadIdx.x][cc];
      const float hx = tf32_hi(v.x), hy = tf32_hi(v.y);
      hb[(long)c * ldt + 2 * r] = hx;
      hb[(long)c * ldt + 2 * r + 1] = hy;
      lb[(long)c * ldt + 2 * r] = v.x - hx;
      lb[(long)c * ldt + 2 * r + 1] = v.y - hy;
    }
  }
}

int split_transpose(const float2* X, int rows, int cols, int batch, float* hi, float* lo, long ldt, cudaStream_t s) {
  if (rows <= 0 || cols <= 0 || batch <= 0) return TSVD_OK;
  if (batch > 65535) return TSVD_ERR_UNSUPPORTED;
  // zero the padding columns of every row once (2 rows .. ldt)
  if (ldt > 2L * rows) {
    if (cudaMemset2DAsync(hi + 2L * rows, ldt * sizeof(float), 0, (ldt - 2L * rows) * sizeof(float),
                          (size_t)batch * cols, s) != cudaSuccess ||
        cudaMemset2DAsync(lo + 2L * rows, ldt * sizeof(float), 0, (ldt - 2L * rows) * sizeof(float),
                          (size_t)batch * cols, s) != cudaSuccess)
      return TSVD_ERR_CUDA;
  }
  dim3 grid(cdiv(cols, 32), cdiv(rows, 32), batch), block(32, 8);
  k_split_transpose<<<grid, block, 0, s>>>(X, rows, cols, cols, (long)rows * cols, hi, lo, ldt, (long)cols * ldt);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

int split_transpose_ld(const float2* X, int rows, int cols, long ldx, long sx, int batch, float* hi, float* lo,
                       long ldt, long st, cudaStream_t s) {
  if (rows <= 0 || cols <= 0 || batch <= 0) return TSVD_OK;
  if (batch > 65535) return TSVD_ERR_UNSUPPORTED;
  dim3 grid(cdiv(cols, 32), cdiv(rows, 32), batch), block(32, 8);
  k_split_transpose<<<grid, block, 0, s>>>(X, rows, cols, ldx, sx, hi, lo, ldt, st);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

// per slice: the columns of a complex X (rows x cols, leading dim ldx) as real rows of
// length `rows`: row 2c the real parts of column c, row 2c+1 the imaginary parts, split
// into hi / lo (leading dim ldt, batch stride st); 32 x 32 complex tiles through shared memory
__global__ void k_split_deinterleave(const float2* __restrict__ X, int rows, int cols, long ldx, long sx,
                                     float* __restrict__ hi, float* __restrict__ lo, long ldt, long st) {
  __shared__ float2 t[32][33];
  const int b = blockIdx.z;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const float2* Xb = X + (long)b * sx;
  for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
    const int r = r0 + rr, c = c0 + threadIdx.x;
    t[rr][threadIdx.x] = (r < rows && c < cols) ? Xb[(long)r * ldx + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float* hb = hi + (long)b * st;
  float* lb = lo + (long)b * st;
  for (int cc = threadIdx.y; cc < 32; cc += blockDim.y) {
    const int c = c0 + cc, r = r0 + threadIdx.x;
    if (c < cols && r < rows) {
      const float2 v = t[threadIdx.x][cc];
      const float hx = tf32_hi(v.x), hy = tf32_hi(v.y);
      hb[(long)(2 * c) * ldt + r] = hx;
      hb[(long)(2 * c + 1) * ldt + r] = hy;
      lb[(long)(2 * c) * ldt + r] = v.x - hx;
      lb[(long)(2 * c + 1) * ldt + r] = v.y - hy;
    }
  }
}

int split_deinterleave(const float2* X, int rows, int cols, long ldx, long sx, int batch, float* hi, float* lo,
                       long ldt, long st, cudaStream_t s) {
  if (rows <= 0 || cols <= 0 || batch <= 0) return TSVD_OK;
  if (batch > 65535) return TSVD_ERR_UNSUPPORTED;
  dim3 grid(cdiv(cols, 32), cdiv(rows, 32), batch), block(32, 8);
  k_split_deinterleave<<<grid, block, 0, s>>>(X, rows, cols, ldx, sx, hi, lo, ldt, st);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

// expanded real form (as expand_thin, FP32) split into hi / lo; same tiling
__global__ void __launch_bounds__(256) k_expand_split(const float2* __restrict__ Y, long ldy, long sy, int K, int N,
                                                      float* __restrict__ Eh, float* __restrict__ El, long lde,
                                                      long se, int mode) {
  __shared__ float2 t[32][33];
  const int b = blockIdx.z, k0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  const float2* Yb = Y + (long)b * sy;
  for (int kk = threadIdx.y; kk < 32; kk += blockDim.y) {
    const int k = k0 + kk, n = n0 + threadIdx.x;
    t[kk][threadIdx.x] = (k < K && n < N) ? Yb[(long)k * ldy + n] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int nn = threadIdx.y; nn < 32; nn += blockDim.y) {
    const int n = n0 + nn, k = k0 + threadIdx.x;
    if (n >= N || k >= K) continue;
    const float2 y = t[threadIdx.x][nn];
    const float v[4] = {y.x, mode == 0 ? -y.y : y.y, y.y, mode == 0 ? y.x : -y.x};
    const long o0 = (long)b * se + (long)(2 * n) * lde + 2 * k;
    const long off[4] = {o0, o0 + 1, o0 + lde, o0 + lde + 1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float h = tf32_hi(v[q]);
      Eh[off[q]] = h;
      El[off[q]] = v[q] - h;
    }
  }
}

int expand_thin_split(const float2* Y, long ldy, long sy, int K, int N, float* Eh, float* El, long lde, long se,
                      int batch, int mode, cudaStream_t s) {
  if ((long)batch * K * N <= 0) return TSVD_OK;
  if (batch > 65535 || cdiv(K, 32) > 65535) return TSVD_ERR_UNSUPPORTED;
  dim3 grid(cdiv(N, 32), cdiv(K, 32), batch), block(32, 8);
  k_expand_split<<<grid, block, 0, s>>>(Y, ldy, sy, K, N, Eh, El, lde, se, mode);
  TSVD_LAUNCHED();
  return TSVD_OK;
}

}  // namespace tsvd
