// BF16 GEMM on the fifth-generation tensor cores (tcgen05), for the dense layers of the learned pose
// proposal: P_z[M, N] = A[M, K_z] B[N, K_z]^T, A and B row-major BF16 (K contiguous: both operands
// K-major), FP32 accumulation in tensor memory. K is split into gridDim.z ranges of whole 64-wide
// slices (split-K); range z writes its FP32 partial product P_z to C + z M N, and a reduction kernel
// adds the partials and applies the layer's epilogue.
//
// One CTA of 128 threads per 128 x 128 output tile and K range, warp-specialised:
//   - thread 0 (producer) streams the A and B tiles of each 64-wide K slice with TMA
//     (cp.async.bulk.tensor.2d, 128-byte swizzle: 128 rows x 128 bytes = 16 KB per operand) into a
//     3-stage ring; a stage's "full" mbarrier expects the 32 KB of its two copies;
//   - thread 32 (MMA issuer) waits for a stage to be full, issues four 128 x 128 x 16
//     tcgen05.mma.kind::f16 into the 128-column TMEM accumulator and commits them to the stage's
//     "empty" mbarrier, which the producer waits on before refilling that stage; after the last slice
//     it commits once more to the "done" mbarrier;
//   - all four warps wait for "done", read their 32 TMEM lanes (rows) with tcgen05.ld and store the
//     rows below M.
// TMA reads rows past M or N as zeros. Every mbarrier wait is bounded; on a timeout the thread sets
// *err and the CTA skips its stores, but it leaves no asynchronous work behind before it frees its
// TMEM and exits: the MMA issuer commits to "done" whether or not it finished (a commit completes once
// every tcgen05.mma the thread issued before it has completed), and the producer waits (bounded) for
// the TMA copies of the last stages it filled to land.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "internal.cuh"

namespace xslam {

namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64;
constexpr int kTileBytes = kBM * kBK * 2;  // 16 KB per operand tile
constexpr int kStages = 3;  // 97 KB of stages: two CTAs per SM
constexpr unsigned kSpin = 1u << 22;        // try_wait polls before a wait gives up

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor of a K-major operand tile written by TMA with 128-byte swizzle: rows of
// 128 bytes, 8-row atoms of 1024 bytes (stride byte offset), leading byte offset unused (1), version 1,
// layout type 2 (128-byte swizzle). The tile base is 1024-byte aligned.
__device__ __forceinline__ unsigned long long make_desc_sw128(unsigned addr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((addr >> 4) & 0x3FFFu);
  d |= 1ull << 16;
  d |= (unsigned long long)(1024 >> 4) << 32;
  d |= 1ull << 46;
  d |= 2ull << 61;
  return d;
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, M x N
__host__ __device__ constexpr unsigned make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the completion of the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  for (unsigned it = 0; it < kSpin; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// 2-D TMA load of the box at element coordinates (x = K index, y = row) into shared memory
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, int x, int y, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

}  // namespace

__global__ void __launch_bounds__(128) k_gemm_bf16(const __grid_constant__ CUtensorMap tmA,
                                                  const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
                                                  int kb_per_split, float* __restrict__ C, int* err) {
  pdl_enter();
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long full[kStages], empty[kStages], done;
  __shared__ unsigned s_tmem;
  __shared__ int s_bad;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  // the 128-byte swizzle atoms are 1024 bytes: align the stage ring to 1024
  const unsigned sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
  if (threadIdx.x == 0) {
    s_bad = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&tmB)) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(&s_tmem)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = s_tmem;
  const int kb0 = blockIdx.z * kb_per_split;
  const int nk = min(K / kBK - kb0, kb_per_split);  // >= 1 by construction of the grid
  const int kbase = kb0 * kBK;

  if (threadIdx.x == 0) {
    // producer: stage st = s mod S holds slice s; its k-th refill waits for the k-th "empty" phase
    int issued = 0;
    for (int s = 0; s < nk; ++s) {
      const int st = s % kStages;
      if (s >= kStages && !mbar_wait(smem_u32(&empty[st]), (unsigned)((s / kStages - 1) & 1))) {
        s_bad = 1;
        atomicExch(err, 1);
        break;
      }
      const unsigned a_s = sbase + st * 2 * kTileBytes, b_s = a_s + kTileBytes;
      const unsigned bar = smem_u32(&full[st]);
      mbar_expect_tx(bar, 2u * kTileBytes);
      tma_load_2d(a_s, &tmA, kbase + s * kBK, m0, bar);
      tma_load_2d(b_s, &tmB, kbase + s * kBK, n0, bar);
      issued = s + 1;
    }
    // the copies into the last stages may still be in flight if the MMA issuer stopped early: the CTA
    // must not exit while TMA still writes its shared memory (each stage's last use is its final phase)
    for (int s = issued > kStages ? issued - kStages : 0; s < issued; ++s)
      if (!mbar_wait(smem_u32(&full[s % kStages]), (unsigned)((s / kStages) & 1))) atomicExch(err, 1);
  } else if (threadIdx.x == 32) {
    // MMA issuer
    const unsigned idesc = make_idesc(kBM, kBN);
    bool ok = true;
    for (int s = 0; s < nk; ++s) {
      const int st = s % kStages;
      if (!mbar_wait(smem_u32(&full[st]), (unsigned)((s / kStages) & 1))) {
        ok = false;
        atomicExch(err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned a_s = sbase + st * 2 * kTileBytes, b_s = a_s + kTileBytes;
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        // K step of 16 elements = 32 bytes inside the 128-byte swizzled rows
        const unsigned long long ad = make_desc_sw128(a_s + kk * 32);
        const unsigned long long bd = make_desc_sw128(b_s + kk * 32);
        const unsigned acc = (s > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty[st]))
                   : "memory");
    }
    // commit to "done" on every path: it completes when all MMAs issued above have completed, so the
    // wait below also covers an issuer that stopped early
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&done))
                 : "memory");
    if (!ok) s_bad = 1;
  }
  __syncwarp();
  // every MMA of the CTA has completed once "done" completes its first phase; the commit above is
  // issued on every path and MMAs wait on nothing, so this wait ends unless the issuer never ran
  const bool fin = mbar_wait(smem_u32(&done), 0u);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!fin && threadIdx.x == 64) atomicExch(err, 1);
  __syncthreads();
  if (fin && !s_bad) {
    const int row = m0 + warp * 32 + lane;
    float* crow = C + (size_t)blockIdx.z * M * N + (size_t)row * N;
#pragma unroll 1
    for (int c0 = 0; c0 < kBN; c0 += 16) {
      unsigned v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
          "[%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
            "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int col = n0 + c0;
      if (row < M && col < N) {
        if (col + 16 <= N && (N & 3) == 0) {
          float4* dst = reinterpret_cast<float4*>(crow + col);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            dst[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]), __uint_as_float(v[4 * j + 2]),
                                 __uint_as_float(v[4 * j + 3]));
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (col + j < N) crow[col + j] = __uint_as_float(v[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
  }
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// tensor map of a row-major [rows x K] BF16 matrix, box 64 (K) x 128 (rows), 128-byte swizzle, zero fill
cudaError_t make_map(CUtensorMap* map, const void* base, int rows, int K) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

size_t gemm_smem_bytes() { return (size_t)kStages * 2 * kTileBytes + 1024; }

cudaError_t gemm_configure() {
  return cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem_bytes());
}

GemmPlan gemm_plan(int M, int N, int K, int target_ctas) {
  GemmPlan g;
  const int tiles = ((M + kBM - 1) / kBM) * ((N + kBN - 1) / kBN);
  const int nkb = K / kBK;
  int splits = (target_ctas + tiles - 1) / tiles;
  if (splits > nkb) splits = nkb;
  if (splits < 1) splits = 1;
  g.kb_per_split = (nkb + splits - 1) / splits;
  g.splits = (nkb + g.kb_per_split - 1) / g.kb_per_split;
  return g;
}

bool gemm_shape_ok(int M, int N, int K) { return M >= 1 && N >= 1 && K >= kBK && K % kBK == 0; }

cudaError_t launch_gemm_bf16(const void* A, const void* B, int M, int N, int K, const GemmPlan& g, float* C, int* err,
                             cudaStream_t s) {
  alignas(64) CUtensorMap ta, tb;
  cudaError_t e = make_map(&ta, A, M, K);
  if (e == cudaSuccess) e = make_map(&tb, B, N, K);
  if (e != cudaSuccess) return e;
  dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, g.splits);
  return launch_pdl(k_gemm_bf16, grid, dim3(128), gemm_smem_bytes(), s, ta, tb, M, N, K, g.kb_per_split, C, err);
}

}  // namespace xslam
