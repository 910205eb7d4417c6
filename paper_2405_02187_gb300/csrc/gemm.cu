// BF16 GEMM on the fifth-generation tensor cores (tcgen05), for the dense layers of the learned pose
// proposal: P_z[M, N] = A[M, K_z] B[N, K_z]^T, A and B row-major BF16 (K contiguous: both operands
// K-major), FP32 accumulation in tensor memory. K is split into gridDim.z ranges of whole 64-wide
// slices (split-K); range z writes its FP32 partial product P_z to C + z M N, and a reduction kernel
// adds the partials and applies the layer's epilogue.
//
// One CTA of 128 threads per 128 x 128 output tile and K range. Per 64-wide slice of K the CTA copies
// the A and B tiles (2 x 16 KB) into shared memory in the canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices, 128 bytes apart along K (leading byte offset) and 1024 bytes apart
// along M/N (stride byte offset); two stages, so the copy of slice s + 1 overlaps the MMAs of slice s.
// Rows past M or N are zero-filled in shared memory and never read from global memory. One thread
// issues the four 128 x 128 x 16 MMAs of a slice into the 128-column TMEM accumulator and commits
// them to the stage's mbarrier. After the last slice every warp reads its 32 TMEM lanes (rows) with
// tcgen05.ld and stores the rows below M. Every mbarrier wait is bounded; on a timeout the CTA sets
// *err, skips its stores and still releases its TMEM.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace xslam {

namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64;
constexpr int kTileBytes = kBM * kBK * 2;  // 16 KB per operand tile
constexpr int kStages = 2;
constexpr unsigned kSpin = 1u << 22;  // try_wait polls before a wait gives up

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle (layout type 0), version 1
__device__ __forceinline__ unsigned long long make_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  unsigned long long d = 0;
  d |= (unsigned long long)((addr >> 4) & 0x3FFFu);
  d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;
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

// bounded wait; false on timeout
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  for (unsigned it = 0; it < kSpin; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void cp_async16(unsigned dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// copy the 128 x 64 BF16 tile starting at (row0, k0) of a row-major [rows, K] matrix into the core-matrix
// layout at smem address dst (rows beyond `rows` are zero-filled)
__device__ __forceinline__ void load_tile(unsigned dst, const __nv_bfloat16* __restrict__ src, int rows, int K, int row0,
                                          int k0) {
  for (int c = threadIdx.x; c < kBM * (kBK / 8); c += blockDim.x) {
    const int r = c >> 3, kc = c & 7;
    const unsigned off = (unsigned)((r >> 3) * 1024 + kc * 128 + (r & 7) * 16);
    if (row0 + r < rows) {
      cp_async16(dst + off, src + (size_t)(row0 + r) * K + k0 + kc * 8);
    } else {
      asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(dst + off), "r"(0) : "memory");
    }
  }
}

}  // namespace

__global__ void __launch_bounds__(128) k_gemm_bf16(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B,
                                                  int M, int N, int K, int kb_per_split, float* __restrict__ C, int* err) {
  pdl_enter();
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) unsigned long long bars[kStages];
  __shared__ unsigned s_tmem;
  __shared__ int s_bad;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  const unsigned sbase = smem_u32(smem);
  if (threadIdx.x == 0) {
    s_bad = 0;
    for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(&bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(&s_tmem)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = s_tmem;
  const unsigned idesc = make_idesc(kBM, kBN);
  const int kb0 = blockIdx.z * kb_per_split;
  const int nk = min(K / kBK - kb0, kb_per_split);  // >= 1 by construction of the grid
  const int kbase = kb0 * kBK;
  unsigned phase[kStages] = {0, 0};

  // prologue: slice 0 into stage 0
  load_tile(sbase, A, M, K, m0, kbase);
  load_tile(sbase + kTileBytes, B, N, K, n0, kbase);
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (int s = 0; s < nk; ++s) {
    const int st = s & 1;
    const unsigned a_s = sbase + st * 2 * kTileBytes, b_s = a_s + kTileBytes;
    // the copies of slice s are complete and visible to the tensor core (async proxy)
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && !s_bad) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        const unsigned long long ad = make_desc(a_s + kk * 256, 128, 1024);
        const unsigned long long bd = make_desc(b_s + kk * 256, 128, 1024);
        const unsigned acc = (s > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bars[st]))
                   : "memory");
    }
    // before stage st ^ 1 is refilled, the MMAs of slice s - 1 (which read it) must have completed
    if (s + 1 < nk) {
      if (s >= 1 && threadIdx.x == 0 && !s_bad) {
        if (!mbar_wait(smem_u32(&bars[st ^ 1]), phase[st ^ 1])) s_bad = 1;
      }
      if (s >= 1) phase[st ^ 1] ^= 1u;
      __syncthreads();
      const unsigned a_n = sbase + (st ^ 1) * 2 * kTileBytes;
      load_tile(a_n, A, M, K, m0, kbase + (s + 1) * kBK);
      load_tile(a_n + kTileBytes, B, N, K, n0, kbase + (s + 1) * kBK);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
  }
  // the last slice's commit (and with it every earlier MMA) has completed
  if (threadIdx.x == 0 && !s_bad) {
    const int last = (nk - 1) & 1;
    if (!mbar_wait(smem_u32(&bars[last]), phase[last])) s_bad = 1;
    // an earlier, still unconsumed commit of the other stage
    if (nk >= 2 && !s_bad && !mbar_wait(smem_u32(&bars[last ^ 1]), phase[last ^ 1])) s_bad = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!s_bad) {
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
  } else if (threadIdx.x == 0) {
    atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
  }
}

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
  dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, g.splits);
  return launch_pdl(k_gemm_bf16, grid, dim3(128), gemm_smem_bytes(), s, (const __nv_bfloat16*)A,
                    (const __nv_bfloat16*)B, M, N, K, g.kb_per_split, C, err);
}

}  // namespace xslam
