// K-major contractions of the triage surrogate on the 5th-generation tensor
// cores (paper Sec. 3.5: affinity predictor on ligand features).
//
//   C = epi(A B^T)  with A [M][K] BF16 and B [N][K] BF16 (K contiguous in
//   both), FP32 accumulation, BF16 output C [M][N].  Epilogues:
//     EPI_BIAS_RELU  forward layer   C = relu(acc + bias)   (B = W^T)
//     EPI_RELU_MASK  data gradient   C = acc * (mask > 0)   (B = W)
//
// One CTA computes a 128 x 256 tile.  One elected thread streams 64-wide K
// slices of X and Wt into shared memory with TMA (128-byte swizzle, three
// stages, mbarrier transaction counts) and issues tcgen05.mma (kind::f16,
// M = 128, N = 256, K = 16 per instruction) into a 256-column FP32
// accumulator in tensor memory; tcgen05.commit signals each stage's release
// and the final completion.  All four warps then read their 32 accumulator
// rows with tcgen05.ld, add the bias, apply ReLU and store BF16.
//
// Every mbarrier wait is bounded by the global timer: on a timeout the kernel
// records an error, drains what it issued (bounded again), frees its tensor
// memory and returns, so the host reports LIGATE_ERR_TIMEOUT instead of
// hanging.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "ligate_internal.h"
#include "mlp.h"

namespace ligate {
namespace mlp {
namespace {

constexpr int TM = 128, TN = 256, TK = 64, STAGES = 3;
constexpr int A_BYTES = TM * TK * 2, B_BYTES = TN * TK * 2;  // 16 KB + 32 KB per stage
constexpr int TMEM_COLS = 256;
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ uint32_t saddr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on phase `parity`; false after WAIT_NS.
__device__ bool mbar_wait(uint64_t *bar, unsigned parity) {
  const unsigned long long t0 = now_ns();
  while (!mbar_test(bar, parity))
    if (now_ns() - t0 > WAIT_NS) return false;
  return true;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(saddr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(saddr(bar)), "r"(x), "r"(y)
      : "memory");
}
// Shared-memory matrix descriptor, K-major operand with 128-byte swizzle:
// start address >> 4 in bits [0,14), stride between 8-row groups (1024 B)
// >> 4 in [32,46), descriptor version 1 in [46,48), swizzle mode 2 in [61,64).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor of kind::f16: FP32 accumulator (bits [4,6) = 1),
// BF16 A and B ([7,10) = 1, [10,13) = 1), both K-major, N >> 3 in [17,23),
// M >> 4 in [24,29).
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   saddr(bar))
               : "memory");
}

// Fault flag for tests of the timeout path (ligate_debug_inject_fault):
// nothing in normal operation sets it.
__device__ int g_fault_skip_loads = 0;

struct __align__(1024) Smem {
  uint8_t a[STAGES][A_BYTES];
  uint8_t b[STAGES][B_BYTES];
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t done;
  uint32_t tmem_base;
};

template <int EPI>
__global__ void __launch_bounds__(128, 1)
    gemm_tc05_kernel(const __grid_constant__ CUtensorMap tm_a, const __grid_constant__ CUtensorMap tm_b,
                     int M, int K, const float *__restrict__ bias,
                     const __nv_bfloat16 *__restrict__ mask, __nv_bfloat16 *__restrict__ out,
                     int ldc, int *__restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  Smem &s = *reinterpret_cast<Smem *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int nk = K / TK;

  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) { mbar_init(&s.full[i], 1); mbar_init(&s.empty[i], 1); }
    mbar_init(&s.done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // one warp allocates the accumulator columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(&s.tmem_base)), "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s.tmem_base;

  __shared__ int ok_shared;
  if (threadIdx.x == 0) {
    bool ok = true;
    int issued = 0;  // K slices whose loads were issued
    // test hook: a CTA that takes the fault flag issues no loads, so its
    // bounded wait on the first stage runs out and the error path runs
    const bool skip_loads = atomicExch(&g_fault_skip_loads, 0) != 0;
    for (int kb = 0; kb < nk && kb < STAGES && !skip_loads; ++kb, ++issued) {
      mbar_expect_tx(&s.full[kb], A_BYTES + B_BYTES);
      tma_load_2d(s.a[kb], &tm_a, &s.full[kb], kb * TK, m0);
      tma_load_2d(s.b[kb], &tm_b, &s.full[kb], kb * TK, n0);
    }
    int consumed = 0;
    for (int kb = 0; kb < nk && ok; ++kb) {
      const int st = kb % STAGES;
      const unsigned ph = (kb / STAGES) & 1u;
      if (!mbar_wait(&s.full[st], ph)) { ok = false; break; }
      consumed = kb + 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t da = sdesc(saddr(s.a[st])), db = sdesc(saddr(s.b[st]));
#pragma unroll
      for (int kk = 0; kk < TK / 16; ++kk)  // 16 BF16 = 32 B per step: +2 in the address field
        mma_f16(tmem, da + 2 * kk, db + 2 * kk, (kb > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&s.empty[st]);
      if (kb + STAGES < nk) {  // refill this stage once its MMAs are done
        if (!mbar_wait(&s.empty[st], ph)) { ok = false; break; }
        mbar_expect_tx(&s.full[st], A_BYTES + B_BYTES);
        tma_load_2d(s.a[st], &tm_a, &s.full[st], (kb + STAGES) * TK, m0);
        tma_load_2d(s.b[st], &tm_b, &s.full[st], (kb + STAGES) * TK, n0);
        ++issued;
      }
    }
    if (!ok) {  // drain loads still in flight (bounded), then report
      for (int kb = consumed; kb < issued; ++kb)
        (void)mbar_wait(&s.full[kb % STAGES], (kb / STAGES) & 1u);
      atomicExch(err, 1);
    }
    mma_commit(&s.done);  // arrives once every MMA issued so far has completed
    ok_shared = ok ? 1 : 0;
  }
  __syncthreads();
  const bool done_ok = mbar_wait(&s.done, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!done_ok && lane == 0) atomicExch(err, 1);
  // block-uniform decision: tcgen05.ld is warp-collective
  if (__syncthreads_and(ok_shared && done_ok)) {
    // warp w owns accumulator rows 32 w .. 32 w + 31 (tensor-memory lanes)
    const int row = m0 + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < TN; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
            "=r"(r[14]), "=r"(r[15])
          : "r"(trow + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {
        __align__(16) __nv_bfloat162 o[8];
        __align__(16) __nv_bfloat162 hm[8];
        if (EPI == EPI_RELU_MASK) {
          const uint4 *src = reinterpret_cast<const uint4 *>(mask + (size_t)row * ldc + n0 + c0);
          *reinterpret_cast<uint4 *>(&hm[0]) = src[0];
          *reinterpret_cast<uint4 *>(&hm[4]) = src[1];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int n = n0 + c0 + 2 * q;
          float v0 = __uint_as_float(r[2 * q]), v1 = __uint_as_float(r[2 * q + 1]);
          if (EPI == EPI_BIAS_RELU) {
            v0 = fmaxf(v0 + bias[n], 0.f);
            v1 = fmaxf(v1 + bias[n + 1], 0.f);
          } else {
            if (!(__bfloat162float(hm[q].x) > 0.f)) v0 = 0.f;
            if (!(__bfloat162float(hm[q].y) > 0.f)) v1 = 0.f;
          }
          o[q] = __floats2bfloat162_rn(v0, v1);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(out + (size_t)row * ldc + n0 + c0);
        dst[0] = *reinterpret_cast<const uint4 *>(&o[0]);
        dst[1] = *reinterpret_cast<const uint4 *>(&o[4]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                 : "memory");
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// 2-D BF16 map of a row-major [rows][cols] matrix with a (64 x box_rows) box.
bool make_map(CUtensorMap *m, const void *base, int rows, int cols, int box_rows) {
  EncodeTiledFn f = encode_fn();
  if (!f) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return f(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool tc05_supported(int M, int N, int K) {
  return M > 0 && N % TN == 0 && K % TK == 0 && K >= TK && encode_fn() != nullptr;
}

cudaError_t gemm_tc05(int epi, const __nv_bfloat16 *a, int M, int K, const __nv_bfloat16 *b, int N,
                      const float *bias, const __nv_bfloat16 *mask, __nv_bfloat16 *out, int *err,
                      cudaStream_t s) {
  if (!tc05_supported(M, N, K) || (epi != EPI_BIAS_RELU && epi != EPI_RELU_MASK) ||
      (reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(out)) & 15)
    return cudaErrorInvalidValue;
  CUtensorMap ta, tb;
  if (!make_map(&ta, a, M, K, TM) || !make_map(&tb, b, N, K, TN)) return cudaErrorInvalidValue;
  const int smem = (int)sizeof(Smem) + 1024;
  // per-device attribute set-up is cheap; repeat it rather than cache per device
  cudaError_t e = cudaFuncSetAttribute(gemm_tc05_kernel<EPI_BIAS_RELU>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_tc05_kernel<EPI_RELU_MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
  if (e != cudaSuccess) return e;
  dim3 grid(N / TN, (M + TM - 1) / TM);
  if (epi == EPI_BIAS_RELU)
    gemm_tc05_kernel<EPI_BIAS_RELU><<<grid, 128, smem, s>>>(ta, tb, M, K, bias, nullptr, out, N, err);
  else
    gemm_tc05_kernel<EPI_RELU_MASK><<<grid, 128, smem, s>>>(ta, tb, M, K, nullptr, mask, out, N, err);
  return cudaGetLastError();
}

cudaError_t inject_skip_loads_once() {
  const int one = 1;
  return cudaMemcpyToSymbol(g_fault_skip_loads, &one, sizeof(int));
}

// Wt[n][k] = bf16(W[k][n]) for a row-major [K][N] FP32 weight matrix.
__global__ void transpose_bf16_kernel(const float *__restrict__ w, int K, int N,
                                      __nv_bfloat16 *__restrict__ wt) {
  __shared__ float tile[32][33];
  const int k0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, n = n0 + threadIdx.x;
    tile[r][threadIdx.x] = (k < K && n < N) ? w[(size_t)k * N + n] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int n = n0 + r, k = k0 + threadIdx.x;
    if (n < N && k < K) wt[(size_t)n * K + k] = __float2bfloat16_rn(tile[threadIdx.x][r]);
  }
}

cudaError_t transpose_bf16(const float *w, int K, int N, __nv_bfloat16 *wt, cudaStream_t s) {
  dim3 grid((N + 31) / 32, (K + 31) / 32), block(32, 8);
  transpose_bf16_kernel<<<grid, block, 0, s>>>(w, K, N, wt);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace ligate
