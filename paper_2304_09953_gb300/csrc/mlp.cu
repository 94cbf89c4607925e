// Triage surrogate network on the tensor cores (paper Sec. 3.5: an affinity
// predictor on ligand features, trained on data the workflow generates).
//
// MLP 256 -> 512 -> 512 -> 512 -> 1, ReLU on hidden layers.  Weights and
// activations in BF16, products accumulated in FP32 by mma.sync m16n8k16,
// FP32 master weights updated by Adam.  One tiled GEMM kernel serves the
// three product shapes of a training step:
//   forward      H_l = relu(H_{l-1} W_l + b_l)        A row-major, B row-major
//   data grad    dH_{l-1} = dZ_l W_l^T (then ReLU mask) A row-major, B = W^T
//   weight grad  dW_l = H_{l-1}^T dZ_l                 A = H^T,      B row-major
// Operand layouts are template flags; ldmatrix (.trans where the tile is
// stored k-major) feeds the fragments.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "ligate_internal.h"
#include "mlp.h"

namespace ligate {
namespace mlp {

constexpr int BM = 128, BN = 128, BKT = 32, PAD = 8;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3,
                                        const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3,
                                          const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// C[M][N] = sum_k A(m,k) B(k,n).  A(m,k) = A[m*sAm + k*sAk], B(k,n) =
// B[k*sBk + n*sBn]; the contiguous dimension (stride 1) is given by the
// template flags and must be a multiple of 8 elements with 16 B aligned
// rows; the other dimension is bounds-checked (zero fill).
template <bool A_KCONTIG, bool B_KCONTIG, int EPI>
__global__ void __launch_bounds__(256) gemm_kernel(GemmArgs g) {
  // A tile: [BM][BKT+PAD] if k-contiguous else [BKT][BM+PAD]; same for B with BN.
  __shared__ __align__(16) __nv_bfloat16 As[A_KCONTIG ? BM * (BKT + PAD) : BKT * (BM + PAD)];
  __shared__ __align__(16) __nv_bfloat16 Bs[B_KCONTIG ? BN * (BKT + PAD) : BKT * (BN + PAD)];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 2, wn = warp & 3;  // 2 x 4 warps, warp tile 64 x 32
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

  const __nv_bfloat16 *A = g.A, *B = g.B;
  for (int k0 = 0; k0 < g.K; k0 += BKT) {
    // ---- global -> shared
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int c = tid + r * 256;  // 512 16-byte chunks per tile
      uint4 v = make_uint4(0, 0, 0, 0);
      if (A_KCONTIG) {
        const int row = c >> 2, kc = (c & 3) * 8;
        const int m = m0 + row, k = k0 + kc;
        if (m < g.M && k < g.K) v = *reinterpret_cast<const uint4 *>(A + (size_t)m * g.sAm + k);
        *reinterpret_cast<uint4 *>(&As[row * (BKT + PAD) + kc]) = v;
      } else {
        const int krow = c >> 4, mc = (c & 15) * 8;
        const int m = m0 + mc, k = k0 + krow;
        if (k < g.K && m < g.M) v = *reinterpret_cast<const uint4 *>(A + (size_t)k * g.sAk + m);
        *reinterpret_cast<uint4 *>(&As[krow * (BM + PAD) + mc]) = v;
      }
      uint4 w = make_uint4(0, 0, 0, 0);
      if (B_KCONTIG) {
        const int row = c >> 2, kc = (c & 3) * 8;
        const int n = n0 + row, k = k0 + kc;
        if (n < g.N && k < g.K) w = *reinterpret_cast<const uint4 *>(B + (size_t)n * g.sBn + k);
        *reinterpret_cast<uint4 *>(&Bs[row * (BKT + PAD) + kc]) = w;
      } else {
        const int krow = c >> 4, nc = (c & 15) * 8;
        const int n = n0 + nc, k = k0 + krow;
        if (k < g.K && n < g.N) w = *reinterpret_cast<const uint4 *>(B + (size_t)k * g.sBk + n);
        *reinterpret_cast<uint4 *>(&Bs[krow * (BN + PAD) + nc]) = w;
      }
    }
    __syncthreads();
    // ---- tensor-core products over the two k16 steps of the tile
#pragma unroll
    for (int ks = 0; ks < BKT; ks += 16) {
      uint32_t af[4][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int mb = wm * 64 + i * 16;
        if (A_KCONTIG) {
          const __nv_bfloat16 *p = &As[(mb + (lane & 15)) * (BKT + PAD) + ks + (lane >> 4) * 8];
          ldsm_x4(af[i][0], af[i][1], af[i][2], af[i][3], p);
        } else {
          const int r = lane & 7, mi = (lane >> 3) & 1, ki = lane >> 4;
          const __nv_bfloat16 *p = &As[(ks + ki * 8 + r) * (BM + PAD) + mb + mi * 8];
          ldsm_x4_t(af[i][0], af[i][1], af[i][2], af[i][3], p);
        }
      }
#pragma unroll
      for (int j = 0; j < 4; j += 2) {
        const int nb = wn * 32 + j * 8;
        if (B_KCONTIG) {
          // lanes 0-7: n 0-7 k0 | 8-15: n 0-7 k8 | 16-23: n 8-15 k0 | 24-31: n 8-15 k8
          const int r = lane & 7, ki = (lane >> 3) & 1, ni = lane >> 4;
          const __nv_bfloat16 *p = &Bs[(nb + ni * 8 + r) * (BKT + PAD) + ks + ki * 8];
          ldsm_x4(bf[j][0], bf[j][1], bf[j + 1][0], bf[j + 1][1], p);
        } else {
          const int r = lane & 7, ki = (lane >> 3) & 1, ni = lane >> 4;
          const __nv_bfloat16 *p = &Bs[(ks + ki * 8 + r) * (BN + PAD) + nb + ni * 8];
          ldsm_x4_t(bf[j][0], bf[j][1], bf[j + 1][0], bf[j + 1][1], p);
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j][0], bf[j][1]);
    }
    __syncthreads();
  }
  // ---- epilogue
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = m0 + wm * 64 + i * 16 + (lane >> 2) + h * 8;
        const int n = n0 + wn * 32 + j * 8 + (lane & 3) * 2;
        if (m >= g.M || n >= g.N) continue;
        float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
        if (EPI == EPI_BIAS_RELU) {
          v0 = fmaxf(v0 + g.bias[n], 0.f);
          v1 = fmaxf(v1 + g.bias[n + 1], 0.f);
          *reinterpret_cast<__nv_bfloat162 *>(g.Cb + (size_t)m * g.ldc + n) = __floats2bfloat162_rn(v0, v1);
        } else if (EPI == EPI_RELU_MASK) {
          const __nv_bfloat162 hm = *reinterpret_cast<const __nv_bfloat162 *>(g.mask + (size_t)m * g.ldc + n);
          if (!(__bfloat162float(hm.x) > 0.f)) v0 = 0.f;
          if (!(__bfloat162float(hm.y) > 0.f)) v1 = 0.f;
          *reinterpret_cast<__nv_bfloat162 *>(g.Cb + (size_t)m * g.ldc + n) = __floats2bfloat162_rn(v0, v1);
        } else {
          *reinterpret_cast<float2 *>(g.Cf + (size_t)m * g.ldc + n) = make_float2(v0, v1);
        }
      }
}

template <bool AK, bool BKc, int EPI>
static cudaError_t gemm_t(const GemmArgs &g, cudaStream_t s) {
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM);
  gemm_kernel<AK, BKc, EPI><<<grid, 256, 0, s>>>(g);
  return cudaGetLastError();
}

cudaError_t gemm(int kind, const GemmArgs &g, cudaStream_t s) {
  switch (kind) {
    case GEMM_FWD: return gemm_t<true, false, EPI_BIAS_RELU>(g, s);
    case GEMM_DGRAD: return gemm_t<true, true, EPI_RELU_MASK>(g, s);
    default: return gemm_t<false, false, EPI_F32>(g, s);
  }
}

// ---------------------------------------------------------------------------
// Small kernels of a training / inference step.

// Standardise gathered rows: x[b][f] = bf16((desc[idx[b]][f] - mu[f]) * inv_sd[f]).
__global__ void gather_std_kernel(const float *__restrict__ desc, const int *__restrict__ idx,
                                  int rows, int row0, const float *__restrict__ mu,
                                  const float *__restrict__ inv_sd, const float *__restrict__ labels,
                                  float ly_mu, float ly_inv, __nv_bfloat16 *__restrict__ x,
                                  float *__restrict__ t) {
  const int b = blockIdx.x;
  if (b >= rows) return;
  const int src = idx ? idx[b] : row0 + b;
  for (int f = threadIdx.x; f < 256; f += blockDim.x)
    x[(size_t)b * 256 + f] = __float2bfloat16_rn((desc[(size_t)src * 256 + f] - mu[f]) * inv_sd[f]);
  if (t && threadIdx.x == 0) t[b] = (labels[src] - ly_mu) * ly_inv;
}

// Last layer y[b] = H3[b] . w4 + b4 (one warp per row); with targets, also
// dy = 2 (y - t) / B, the squared error sum, and dZ3 = dy w4^T masked by
// H3 > 0 (BF16).
__global__ void head_kernel(const __nv_bfloat16 *__restrict__ h3, const __nv_bfloat16 *__restrict__ w4,
                            const float *__restrict__ b4, int rows, const float *__restrict__ t,
                            float *__restrict__ y, float *__restrict__ dy, float inv_b2,
                            double *__restrict__ sse, __nv_bfloat16 *__restrict__ dz3) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= rows) return;
  const __nv_bfloat16 *h = h3 + (size_t)warp * 512;
  float s = 0.f;
  for (int k = lane; k < 512; k += 32) s = fmaf(__bfloat162float(h[k]), __bfloat162float(w4[k]), s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  s += b4[0];
  if (lane == 0 && y) y[warp] = s;
  if (!t) return;
  const float e = s - t[warp];
  const float d = inv_b2 * e;  // 2 (y - t) / B
  if (lane == 0) {
    dy[warp] = d;
    atomicAdd(sse, (double)e * e);
  }
  for (int k = lane; k < 512; k += 32) {
    const float hv = __bfloat162float(h[k]);
    dz3[(size_t)warp * 512 + k] = __float2bfloat16_rn(hv > 0.f ? d * __bfloat162float(w4[k]) : 0.f);
  }
}

// Gradients of the last layer: gw4[k] = sum_b H3[b][k] dy[b], gb4 = sum_b dy[b].
__global__ void head_grad_kernel(const __nv_bfloat16 *__restrict__ h3, const float *__restrict__ dy,
                                 int rows, float *__restrict__ gw4, float *__restrict__ gb4) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < 512) {
    float s = 0.f;
    for (int b = 0; b < rows; ++b) s = fmaf(__bfloat162float(h3[(size_t)b * 512 + k]), dy[b], s);
    gw4[k] = s;
  }
  if (k == 0) {
    float s = 0.f;
    for (int b = 0; b < rows; ++b) s += dy[b];
    gb4[0] = s;
  }
}

// Column sums of BF16 dZ[rows][cols] (bias gradients).
__global__ void colsum_kernel(const __nv_bfloat16 *__restrict__ dz, int rows, int cols,
                              float *__restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int b = 0; b < rows; ++b) s += __bfloat162float(dz[(size_t)b * cols + c]);
  out[c] = s;
}

// Adam (Kingma & Ba, Algorithm 1) on FP32 master weights, then the BF16 copy.
__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, __nv_bfloat16 *__restrict__ wb, int n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void to_bf16_kernel(const float *__restrict__ a, __nv_bfloat16 *__restrict__ b, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

// Per-feature mean and 1/std (population; zero spread -> 1) of desc[n][256],
// accumulated in FP64: one block per feature.
__global__ void feature_stats_kernel(const float *__restrict__ desc, int n, float *__restrict__ mu,
                                     float *__restrict__ inv_sd) {
  const int f = blockIdx.x;
  __shared__ double s1[256], s2[256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = desc[(size_t)i * 256 + f];
    a += v;
    b += v * v;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) { s1[threadIdx.x] += s1[threadIdx.x + o]; s2[threadIdx.x] += s2[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double m = s1[0] / n;
    double var = s2[0] / n - m * m;
    if (var < 0) var = 0;
    const double sd = sqrt(var);
    mu[f] = (float)m;
    inv_sd[f] = sd > 1e-12 ? (float)(1.0 / sd) : 1.f;
  }
}

// Mean and std of labels[n] (FP64), single block.
__global__ void label_stats_kernel(const float *__restrict__ y, int n, double *__restrict__ out) {
  __shared__ double s1[256], s2[256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) { a += y[i]; b += (double)y[i] * y[i]; }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) { s1[threadIdx.x] += s1[threadIdx.x + o]; s2[threadIdx.x] += s2[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double m = s1[0] / n;
    double var = s2[0] / n - m * m;
    out[0] = m;
    out[1] = var > 0 ? sqrt(var) : 1.0;
  }
}

// Predictions back to label units.
__global__ void unstd_kernel(float *__restrict__ y, int n, float mu, float sd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = y[i] * sd + mu;
}

// ---------------------------------------------------------------------------
// Ranking: bitonic sort of (order-preserving key of the prediction, index)
// packed in 64 bits, so ties resolve by smaller index.
__device__ __forceinline__ uint32_t ordered_key(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void make_keys_kernel(const float *__restrict__ pred, int n, int n2,
                                 unsigned long long *__restrict__ keys) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n2) return;
  if (i < n) {
    const float p = pred[i];
    const uint32_t k = isnan(p) ? 0xffffffffu : ordered_key(p);
    keys[i] = ((unsigned long long)k << 32) | (uint32_t)i;
  } else {
    keys[i] = ~0ull;
  }
}

__global__ void bitonic_global_kernel(unsigned long long *__restrict__ a, int n2, int k, int j) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n2) return;
  const int l = i ^ j;
  if (l > i) {
    const unsigned long long x = a[i], y = a[l];
    const bool up = (i & k) == 0;
    if ((x > y) == up) { a[i] = y; a[l] = x; }
  }
}

// All stages j <= 1024 of size k inside one 2048-element shared tile.
__global__ void bitonic_shared_kernel(unsigned long long *__restrict__ a, int n2, int k) {
  __shared__ unsigned long long s[2048];
  const int base = blockIdx.x * 2048;
  for (int q = threadIdx.x; q < 2048; q += blockDim.x) s[q] = a[base + q];
  __syncthreads();
  for (int j = (k >> 1) < 1024 ? (k >> 1) : 1024; j > 0; j >>= 1) {
    for (int q = threadIdx.x; q < 2048; q += blockDim.x) {
      const int l = q ^ j;
      if (l > q) {
        const int gi = base + q;
        const unsigned long long x = s[q], y = s[l];
        const bool up = (gi & k) == 0;
        if ((x > y) == up) { s[q] = y; s[l] = x; }
      }
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < 2048; q += blockDim.x) a[base + q] = s[q];
}

__global__ void take_idx_kernel(const unsigned long long *__restrict__ keys, int k,
                                int32_t *__restrict__ idx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) idx[i] = (int32_t)(keys[i] & 0xffffffffu);
}

cudaError_t sort_select(const float *pred, int n, int k, unsigned long long *keys, int n2,
                        int32_t *idx, cudaStream_t s) {
  make_keys_kernel<<<(n2 + 255) / 256, 256, 0, s>>>(pred, n, n2, keys);
  for (int kk = 2; kk <= n2; kk <<= 1) {
    for (int j = kk >> 1; j >= 2048; j >>= 1)
      bitonic_global_kernel<<<(n2 + 255) / 256, 256, 0, s>>>(keys, n2, kk, j);
    bitonic_shared_kernel<<<n2 / 2048, 1024, 0, s>>>(keys, n2, kk);
  }
  if (k > 0) take_idx_kernel<<<(k + 255) / 256, 256, 0, s>>>(keys, k, idx);
  return cudaGetLastError();
}

// Launch helpers used by the surrogate object.
cudaError_t gather_std(const float *desc, const int *idx, int rows, int row0, const float *mu,
                       const float *inv_sd, const float *labels, float ly_mu, float ly_inv,
                       __nv_bfloat16 *x, float *t, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  gather_std_kernel<<<rows, 128, 0, s>>>(desc, idx, rows, row0, mu, inv_sd, labels, ly_mu, ly_inv, x, t);
  return cudaGetLastError();
}
cudaError_t head(const __nv_bfloat16 *h3, const __nv_bfloat16 *w4, const float *b4, int rows,
                 const float *t, float *y, float *dy, float inv_b2, double *sse, __nv_bfloat16 *dz3,
                 cudaStream_t s) {
  head_kernel<<<(rows * 32 + 255) / 256, 256, 0, s>>>(h3, w4, b4, rows, t, y, dy, inv_b2, sse, dz3);
  return cudaGetLastError();
}
cudaError_t head_grad(const __nv_bfloat16 *h3, const float *dy, int rows, float *gw4, float *gb4,
                      cudaStream_t s) {
  head_grad_kernel<<<2, 256, 0, s>>>(h3, dy, rows, gw4, gb4);
  return cudaGetLastError();
}
cudaError_t colsum(const __nv_bfloat16 *dz, int rows, int cols, float *out, cudaStream_t s) {
  colsum_kernel<<<(cols + 127) / 128, 128, 0, s>>>(dz, rows, cols, out);
  return cudaGetLastError();
}
cudaError_t adam(float *w, const float *g, float *m, float *v, __nv_bfloat16 *wb, int n, float lr,
                 float b1, float b2, float eps, float c1, float c2, cudaStream_t s) {
  adam_kernel<<<(n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048, 256, 0, s>>>(w, g, m, v, wb, n, lr,
                                                                               b1, b2, eps, c1, c2);
  return cudaGetLastError();
}
cudaError_t to_bf16(const float *a, __nv_bfloat16 *b, int n, cudaStream_t s) {
  to_bf16_kernel<<<(n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048, 256, 0, s>>>(a, b, n);
  return cudaGetLastError();
}
cudaError_t feature_stats(const float *desc, int n, float *mu, float *inv_sd, cudaStream_t s) {
  feature_stats_kernel<<<256, 256, 0, s>>>(desc, n, mu, inv_sd);
  return cudaGetLastError();
}
cudaError_t label_stats(const float *y, int n, double *out, cudaStream_t s) {
  label_stats_kernel<<<1, 256, 0, s>>>(y, n, out);
  return cudaGetLastError();
}
cudaError_t unstd(float *y, int n, float mu, float sd, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  unstd_kernel<<<(n + 255) / 256, 256, 0, s>>>(y, n, mu, sd);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace ligate
