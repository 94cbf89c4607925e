// Kernels of the triage surrogate network (mlp.cu), used by surrogate.cu.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ligate {
namespace mlp {

enum { EPI_BIAS_RELU = 0, EPI_RELU_MASK = 1, EPI_F32 = 2 };
enum { GEMM_FWD = 0, GEMM_DGRAD = 1, GEMM_WGRAD = 2 };

struct GemmArgs {
  const __nv_bfloat16 *A, *B;
  int M, N, K;
  long long sAm, sAk, sBk, sBn;  // element strides (the contiguous one is 1)
  const float *bias;             // EPI_BIAS_RELU
  const __nv_bfloat16 *mask;     // EPI_RELU_MASK: ReLU output of the forward layer
  __nv_bfloat16 *Cb;             // BF16 output
  float *Cf;                     // FP32 output
  int ldc;
};

cudaError_t gemm(int kind, const GemmArgs &g, cudaStream_t s);
cudaError_t gather_std(const float *desc, const int *idx, int rows, int row0, const float *mu,
                       const float *inv_sd, const float *labels, float ly_mu, float ly_inv,
                       __nv_bfloat16 *x, float *t, cudaStream_t s);
cudaError_t head(const __nv_bfloat16 *h3, const __nv_bfloat16 *w4, const float *b4, int rows,
                 const float *t, float *y, float *dy, float inv_b2, double *sse, __nv_bfloat16 *dz3,
                 cudaStream_t s);
cudaError_t head_grad(const __nv_bfloat16 *h3, const float *dy, int rows, float *gw4, float *gb4,
                      cudaStream_t s);
cudaError_t colsum(const __nv_bfloat16 *dz, int rows, int cols, float *out, cudaStream_t s);
cudaError_t adam(float *w, const float *g, float *m, float *v, __nv_bfloat16 *wb, int n, float lr,
                 float b1, float b2, float eps, float c1, float c2, cudaStream_t s);
cudaError_t to_bf16(const float *a, __nv_bfloat16 *b, int n, cudaStream_t s);
cudaError_t feature_stats(const float *desc, int n, float *mu, float *inv_sd, cudaStream_t s);
cudaError_t label_stats(const float *y, int n, double *out, cudaStream_t s);
cudaError_t unstd(float *y, int n, float mu, float sd, cudaStream_t s);
cudaError_t sort_select(const float *pred, int n, int k, unsigned long long *keys, int n2,
                        int32_t *idx, cudaStream_t s);

// tcgen05 path (mlp_tc05.cu) for K-major A [M][K] and B [N][K]:
// C[M][N] = epi(A B^T), epi EPI_BIAS_RELU or EPI_RELU_MASK; needs N % 256 == 0,
// K % 64 == 0, 16-byte aligned pointers.  *err is set to 1 when a bounded
// wait ran out (results then undefined).
bool tc05_supported(int M, int N, int K);
cudaError_t gemm_tc05(int epi, const __nv_bfloat16 *a, int M, int K, const __nv_bfloat16 *b, int N,
                      const float *bias, const __nv_bfloat16 *mask, __nv_bfloat16 *out, int *err,
                      cudaStream_t s);
// Test hook: the next CTA of a tcgen05 contraction issues no loads, so its
// bounded wait runs out (err set, LIGATE_ERR_TIMEOUT at the next check).
cudaError_t inject_skip_loads_once();
// wt[n][k] = bf16(w[k][n]) for row-major FP32 w [K][N].
cudaError_t transpose_bf16(const float *w, int K, int N, __nv_bfloat16 *wt, cudaStream_t s);

}  // namespace mlp
}  // namespace ligate
