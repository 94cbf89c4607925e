// Ligand descriptors and the triage surrogate network (paper Sec. 3.5:
// affinity prediction from ligand features, from cheap regressions up to
// deep networks chosen by cost).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ligate_internal.h"
#include "mlp.h"

namespace ligate {

// One warp per ligand: type counts, distinct-type-pair distance histograms
// (8 bins, edges (1.5 k) A, k = 1..7; the bin is decided on d^2 computed in
// FP32 as (dx*dx + dy*dy) + dz*dz without contraction, against the exactly
// representable squared edges), rotatable-bond count; log1p of every count.
__global__ void descriptor_kernel(const LigDesc *__restrict__ lig, const float4 *__restrict__ atoms,
                                  int n_ligands, float *__restrict__ out) {
  __shared__ unsigned int hist[8][28 * 8 + 8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int li = blockIdx.x * (blockDim.x >> 5) + warp;
  unsigned int *h = hist[warp];
  for (int q = lane; q < 28 * 8 + 8; q += 32) h[q] = 0;
  __syncwarp();
  if (li < n_ligands) {
    const LigDesc d = lig[li];
    const float4 *a = atoms + d.atom_base;
    for (int i = lane; i < d.n_atoms; i += 32) atomicAdd(&h[224 + __float_as_int(a[i].w)], 1u);
    const int npairs = d.n_atoms * (d.n_atoms - 1) / 2;
    for (int q = lane; q < npairs; q += 32) {
      // pair index q -> (i, j), i < j, row-major over the upper triangle
      int i = 0, rem = q, row = d.n_atoms - 1;
      while (rem >= row) { rem -= row; ++i; --row; }
      const int j = i + 1 + rem;
      const float4 x = a[i], y = a[j];
      int ta = __float_as_int(x.w), tb = __float_as_int(y.w);
      if (ta == tb) continue;
      if (ta > tb) { const int t = ta; ta = tb; tb = t; }
      const int p = ta * 8 - ta * (ta + 1) / 2 + (tb - ta - 1);
      const float dx = __fsub_rn(x.x, y.x), dy = __fsub_rn(x.y, y.y), dz = __fsub_rn(x.z, y.z);
      const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
      int bin = 0;
      bin += d2 >= 2.25f; bin += d2 >= 9.0f; bin += d2 >= 20.25f; bin += d2 >= 36.0f;
      bin += d2 >= 56.25f; bin += d2 >= 81.0f; bin += d2 >= 110.25f;
      atomicAdd(&h[p * 8 + bin], 1u);
    }
  }
  __syncwarp();
  if (li < n_ligands) {
    float *o = out + (size_t)li * 256;
    const int nrot = lig[li].n_rot;
    for (int q = lane; q < 256; q += 32) {
      float v = 0.f;
      if (q < 8) v = log1pf((float)h[224 + q]);
      else if (q < 232) v = log1pf((float)h[q - 8]);
      else if (q == 232) v = log1pf((float)nrot);
      o[q] = v;
    }
  }
}

}  // namespace ligate

using namespace ligate;


extern "C" ligate_status ligate_descriptors(const ligate_batch *b, float *out, void *stream) {
  if (!b || (!out && b->d.n_ligands)) { set_error("descriptors: NULL argument"); return LIGATE_ERR_INVALID; }
  if (b->d.n_ligands == 0) return LIGATE_OK;
  if (b->max_type >= 8) { set_error("descriptors: need atom types < 8"); return LIGATE_ERR_UNSUPPORTED; }
  const int wpb = 8;
  descriptor_kernel<<<(b->d.n_ligands + wpb - 1) / wpb, 32 * wpb, 0, (cudaStream_t)stream>>>(
      b->d.lig, b->d.atoms, b->d.n_ligands, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "descriptor kernel");
  return LIGATE_OK;
}

// ---------------------------------------------------------------------------
// Surrogate network object: FP32 master weights + Adam moments, BF16 copy
// for the tensor cores, standardisation statistics, activation workspace.
namespace {

constexpr int F0 = 256, F1 = 512;
// offsets of W1, b1, W2, b2, W3, b3, W4, b4 in the flat parameter vector
constexpr int OW1 = 0, OB1 = OW1 + F0 * F1, OW2 = OB1 + F1, OB2 = OW2 + F1 * F1, OW3 = OB2 + F1,
              OB3 = OW3 + F1 * F1, OW4 = OB3 + F1, OB4 = OW4 + F1, NPAR = OB4 + 1;
static_assert(NPAR == LIGATE_SURROGATE_PARAMS, "parameter count");

uint64_t sm64(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
double u01(uint64_t &s) { return (double)(sm64(s) >> 11) * 0x1.0p-53; }

}  // namespace

struct ligate_surrogate {
  float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
  __nv_bfloat16 *wb = nullptr;
  float *mu = nullptr, *inv_sd = nullptr;
  double *lstat = nullptr, *sse = nullptr;
  double label_mu = 0.0, label_sd = 1.0;
  bool stats = false;
  long long step = 0;
  int cap = 0;
  __nv_bfloat16 *x = nullptr, *h1 = nullptr, *h2 = nullptr, *h3 = nullptr;
  __nv_bfloat16 *dz1 = nullptr, *dz2 = nullptr, *dz3 = nullptr;
  float *t = nullptr, *y = nullptr, *dy = nullptr;
  int *idx = nullptr;
  int idx_cap = 0;
  // tcgen05 path: transposed BF16 hidden weights W1^T [512][256], W2^T,
  // W3^T [512][512] (K-major B operands of the forward layers) and the
  // timeout flag of its bounded waits
  bool tc05 = false;
  __nv_bfloat16 *wt = nullptr;
  int *err = nullptr;
};

namespace {

void free_work(ligate_surrogate *s) {
  cudaFree(s->x); cudaFree(s->h1); cudaFree(s->h2); cudaFree(s->h3);
  cudaFree(s->dz1); cudaFree(s->dz2); cudaFree(s->dz3);
  cudaFree(s->t); cudaFree(s->y); cudaFree(s->dy);
  s->x = s->h1 = s->h2 = s->h3 = s->dz1 = s->dz2 = s->dz3 = nullptr;
  s->t = s->y = s->dy = nullptr;
  s->cap = 0;
}

cudaError_t ensure_work(ligate_surrogate *s, int rows) {
  if (rows <= s->cap) return cudaSuccess;
  free_work(s);
  const size_t r = (size_t)rows;
  cudaError_t e;
  if ((e = cudaMalloc(&s->x, r * F0 * 2)) || (e = cudaMalloc(&s->h1, r * F1 * 2)) ||
      (e = cudaMalloc(&s->h2, r * F1 * 2)) || (e = cudaMalloc(&s->h3, r * F1 * 2)) ||
      (e = cudaMalloc(&s->dz1, r * F1 * 2)) || (e = cudaMalloc(&s->dz2, r * F1 * 2)) ||
      (e = cudaMalloc(&s->dz3, r * F1 * 2)) || (e = cudaMalloc(&s->t, r * 4)) ||
      (e = cudaMalloc(&s->y, r * 4)) || (e = cudaMalloc(&s->dy, r * 4))) {
    free_work(s);
    return e;
  }
  s->cap = rows;
  return cudaSuccess;
}

constexpr int TW1 = 0, TW2 = TW1 + F0 * F1, TW3 = TW2 + F1 * F1, NTW = TW3 + F1 * F1;

// Re-derive the transposed BF16 forward weights from the FP32 masters.
cudaError_t refresh_wt(ligate_surrogate *s, cudaStream_t st) {
  if (!s->tc05) return cudaSuccess;
  cudaError_t e;
  if ((e = mlp::transpose_bf16(s->w + OW1, F0, F1, s->wt + TW1, st))) return e;
  if ((e = mlp::transpose_bf16(s->w + OW2, F1, F1, s->wt + TW2, st))) return e;
  return mlp::transpose_bf16(s->w + OW3, F1, F1, s->wt + TW3, st);
}

// LIGATE_OK, or LIGATE_ERR_TIMEOUT once a tcgen05 wait ran out (flag
// cleared); synchronises st.
ligate_status check_err(ligate_surrogate *s, cudaStream_t st, const char *what) {
  if (!s->tc05) return LIGATE_OK;
  int h = 0;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(&h, s->err, 4, cudaMemcpyDeviceToHost, st)) || (e = cudaStreamSynchronize(st)))
    return cuda_fail(e, what);
  if (h) {
    cudaMemsetAsync(s->err, 0, 4, st);
    cudaStreamSynchronize(st);
    set_error("%s: a tensor-core pipeline wait ran out", what);
    return LIGATE_ERR_TIMEOUT;
  }
  return LIGATE_OK;
}

mlp::GemmArgs fwd_args(const __nv_bfloat16 *in, int fan_in, const __nv_bfloat16 *W, const float *b,
                       __nv_bfloat16 *out, int rows) {
  mlp::GemmArgs a{};
  a.A = in; a.B = W; a.M = rows; a.N = F1; a.K = fan_in;
  a.sAm = fan_in; a.sAk = 1; a.sBk = F1; a.sBn = 1;
  a.bias = b; a.Cb = out; a.ldc = F1;
  return a;
}

// Forward of the hidden layers on x (standardised BF16 rows).
cudaError_t forward_hidden(ligate_surrogate *s, int rows, cudaStream_t st) {
  cudaError_t e;
  if (s->tc05) {
    if ((e = mlp::gemm_tc05(mlp::EPI_BIAS_RELU, s->x, rows, F0, s->wt + TW1, F1, s->w + OB1, nullptr, s->h1,
                            s->err, st)) ||
        (e = mlp::gemm_tc05(mlp::EPI_BIAS_RELU, s->h1, rows, F1, s->wt + TW2, F1, s->w + OB2, nullptr, s->h2,
                            s->err, st)))
      return e;
    return mlp::gemm_tc05(mlp::EPI_BIAS_RELU, s->h2, rows, F1, s->wt + TW3, F1, s->w + OB3, nullptr, s->h3,
                          s->err, st);
  }
  if ((e = mlp::gemm(mlp::GEMM_FWD, fwd_args(s->x, F0, s->wb + OW1, s->w + OB1, s->h1, rows), st))) return e;
  if ((e = mlp::gemm(mlp::GEMM_FWD, fwd_args(s->h1, F1, s->wb + OW2, s->w + OB2, s->h2, rows), st))) return e;
  return mlp::gemm(mlp::GEMM_FWD, fwd_args(s->h2, F1, s->wb + OW3, s->w + OB3, s->h3, rows), st);
}

// Backward from dz3 (set by the head kernel) into s->g.
cudaError_t backward(ligate_surrogate *s, int rows, cudaStream_t st) {
  cudaError_t e;
  if ((e = mlp::head_grad(s->h3, s->dy, rows, s->g + OW4, s->g + OB4, st))) return e;
  struct L { const __nv_bfloat16 *in; int fan_in; int ow, ob; __nv_bfloat16 *dz, *dz_prev; const __nv_bfloat16 *hin; };
  const L layers[3] = {{s->h2, F1, OW3, OB3, s->dz3, s->dz2, s->h2},
                       {s->h1, F1, OW2, OB2, s->dz2, s->dz1, s->h1},
                       {s->x, F0, OW1, OB1, s->dz1, nullptr, nullptr}};
  for (const L &l : layers) {
    mlp::GemmArgs wg{};  // dW = in^T dZ
    wg.A = l.in; wg.B = l.dz; wg.M = l.fan_in; wg.N = F1; wg.K = rows;
    wg.sAm = 1; wg.sAk = l.fan_in; wg.sBk = F1; wg.sBn = 1;
    wg.Cf = s->g + l.ow; wg.ldc = F1;
    if ((e = mlp::gemm(mlp::GEMM_WGRAD, wg, st))) return e;
    if ((e = mlp::colsum(l.dz, rows, F1, s->g + l.ob, st))) return e;
    if (l.dz_prev) {  // dZ_prev = (dZ W^T) * (H_prev > 0)
      mlp::GemmArgs dg{};
      dg.A = l.dz; dg.B = s->wb + l.ow; dg.M = rows; dg.N = l.fan_in; dg.K = F1;
      dg.sAm = F1; dg.sAk = 1; dg.sBk = 1; dg.sBn = F1;
      dg.mask = l.hin; dg.Cb = l.dz_prev; dg.ldc = l.fan_in;
      if (s->tc05)  // B[n][k] = W[n][k]: the row-major weights are already K-major here
        e = mlp::gemm_tc05(mlp::EPI_RELU_MASK, l.dz, rows, F1, s->wb + l.ow, l.fan_in, nullptr, l.hin,
                           l.dz_prev, s->err, st);
      else
        e = mlp::gemm(mlp::GEMM_DGRAD, dg, st);
      if (e) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace

extern "C" ligate_status ligate_surrogate_create(const float *init, uint64_t seed, ligate_surrogate **out) {
  if (!out) { set_error("surrogate_create: out is NULL"); return LIGATE_ERR_INVALID; }
  *out = nullptr;
  std::vector<float> h(NPAR, 0.f);
  if (init) {
    for (int i = 0; i < NPAR; ++i)
      if (!isfinite(init[i])) { set_error("surrogate_create: non-finite weight %d", i); return LIGATE_ERR_INVALID; }
    std::copy(init, init + NPAR, h.begin());
  } else {  // He-normal weights (Box-Muller over SplitMix64), zero biases
    uint64_t st = seed ^ 0x5851F42D4C957F2DULL;
    auto fill = [&](int off, int fan_in, int count) {
      const double sd = sqrt(2.0 / fan_in);
      for (int i = 0; i < count; i += 2) {
        double a = u01(st), b = u01(st);
        if (a < 1e-300) a = 1e-300;
        const double r = sqrt(-2.0 * log(a));
        h[off + i] = (float)(sd * r * cos(6.283185307179586 * b));
        if (i + 1 < count) h[off + i + 1] = (float)(sd * r * sin(6.283185307179586 * b));
      }
    };
    fill(OW1, F0, F0 * F1);
    fill(OW2, F1, F1 * F1);
    fill(OW3, F1, F1 * F1);
    fill(OW4, F1, F1);
  }
  ligate_surrogate *s = new ligate_surrogate();
  cudaError_t e;
  if ((e = cudaMalloc(&s->w, NPAR * 4)) || (e = cudaMalloc(&s->m, NPAR * 4)) ||
      (e = cudaMalloc(&s->v, NPAR * 4)) || (e = cudaMalloc(&s->g, NPAR * 4)) ||
      (e = cudaMalloc(&s->wb, NPAR * 2)) || (e = cudaMalloc(&s->mu, F0 * 4)) ||
      (e = cudaMalloc(&s->inv_sd, F0 * 4)) || (e = cudaMalloc(&s->lstat, 16)) ||
      (e = cudaMalloc(&s->sse, 8)) || (e = cudaMemcpy(s->w, h.data(), NPAR * 4, cudaMemcpyHostToDevice)) ||
      (e = cudaMemset(s->m, 0, NPAR * 4)) || (e = cudaMemset(s->v, 0, NPAR * 4)) ||
      (e = cudaMemset(s->g, 0, NPAR * 4)) || (e = mlp::to_bf16(s->w, s->wb, NPAR, 0)) ||
      (e = cudaDeviceSynchronize())) {
    ligate_surrogate_destroy(s);
    return cuda_fail(e, "surrogate_create");
  }
  // K-major contractions on tcgen05 unless LIGATE_MLP_GEMM=mma selects the
  // mma.sync kernels (same operands and rounding points; used to compare)
  const char *sel = getenv("LIGATE_MLP_GEMM");
  s->tc05 = !(sel && strcmp(sel, "mma") == 0) && mlp::tc05_supported(1, F1, F0);
  if (s->tc05 &&
      ((e = cudaMalloc(&s->wt, (size_t)NTW * 2)) || (e = cudaMalloc(&s->err, 4)) ||
       (e = cudaMemset(s->err, 0, 4)) || (e = refresh_wt(s, 0)) || (e = cudaDeviceSynchronize()))) {
    ligate_surrogate_destroy(s);
    return cuda_fail(e, "surrogate_create");
  }
  std::vector<float> mu(F0, 0.f), one(F0, 1.f);
  cudaMemcpy(s->mu, mu.data(), F0 * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(s->inv_sd, one.data(), F0 * 4, cudaMemcpyHostToDevice);
  *out = s;
  return LIGATE_OK;
}

extern "C" void ligate_surrogate_destroy(ligate_surrogate *s) {
  if (!s) return;
  free_work(s);
  cudaFree(s->w); cudaFree(s->m); cudaFree(s->v); cudaFree(s->g); cudaFree(s->wb);
  cudaFree(s->mu); cudaFree(s->inv_sd); cudaFree(s->lstat); cudaFree(s->sse); cudaFree(s->idx);
  cudaFree(s->wt); cudaFree(s->err);
  delete s;
}

extern "C" ligate_status ligate_surrogate_train(ligate_surrogate *s, const float *desc,
                                                const float *labels, int n, int epochs, int batch,
                                                float lr, uint64_t seed, float *loss_out, void *stream) {
  NvtxRange nvtx_("ligate:surrogate_train");
  if (!s || !desc || !labels) { set_error("surrogate_train: NULL argument"); return LIGATE_ERR_INVALID; }
  if (n < 1 || batch < 8 || batch % 8 != 0 || batch > n || epochs < 0 || !(lr > 0)) {
    set_error("surrogate_train: need 8 <= batch <= n, batch % 8 == 0, epochs >= 0, lr > 0");
    return LIGATE_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (!s->stats) {
    if ((e = mlp::feature_stats(desc, n, s->mu, s->inv_sd, st)) || (e = mlp::label_stats(labels, n, s->lstat, st)))
      return cuda_fail(e, "surrogate statistics");
    double ls[2];
    if ((e = cudaMemcpyAsync(ls, s->lstat, 16, cudaMemcpyDeviceToHost, st)) || (e = cudaStreamSynchronize(st)))
      return cuda_fail(e, "surrogate statistics");
    s->label_mu = ls[0];
    s->label_sd = ls[1] > 1e-12 ? ls[1] : 1.0;
    s->stats = true;
  }
  if ((e = ensure_work(s, batch))) return cuda_fail(e, "surrogate workspace");
  if (s->idx_cap < n) {
    cudaFree(s->idx);
    s->idx = nullptr;
    s->idx_cap = 0;
    if ((e = cudaMalloc(&s->idx, (size_t)n * 4))) return cuda_fail(e, "surrogate workspace");
    s->idx_cap = n;
  }
  const int steps = n / batch;
  std::vector<int> perm(n);
  const float ly_inv = (float)(1.0 / s->label_sd);
  double last = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    uint64_t rs = seed * 0x9E3779B97F4A7C15ULL + (uint64_t)ep + 1;
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int i = n - 1; i > 0; --i) {  // Fisher-Yates
      const int j = (int)(u01(rs) * (i + 1));
      std::swap(perm[i], perm[j < i + 1 ? j : i]);
    }
    if ((e = cudaMemcpyAsync(s->idx, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemsetAsync(s->sse, 0, 8, st)))
      return cuda_fail(e, "surrogate epoch");
    for (int k = 0; k < steps; ++k) {
      ++s->step;
      const double c1 = 1.0 / (1.0 - pow(0.9, (double)s->step));
      const double c2 = 1.0 / (1.0 - pow(0.999, (double)s->step));
      if ((e = mlp::gather_std(desc, s->idx + (size_t)k * batch, batch, 0, s->mu, s->inv_sd, labels,
                               (float)s->label_mu, ly_inv, s->x, s->t, st)) ||
          (e = forward_hidden(s, batch, st)) ||
          (e = mlp::head(s->h3, s->wb + OW4, s->w + OB4, batch, s->t, s->y, s->dy, 2.f / batch,
                         s->sse, s->dz3, st)) ||
          (e = backward(s, batch, st)) ||
          (e = mlp::adam(s->w, s->g, s->m, s->v, s->wb, NPAR, lr, 0.9f, 0.999f, 1e-8f, (float)c1,
                         (float)c2, st)) ||
          (e = refresh_wt(s, st)))
        return cuda_fail(e, "surrogate step");
    }
    double sse = 0.0;
    if ((e = cudaMemcpyAsync(&sse, s->sse, 8, cudaMemcpyDeviceToHost, st)) || (e = cudaStreamSynchronize(st)))
      return cuda_fail(e, "surrogate epoch");
    if (ligate_status r = check_err(s, st, "surrogate epoch")) return r;
    last = steps > 0 ? sse / ((double)steps * batch) : 0.0;
  }
  if (loss_out) *loss_out = (float)last;
  return LIGATE_OK;
}

extern "C" ligate_status ligate_surrogate_grad(const ligate_surrogate *cs, const float *x, const float *t,
                                               int b, float *grad, float *loss_out, void *stream) {
  ligate_surrogate *s = const_cast<ligate_surrogate *>(cs);
  if (!s || !x || !t || !grad) { set_error("surrogate_grad: NULL argument"); return LIGATE_ERR_INVALID; }
  if (b < 1) { set_error("surrogate_grad: b < 1"); return LIGATE_ERR_INVALID; }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = ensure_work(s, b))) return cuda_fail(e, "surrogate workspace");
  double sse = 0.0;
  if ((e = mlp::to_bf16(x, s->x, b * F0, st)) ||
      (e = cudaMemcpyAsync(s->t, t, (size_t)b * 4, cudaMemcpyDeviceToDevice, st)) ||
      (e = cudaMemsetAsync(s->sse, 0, 8, st)) || (e = forward_hidden(s, b, st)) ||
      (e = mlp::head(s->h3, s->wb + OW4, s->w + OB4, b, s->t, s->y, s->dy, 2.f / b, s->sse, s->dz3, st)) ||
      (e = backward(s, b, st)) ||
      (e = cudaMemcpyAsync(grad, s->g, NPAR * 4, cudaMemcpyDeviceToDevice, st)) ||
      (e = cudaMemcpyAsync(&sse, s->sse, 8, cudaMemcpyDeviceToHost, st)) || (e = cudaStreamSynchronize(st)))
    return cuda_fail(e, "surrogate_grad");
  if (ligate_status r = check_err(s, st, "surrogate_grad")) return r;
  if (loss_out) *loss_out = (float)(sse / b);
  return LIGATE_OK;
}

extern "C" ligate_status ligate_surrogate_predict(const ligate_surrogate *cs, const float *desc, int n,
                                                  float *pred, void *stream) {
  NvtxRange nvtx_("ligate:surrogate_predict");
  ligate_surrogate *s = const_cast<ligate_surrogate *>(cs);
  if (!s || (n > 0 && (!desc || !pred)) || n < 0) { set_error("surrogate_predict: bad argument"); return LIGATE_ERR_INVALID; }
  cudaStream_t st = (cudaStream_t)stream;
  const int chunk = 32768;
  cudaError_t e;
  if ((e = ensure_work(s, n < chunk ? (n > 0 ? n : 1) : chunk))) return cuda_fail(e, "surrogate workspace");
  for (int r0 = 0; r0 < n; r0 += chunk) {
    const int rows = n - r0 < chunk ? n - r0 : chunk;
    if ((e = mlp::gather_std(desc, nullptr, rows, r0, s->mu, s->inv_sd, nullptr, 0.f, 0.f, s->x, nullptr, st)) ||
        (e = forward_hidden(s, rows, st)) ||
        (e = mlp::head(s->h3, s->wb + OW4, s->w + OB4, rows, nullptr, pred + r0, nullptr, 0.f, nullptr,
                       nullptr, st)) ||
        (e = mlp::unstd(pred + r0, rows, (float)s->label_mu, (float)s->label_sd, st)))
      return cuda_fail(e, "surrogate_predict");
  }
  return check_err(s, st, "surrogate_predict");
}

extern "C" ligate_status ligate_surrogate_rank(const ligate_surrogate *s, const float *desc, int n,
                                               double keep_frac, int32_t *idx_out, float *pred_out,
                                               void *stream) {
  NvtxRange nvtx_("ligate:surrogate_rank");
  if (!s || n < 0 || !(keep_frac >= 0.0 && keep_frac <= 1.0) || (n > 0 && (!desc || !idx_out))) {
    set_error("surrogate_rank: bad argument");
    return LIGATE_ERR_INVALID;
  }
  if (n == 0) return LIGATE_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int k = (int)ceil((double)n * keep_frac - 1e-9);
  int n2 = 2048;
  while (n2 < n) n2 <<= 1;
  float *pred = pred_out;
  unsigned long long *keys = nullptr;
  cudaError_t e = cudaSuccess;
  if (!pred && (e = cudaMalloc(&pred, (size_t)n * 4))) return cuda_fail(e, "surrogate_rank");
  if ((e = cudaMalloc(&keys, (size_t)n2 * 8))) {
    if (!pred_out) cudaFree(pred);
    return cuda_fail(e, "surrogate_rank");
  }
  ligate_status r = ligate_surrogate_predict(s, desc, n, pred, stream);
  if (r == LIGATE_OK) {
    e = mlp::sort_select(pred, n, k, keys, n2, idx_out, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) r = cuda_fail(e, "surrogate_rank");
  }
  cudaFree(keys);
  if (!pred_out) cudaFree(pred);
  return r;
}

namespace {
__global__ void axpy_kernel(float *__restrict__ acc, const float *__restrict__ x, int n, float a, int first) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) acc[i] = first ? a * x[i] : fmaf(a, x[i], acc[i]);
}
}  // namespace

extern "C" ligate_status ligate_surrogate_rank_ensemble(const ligate_surrogate *const *nets, int n_nets,
                                                        const float *desc, int n, double keep_frac,
                                                        int32_t *idx_out, float *pred_out, void *stream) {
  NvtxRange nvtx_("ligate:surrogate_rank_ensemble");
  if (!nets || n_nets < 1 || n < 0 || !(keep_frac >= 0.0 && keep_frac <= 1.0) || (n > 0 && (!desc || !idx_out))) {
    set_error("surrogate_rank_ensemble: bad argument");
    return LIGATE_ERR_INVALID;
  }
  for (int m = 0; m < n_nets; ++m)
    if (!nets[m]) { set_error("surrogate_rank_ensemble: network %d is NULL", m); return LIGATE_ERR_INVALID; }
  if (n == 0) return LIGATE_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int k = (int)ceil((double)n * keep_frac - 1e-9);
  int n2 = 2048;
  while (n2 < n) n2 <<= 1;
  float *mean = pred_out, *one = nullptr;
  unsigned long long *keys = nullptr;
  cudaError_t e = cudaSuccess;
  ligate_status r = LIGATE_OK;
  if ((!pred_out && (e = cudaMalloc(&mean, (size_t)n * 4))) || (e = cudaMalloc(&one, (size_t)n * 4)) ||
      (e = cudaMalloc(&keys, (size_t)n2 * 8))) {
    r = cuda_fail(e, "surrogate_rank_ensemble");
  }
  // mean = sum_m (1 / n_nets) pred_m, accumulated in network order
  for (int m = 0; m < n_nets && r == LIGATE_OK; ++m) {
    r = ligate_surrogate_predict(nets[m], desc, n, one, stream);
    if (r != LIGATE_OK) break;
    axpy_kernel<<<(n + 255) / 256, 256, 0, st>>>(mean, one, n, 1.f / (float)n_nets, m == 0);
    if ((e = cudaGetLastError()) != cudaSuccess) r = cuda_fail(e, "surrogate_rank_ensemble");
  }
  if (r == LIGATE_OK) {
    e = mlp::sort_select(mean, n, k, keys, n2, idx_out, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) r = cuda_fail(e, "surrogate_rank_ensemble");
  }
  cudaFree(keys);
  cudaFree(one);
  if (!pred_out) cudaFree(mean);
  return r;
}

extern "C" ligate_status ligate_surrogate_get_weights(const ligate_surrogate *s, float *out) {
  if (!s || !out) { set_error("surrogate_get_weights: NULL argument"); return LIGATE_ERR_INVALID; }
  cudaError_t e = cudaMemcpy(out, s->w, NPAR * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "surrogate_get_weights");
  return LIGATE_OK;
}

extern "C" int ligate_surrogate_engine(const ligate_surrogate *s) { return s ? (s->tc05 ? 1 : 0) : -1; }

extern "C" ligate_status ligate_debug_inject_fault(int kind) {
  if (kind != 1) { set_error("debug_inject_fault: unknown kind %d", kind); return LIGATE_ERR_INVALID; }
  cudaError_t e = mlp::inject_skip_loads_once();
  if (e != cudaSuccess) return cuda_fail(e, "debug_inject_fault");
  return LIGATE_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint: a little-endian binary file: 8-byte magic "LGSURR01", int32
// parameter count, int32 feature count, int64 Adam step, FP64 label mean and
// standard deviation, int32 statistics flag, then FP32 arrays: weights,
// Adam first and second moments (parameter count each), feature means and
// inverse standard deviations (feature count each).
namespace {
const char kMagic[8] = {'L', 'G', 'S', 'U', 'R', 'R', '0', '1'};
}

extern "C" ligate_status ligate_surrogate_save(const ligate_surrogate *s, const char *path) {
  if (!s || !path) { set_error("surrogate_save: NULL argument"); return LIGATE_ERR_INVALID; }
  std::vector<float> buf((size_t)3 * NPAR + 2 * F0);
  cudaError_t e;
  if ((e = cudaMemcpy(buf.data(), s->w, (size_t)NPAR * 4, cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(buf.data() + NPAR, s->m, (size_t)NPAR * 4, cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(buf.data() + 2 * (size_t)NPAR, s->v, (size_t)NPAR * 4, cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(buf.data() + 3 * (size_t)NPAR, s->mu, (size_t)F0 * 4, cudaMemcpyDeviceToHost)) ||
      (e = cudaMemcpy(buf.data() + 3 * (size_t)NPAR + F0, s->inv_sd, (size_t)F0 * 4, cudaMemcpyDeviceToHost)))
    return cuda_fail(e, "surrogate_save");
  FILE *f = fopen(path, "wb");
  if (!f) { set_error("surrogate_save: cannot open %s", path); return LIGATE_ERR_INVALID; }
  const int32_t np = NPAR, nf = F0, st = s->stats ? 1 : 0;
  const int64_t step = s->step;
  bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(&np, 4, 1, f) == 1 && fwrite(&nf, 4, 1, f) == 1 &&
            fwrite(&step, 8, 1, f) == 1 && fwrite(&s->label_mu, 8, 1, f) == 1 &&
            fwrite(&s->label_sd, 8, 1, f) == 1 && fwrite(&st, 4, 1, f) == 1 &&
            fwrite(buf.data(), 4, buf.size(), f) == buf.size();
  ok = (fclose(f) == 0) && ok;
  if (!ok) { set_error("surrogate_save: write to %s failed", path); return LIGATE_ERR_INVALID; }
  return LIGATE_OK;
}

extern "C" ligate_status ligate_surrogate_load(const char *path, ligate_surrogate **out) {
  if (!path || !out) { set_error("surrogate_load: NULL argument"); return LIGATE_ERR_INVALID; }
  *out = nullptr;
  FILE *f = fopen(path, "rb");
  if (!f) { set_error("surrogate_load: cannot open %s", path); return LIGATE_ERR_INVALID; }
  char magic[8];
  int32_t np = 0, nf = 0, st = 0;
  int64_t step = 0;
  double lmu = 0, lsd = 1;
  std::vector<float> buf((size_t)3 * NPAR + 2 * F0);
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMagic, 8) == 0 && fread(&np, 4, 1, f) == 1 &&
            fread(&nf, 4, 1, f) == 1 && np == NPAR && nf == F0 && fread(&step, 8, 1, f) == 1 &&
            fread(&lmu, 8, 1, f) == 1 && fread(&lsd, 8, 1, f) == 1 && fread(&st, 4, 1, f) == 1 &&
            fread(buf.data(), 4, buf.size(), f) == buf.size();
  fclose(f);
  if (!ok || step < 0 || !std::isfinite(lmu) || !(lsd > 0)) {
    set_error("surrogate_load: %s is not a surrogate checkpoint of this network", path);
    return LIGATE_ERR_INVALID;
  }
  for (float x : buf)
    if (!std::isfinite(x)) { set_error("surrogate_load: non-finite value in %s", path); return LIGATE_ERR_INVALID; }
  ligate_surrogate *s = nullptr;
  ligate_status r = ligate_surrogate_create(buf.data(), 0, &s);
  if (r != LIGATE_OK) return r;
  cudaError_t e;
  if ((e = cudaMemcpy(s->m, buf.data() + NPAR, (size_t)NPAR * 4, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(s->v, buf.data() + 2 * (size_t)NPAR, (size_t)NPAR * 4, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(s->mu, buf.data() + 3 * (size_t)NPAR, (size_t)F0 * 4, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(s->inv_sd, buf.data() + 3 * (size_t)NPAR + F0, (size_t)F0 * 4, cudaMemcpyHostToDevice))) {
    ligate_surrogate_destroy(s);
    return cuda_fail(e, "surrogate_load");
  }
  s->step = step;
  s->label_mu = lmu;
  s->label_sd = lsd;
  s->stats = st != 0;
  *out = s;
  return LIGATE_OK;
}

