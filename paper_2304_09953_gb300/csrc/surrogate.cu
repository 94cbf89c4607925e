// Ligand descriptors and the triage surrogate network (paper Sec. 3.5:
// affinity prediction from ligand features, from cheap regressions up to
// deep networks chosen by cost).
#include <cuda_runtime.h>
#include <math.h>

#include "ligate_internal.h"

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

// --- surrogate network: see mlp kernels below -------------------------------
struct ligate_surrogate {
  int dummy;
};

extern "C" ligate_status ligate_surrogate_create(const float *, uint64_t, ligate_surrogate **out) {
  if (out) *out = nullptr;
  set_error("surrogate: not built yet");
  return LIGATE_ERR_UNSUPPORTED;
}
extern "C" void ligate_surrogate_destroy(ligate_surrogate *s) { delete s; }
extern "C" ligate_status ligate_surrogate_train(ligate_surrogate *, const float *, const float *, int,
                                                int, int, float, uint64_t, float *, void *) {
  set_error("surrogate: not built yet");
  return LIGATE_ERR_UNSUPPORTED;
}
extern "C" ligate_status ligate_surrogate_predict(const ligate_surrogate *, const float *, int, float *,
                                                  void *) {
  set_error("surrogate: not built yet");
  return LIGATE_ERR_UNSUPPORTED;
}
extern "C" ligate_status ligate_surrogate_rank(const ligate_surrogate *, const float *, int, double,
                                               int32_t *, float *, void *) {
  set_error("surrogate: not built yet");
  return LIGATE_ERR_UNSUPPORTED;
}
extern "C" ligate_status ligate_surrogate_grad(const ligate_surrogate *, const float *, const float *,
                                               int, float *, float *, void *) {
  set_error("surrogate: not built yet");
  return LIGATE_ERR_UNSUPPORTED;
}
extern "C" ligate_status ligate_surrogate_get_weights(const ligate_surrogate *, float *) {
  set_error("surrogate: not built yet");
  return LIGATE_ERR_UNSUPPORTED;
}
