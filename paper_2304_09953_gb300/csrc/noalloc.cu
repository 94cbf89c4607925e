// Allocation-free docking entry point (ligate_dock_noalloc).
//
// Some callers cannot call cudaMalloc: a serving process that reserves all
// device memory for its own pool at start-up, or a latency-bound loop where
// cudaMalloc's implicit device synchronisation is not acceptable.  This entry
// point runs the same docking kernel as ligate_plan_run but keeps every piece
// of scratch (start frames, work items, per-ligand counters, partial top-K
// lists) in one file-scope device array of fixed size, so a call allocates
// nothing on the device or on the host heap.  The pocket, the batch and the
// output buffer are the caller's.
//
// The array is reserved on a device when this file's device code is loaded
// there: under CUDA's default lazy module loading that is the first call of
// this entry point on the device (its address look-up), so a caller that
// reserves the rest of the device for its own pool makes one call first (or
// runs with CUDA_MODULE_LOADING=EAGER).  From then on it stays until the
// process exits.  All calls share it and it keeps the previous call's
// contents; the counters that must start at zero are cleared at the start of
// each call, and two calls whose GPU work overlaps (different streams, or
// different host threads on one device) race on it.  The orientations reach
// the device inside the launches' parameters, not through a host buffer.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "dock_device.cuh"

namespace ligate {
namespace {

constexpr size_t kScratchBytes = (size_t)8 << 20;  // LIGATE_NOALLOC_SCRATCH_BYTES
constexpr int kMaxOrient = 1024, kMaxAnchor = 1024;
constexpr int kChunk = 1024;   // starts per work item
constexpr int kMaxDevices = 64;
constexpr int kQuatBlock = 240;  // quaternions per launch: the parameters stay under 4 KB

static_assert(kScratchBytes == LIGATE_NOALLOC_SCRATCH_BYTES, "scratch size");

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch for each device (host code must not use the
// symbol itself: on the host it names a stand-in, not device memory).
unsigned char *g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Orientations passed by value (copied into the launch's parameters, so no
// host buffer has to outlive the call): start frames of orientations
// first .. first + count - 1 (the same arithmetic as the planned path), and
// with first == 0 the anchors in grid units.
struct QuatBlock {
  float4 q[kQuatBlock];
};

__global__ void noalloc_frames_kernel(const QuatBlock blk, int first, int count, const float *__restrict__ anchors,
                                      int n_anchor, float ox, float oy, float oz, float inv_h,
                                      float *__restrict__ rot, float *__restrict__ anc) {
  const int i = threadIdx.x;
  if (i < count) quat_frame(blk.q[i], inv_h, rot + 9 * (first + i));
  if (first == 0)
    for (int a = i; a < n_anchor; a += blockDim.x) {
      anc[3 * a] = (anchors[3 * a] - ox) * inv_h;
      anc[3 * a + 1] = (anchors[3 * a + 1] - oy) * inv_h;
      anc[3 * a + 2] = (anchors[3 * a + 2] - oz) * inv_h;
    }
}

// Work items (ligand, start range, partial-list slot), computed in place.
__global__ void noalloc_items_kernel(Item *__restrict__ items, int *__restrict__ lig_items,
                                     int *__restrict__ lig_slot0, int n_ligands, int n_starts,
                                     int chunk, int per_lig) {
  const long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (it < (long long)n_ligands * per_lig) {
    const int li = (int)(it / per_lig), c = (int)(it % per_lig);
    Item m;
    m.ligand = li;
    m.row = li;
    m.pad[0] = m.pad[1] = m.pad[2] = 0;
    m.s0 = c * chunk;
    m.s1 = min(n_starts, (c + 1) * chunk);
    m.slot = (int)it;
    items[it] = m;
  }
  if (it < n_ligands) {
    lig_items[it] = per_lig;
    lig_slot0[it] = (int)it * per_lig;
  }
}

int pow2ceil(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

}  // namespace
}  // namespace ligate

using namespace ligate;

extern "C" ligate_status ligate_dock_noalloc(const ligate_pocket *P, const ligate_batch *B,
                                             const ligate_sampling *s, ligate_pose *out,
                                             void *stream) {
  if (!P || !B || !s || (!out && B->d.n_ligands > 0)) {
    set_error("dock_noalloc: NULL pocket, batch, sampling or output");
    return LIGATE_ERR_INVALID;
  }
  const PocketDev &pk = P->d;
  const BatchDev &bt = B->d;
  if (s->n_orient < 1 || s->n_orient > kMaxOrient || s->n_anchor < 1 || s->n_anchor > kMaxAnchor ||
      s->n_anchor > pk.n_anchors || !s->orientations) {
    set_error("dock_noalloc: need 1..%d orientations and 1..min(%d, pocket anchors) anchors",
              kMaxOrient, kMaxAnchor);
    return LIGATE_ERR_UNSUPPORTED;
  }
  if (s->torsion_steps < 1 || s->torsion_steps > LIGATE_MAX_STEPS || s->top_k < 1 ||
      s->top_k > LIGATE_MAX_TOPK) {
    set_error("dock_noalloc: torsion_steps or top_k outside the library limits");
    return LIGATE_ERR_UNSUPPORTED;
  }
  if (!(s->clash_cutoff > 0) || !isfinite(s->clash_weight) || !isfinite(s->penalty)) {
    set_error("dock_noalloc: clash_cutoff must be > 0, weight and penalty finite");
    return LIGATE_ERR_INVALID;
  }
  if (bt.n_ligands > 0 && B->max_type >= pk.n_types) {
    set_error("dock_noalloc: batch uses atom type %d but the pocket has %d maps", B->max_type, pk.n_types);
    return LIGATE_ERR_INVALID;
  }
  int mode;
  const void *maps;
  if (s->precision == LIGATE_FP32 && s->layout == LIGATE_LAYOUT_PLAIN) { mode = MODE_F32_PLAIN; maps = pk.map_f32; }
  else if (s->precision == LIGATE_FP32 && s->layout == LIGATE_LAYOUT_CORNER) { mode = MODE_F32_CORNER; maps = pk.map_f32c; }
  else if (s->precision == LIGATE_BF16 && s->layout == LIGATE_LAYOUT_CORNER) { mode = MODE_BF16_CORNER; maps = pk.map_bf16c; }
  else if (s->precision == LIGATE_FP16 && s->layout == LIGATE_LAYOUT_CORNER) { mode = MODE_F16_CORNER; maps = pk.map_f16c; }
  else { set_error("dock_noalloc: unsupported precision/layout pair"); return LIGATE_ERR_UNSUPPORTED; }
  if (!maps) {
    set_error("dock_noalloc: the pocket was created without this map precision/layout");
    return LIGATE_ERR_UNSUPPORTED;
  }
  // quaternions checked before any device work
  for (int i = 0; i < 4 * s->n_orient; ++i)
    if (!isfinite(s->orientations[i])) { set_error("dock_noalloc: non-finite quaternion"); return LIGATE_ERR_INVALID; }
  const int n = bt.n_ligands;
  if (n == 0) return LIGATE_OK;

  // scratch layout and size check
  const int n_starts = s->n_orient * s->n_anchor;
  const int L = pow2ceil(s->torsion_steps), G = 32 / L;
  const int chunk = std::max(G, kChunk / G * G);
  const int per_lig = (n_starts + chunk - 1) / chunk;
  const long long n_items = (long long)n * per_lig;
  const int K = s->top_k;
  size_t off = 0;
  const size_t o_rot = off;  off = align256(off + sizeof(float) * 9 * kMaxOrient);
  const size_t o_anc = off;  off = align256(off + sizeof(float) * 3 * kMaxAnchor);
  const size_t o_cnt = off;  off = align256(off + sizeof(int) * ((size_t)n + 1));
  const size_t o_lit = off;  off = align256(off + sizeof(int) * (size_t)n);
  const size_t o_ls0 = off;  off = align256(off + sizeof(int) * (size_t)n);
  const size_t o_itm = off;  off = align256(off + sizeof(Item) * (size_t)n_items);
  const size_t o_par = off;  off = align256(off + sizeof(PoseOut) * (size_t)n_items * K);
  if (off > kScratchBytes) {
    set_error("dock_noalloc: %d ligands x %d starts x top-%d need %zu B of scratch; the "
              "allocation-free entry point has %zu B (split the batch or use ligate_plan_run)",
              n, n_starts, K, off, kScratchBytes);
    return LIGATE_ERR_UNSUPPORTED;
  }

  // set-up, once per device, with that device current
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "dock_noalloc");
  if (dev < 0 || dev >= kMaxDevices) { set_error("dock_noalloc: device index %d too large", dev); return LIGATE_ERR_UNSUPPORTED; }
  unsigned char *base;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
      void *ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "dock_noalloc: scratch address");
      g_scratch_ptr[dev] = (unsigned char *)ptr;
    }
    base = g_scratch_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;

  DockParams p;
  memset(&p, 0, sizeof(p));
  p.lig = bt.lig; p.atoms = bt.atoms; p.bonds = bt.bonds; p.elig = bt.elig; p.cand = bt.cand;
  p.n_ligands = n;
  p.maps = maps;
  p.maps_f32 = pk.map_f32;
  p.g.nx = pk.nx; p.g.ny = pk.ny; p.g.nz = pk.nz;
  p.g.fx1 = (float)(pk.nx - 1); p.g.fy1 = (float)(pk.ny - 1); p.g.fz1 = (float)(pk.nz - 1);
  p.g.penalty = s->penalty;
  p.g.cx = 8388608.f + (float)(pk.nx - 2); p.g.cy = 8388608.f + (float)(pk.ny - 2); p.g.cz = 8388608.f + (float)(pk.nz - 2);
  set_map_minima(p, pk, mode);
  p.rot = (const float *)(base + o_rot);
  p.anc = (const float *)(base + o_anc);
  p.n_anchor = s->n_anchor;
  p.n_starts = n_starts;
  p.S = s->torsion_steps; p.L = L; p.G = G; p.K = K;
  fill_step_table(p.S, p.cs_tab);
  p.clash_w = s->clash_weight;
  const double dc2 = (double)s->clash_cutoff * s->clash_cutoff, h2 = pk.spacing * pk.spacing;
  p.inv_dc2_ang = (float)(1.0 / dc2);
  p.inv_dc2_grid = (float)(h2 / dc2);
  p.dc2_grid_margin = (float)(dc2 / h2 * (1.0 + 1e-4));
  p.stats = nullptr;
  p.rescore = s->rescore_fp32 ? 1 : 0;
  p.items = (const Item *)(base + o_itm);
  p.n_items = (int)n_items;
  p.lig_items = (const int *)(base + o_lit);
  p.lig_slot0 = (const int *)(base + o_ls0);
  p.queue = (int *)(base + o_cnt);
  p.done = (int *)(base + o_cnt) + 1;
  p.partial = (PoseOut *)(base + o_par);
  p.out = reinterpret_cast<PoseOut *>(out);
  p.nmax = std::max(32, (bt.max_atoms + 31) / 32 * 32);
  p.wmax = p.nmax / 32;
  p.rmax = bt.max_rot;

  // launch shape: 4 warps per CTA (fewer if shared memory is short), all SMs
  const size_t per_warp = dock_smem_per_warp(p.nmax, p.S, G, p.rmax);
  const int warps = (int)std::min<size_t>(4, std::max<size_t>(1, (size_t)(227 * 1024) / per_warp));
  const size_t smem = per_warp * warps;
  const int occ = dock_kernel_max_ctas_per_sm(mode, 0, 32 * warps, smem);
  if (occ < 1) { set_error("dock_noalloc: kernel cannot be resident"); return LIGATE_ERR_UNSUPPORTED; }
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_fail(e, "dock_noalloc");

  for (int first = 0; first < s->n_orient; first += kQuatBlock) {
    QuatBlock blk;
    const int count = std::min(kQuatBlock, s->n_orient - first);
    for (int q = 0; q < count; ++q) {
      const double *o = s->orientations + 4 * (size_t)(first + q);
      blk.q[q] = make_float4((float)o[0], (float)o[1], (float)o[2], (float)o[3]);
    }
    noalloc_frames_kernel<<<1, 256, 0, st>>>(blk, first, count, pk.anchors, s->n_anchor, (float)pk.origin[0],
                                              (float)pk.origin[1], (float)pk.origin[2], (float)(1.0 / pk.spacing),
                                              (float *)(base + o_rot), (float *)(base + o_anc));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "dock_noalloc: start frames");
  }
  if ((e = cudaMemsetAsync(base + o_cnt, 0, sizeof(int) * ((size_t)n + 1), st)) != cudaSuccess)
    return cuda_fail(e, "dock_noalloc: set-up");
  const long long threads = std::max<long long>(n_items, n);
  noalloc_items_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
      (Item *)(base + o_itm), (int *)(base + o_lit), (int *)(base + o_ls0), n, n_starts, chunk, per_lig);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "dock_noalloc: items");
  if ((e = launch_dock(mode, 0, p, sms * occ, 32 * warps, smem, st)) != cudaSuccess)
    return cuda_fail(e, "dock_noalloc: docking kernel");
  return LIGATE_OK;
}
