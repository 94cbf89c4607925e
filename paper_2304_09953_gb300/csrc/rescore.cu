// Exact rescoring, pose filter and per-pose selector features (paper
// Sec. 2: a more accurate scoring of the generated poses and a filter;
// Sec. 3.5: a high-throughput pose selector).  Poses come from explicit
// (ligand, start, torsion steps) arrays, from a plan's output, or as
// continuous states (refined poses).
#include <math.h>
#include <string.h>

#include <algorithm>

#include "dock_device.cuh"

namespace ligate {

// ---------------------------------------------------------------------------
// Exact rescoring and filter of explicit or planned poses (paper Sec. 2: a
// more accurate scoring of the generated poses, then a filter).  The
// receptor term is the maps' pair potential evaluated at each atom:
// min(cap, sum_j eps_tj ((r0/r)^12 - 2 (r0/r)^6)) over receptor atoms within
// the cutoff, r floored at rmin (grid units throughout); the clash term is
// the docking score's.  The CTA stages all receptor atoms (sorted by cell of
// a grid whose cells are at least the cutoff wide) and the cells' start
// offsets in shared memory; each warp takes poses, builds the pose, and for
// every ligand atom its lanes split the atoms of the 9 rows of 3 cells
// around it (conflict-free consecutive reads); atoms farther away are
// beyond the cutoff.
__global__ void __launch_bounds__(256) rescore_kernel(const DockParams p, const RecParams r, int n_poses,
                                                     const int32_t *__restrict__ lig_idx,
                                                     const int32_t *__restrict__ start_id,
                                                     const uint8_t *__restrict__ tors,
                                                     const PoseOut *__restrict__ poses,
                                                     const int32_t *__restrict__ row_lig,
                                                     const StateSrc ss,
                                                     ligate_rescored *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ncells = r.ncx * r.ncy * r.ncz;
  float4 *rec = reinterpret_cast<float4 *>(smem_raw);
  float2 *pair = reinterpret_cast<float2 *>(rec + r.n_rec);
  int *cell = reinterpret_cast<int *>(pair + ((r.n_types * r.n_types + 1) & ~1));
  unsigned char *slots = reinterpret_cast<unsigned char *>(cell + ((ncells + 1 + 3) & ~3));
  for (int j = threadIdx.x; j < r.n_rec; j += blockDim.x) rec[j] = r.rec[j];
  for (int j = threadIdx.x; j < r.n_types * r.n_types; j += blockDim.x) pair[j] = r.pair[j];
  for (int j = threadIdx.x; j <= ncells; j += blockDim.x) cell[j] = r.cell[j];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  // warp slots without a pair list: more warps per CTA share the staged receptor
  const WarpSmem w = warp_smem(slots + (size_t)warp * smem_bytes_per_warp(p.nmax, 0, 1, 0, 0), p.nmax, 1, 0);
  int cur = -1;
  LigDesc d;
  for (int pi = blockIdx.x * W + warp; pi < n_poses; pi += gridDim.x * W) {
    int li, sid;
    uint32_t tt[4] = {0u, 0u, 0u, 0u};
    const unsigned char *st_rec = nullptr;
    if (ss.base) {  // continuous state
      st_rec = ss.base + (size_t)pi * ss.stride;
      li = ss.lig_idx ? ss.lig_idx[pi] : *reinterpret_cast<const int32_t *>(st_rec + ss.lig_offset);
      sid = (ss.score_offset >= 0 && !isfinite(*reinterpret_cast<const float *>(st_rec + ss.score_offset)))
                ? -1 : 0;  // an empty slot of a refined plan output
    } else if (poses) {
      const PoseOut po = poses[pi];
      li = row_lig[pi / p.K];
      sid = po.start_id;
      for (int q = 0; q < 4; ++q) tt[q] = po.tors[q];
    } else {
      li = lig_idx[pi];
      sid = start_id[pi];
      for (int q = 0; q < 16; ++q) tt[q >> 2] |= (uint32_t)tors[(size_t)pi * 16 + q] << (8 * (q & 3));
    }
    if (li < 0 || li >= p.n_ligands || sid < 0 || sid >= p.n_starts) {  // empty slot or bad index
      if (lane == 0) {
        ligate_rescored o;
        o.energy = o.e_inter = o.e_clash = __int_as_float(0x7f800000);
        o.n_outside = o.n_capped = -1;
        o.pass = 0;
        out[pi] = o;
      }
      continue;
    }
    if (li != cur) {
      __syncwarp();
      (void)load_ligand(p, w, li, d, lane);
      cur = li;
    }
    if (st_rec) {
      // state (R, t, phi): torsions on the centred input coordinates about
      // the current axes, then x = R y + t (A) and u = (x - origin) / h
      const float *R = reinterpret_cast<const float *>(st_rec);
      build_state(w.ref, w.pose, w.bonds, d, R, R + 9, R + 12, lane);
      for (int i = lane; i < d.n_atoms; i += 32) {
        float4 u = w.pose[i];
        u.x = (u.x - r.ox) * r.inv_h;
        u.y = (u.y - r.oy) * r.inv_h;
        u.z = (u.z - r.oz) * r.inv_h;
        w.pose[i] = u;
      }
      __syncwarp();
    } else {
      build_pose<MODE_F32_PLAIN>(p, w, w.pose, d, sid, tt, lane);
    }
    float e_inter = 0.f;
    int ncap = 0, nout = 0;
    for (int i = 0; i < d.n_atoms; ++i) {
      const float4 u = w.pose[i];
      const int t = __float_as_int(w.ref[i].w);
      const float2 *prow = pair + t * r.n_types;
      // the 3 x 3 x 3 cells around the atom (clamped to the grid; the index
      // is clamped in floating point first, so far or non-finite coordinates
      // give an empty neighbourhood or edge cells)
      const int cx = (int)floorf(fminf(fmaxf((u.x - r.lox) * r.icx, -2.f), (float)r.ncx + 1.f));
      const int cy = (int)floorf(fminf(fmaxf((u.y - r.loy) * r.icy, -2.f), (float)r.ncy + 1.f));
      const int cz = (int)floorf(fminf(fmaxf((u.z - r.loz) * r.icz, -2.f), (float)r.ncz + 1.f));
      const int x0 = max(cx - 1, 0), x1 = min(cx + 1, r.ncx - 1);
      const int y0 = max(cy - 1, 0), y1 = min(cy + 1, r.ncy - 1);
      const int z0 = max(cz - 1, 0), z1 = min(cz + 1, r.ncz - 1);
      // two receptor atoms per lane per iteration, separate accumulators:
      // the per-pair chain (distance, ratio, sixth and twelfth powers) is
      // long, so independent pairs keep the pipes busy
      float acc[2] = {0.f, 0.f};
      if (x0 <= x1) {
        for (int z = z0; z <= z1; ++z)
          for (int y = y0; y <= y1; ++y) {
            const int row = (z * r.ncy + y) * r.ncx;
            const int j_hi = cell[row + x1 + 1];
            for (int j0 = cell[row + x0] + lane; j0 < j_hi; j0 += 64) {
#pragma unroll
              for (int q = 0; q < 2; ++q) {
                const int j = j0 + 32 * q;
                if (j < j_hi) {
                  const float4 a = rec[j];
                  const float dx = u.x - a.x, dy = u.y - a.y, dz = u.z - a.z;
                  float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                  if (d2 <= r.cut2) {
                    d2 = fmaxf(d2, r.rmin2);
                    const float2 pp = prow[__float_as_int(a.w)];
                    const float q2 = __fdividef(pp.x, d2);
                    const float q6 = q2 * q2 * q2;
                    acc[q] = fmaf(pp.y, fmaf(q6, q6, -2.f * q6), acc[q]);
                  }
                }
              }
            }
          }
      }
      float accs = warp_sum(acc[0] + acc[1]);
      if (accs >= r.cap) { accs = r.cap; ++ncap; }
      e_inter += accs;
      nout += !((u.x >= 0.f) & (u.x <= p.g.fx1) & (u.y >= 0.f) & (u.y <= p.g.fy1) & (u.z >= 0.f) &
                (u.z <= p.g.fz1));
    }
    float cl = 0.f;
    for (int i = lane; i < d.n_atoms; i += 32) {
      const float4 xi = w.pose[i];
      for (int wd = 0; wd < d.n_words; ++wd) {
        uint32_t m = __ldg(p.elig + d.elig_base + i * d.n_words + wd);
        const int lo = i + 1 - 32 * wd;
        if (lo >= 32) m = 0; else if (lo > 0) m &= ~0u << lo;
        while (m) {
          const int j = 32 * wd + __ffs(m) - 1;
          m &= m - 1;
          const float4 xj = w.pose[j];
          const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
          const float t = fmaxf(0.f, fmaf(-fmaf(dx, dx, fmaf(dy, dy, dz * dz)), p.inv_dc2_grid, 1.f));
          cl = fmaf(t, t, cl);
        }
      }
    }
    cl = p.clash_w * warp_sum(cl);
    if (lane == 0) {
      ligate_rescored o;
      o.e_inter = e_inter;
      o.e_clash = cl;
      o.energy = e_inter + cl;
      o.n_outside = nout;
      o.n_capped = ncap;
      o.pass = (nout == 0 && ncap == 0) ? 1 : 0;
      out[pi] = o;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Per-pose selector features (paper Sec. 3.5: a high-throughput pose
// selector).  Per pose 256 FP32: [0, 64) log1p of the counts of atoms whose
// FP32 grid value v falls in bin min(63, max(0, floor((v + 4) * 4)));
// [64, 72) mean v per atom type 0..7; [72] docking score / atoms; [73] clash
// term; [74] log1p(atoms); [75] rotatable bonds; [76] log1p(count of
// v >= 9); rest 0.  One warp per pose; the histogram lives in the warp's
// pair-list slot.  An empty or invalid pose gives all zeros.
__global__ void __launch_bounds__(128) pose_features_kernel(const DockParams p, int n_poses,
                                                           const int32_t *__restrict__ lig_idx,
                                                           const int32_t *__restrict__ start_id,
                                                           const uint8_t *__restrict__ tors,
                                                           const PoseOut *__restrict__ poses,
                                                           const int32_t *__restrict__ row_lig,
                                                           float *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const WarpSmem w = warp_smem(smem_raw + (size_t)warp * smem_bytes_per_warp(p.nmax, 0, 1, 0), p.nmax, 1);
  int *hist = reinterpret_cast<int *>(w.list);
  int cur = -1;
  LigDesc d;
  for (int pi = blockIdx.x * W + warp; pi < n_poses; pi += gridDim.x * W) {
    float *f = out + (size_t)pi * 256;
    int li, sid;
    uint32_t tt[4] = {0u, 0u, 0u, 0u};
    if (poses) {
      const PoseOut po = poses[pi];
      li = row_lig[pi / p.K];
      sid = po.start_id;
      for (int q = 0; q < 4; ++q) tt[q] = po.tors[q];
    } else {
      li = lig_idx[pi];
      sid = start_id[pi];
      for (int q = 0; q < 16; ++q) tt[q >> 2] |= (uint32_t)tors[(size_t)pi * 16 + q] << (8 * (q & 3));
    }
    if (li < 0 || li >= p.n_ligands || sid < 0 || sid >= p.n_starts) {
      for (int k = lane; k < 256; k += 32) f[k] = 0.f;
      continue;
    }
    if (li != cur) {
      __syncwarp();
      (void)load_ligand(p, w, li, d, lane);
      cur = li;
    }
    build_pose<MODE_F32_PLAIN>(p, w, w.pose, d, sid, tt, lane);
    for (int b = lane; b < 64; b += 32) hist[b] = 0;
    __syncwarp();
    float e = 0.f, high = 0.f, ts[8], tn[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) { ts[t] = 0.f; tn[t] = 0.f; }
    for (int i = lane; i < d.n_atoms; i += 32) {
      const float4 u = w.pose[i];
      const float v = grid_eval<MODE_F32_PLAIN>(p.maps_f32, __float_as_int(u.w), u.x, u.y, u.z, p.g);
      e += v;
      int b = (int)floorf((v + 4.f) * 4.f);
      b = min(63, max(0, b));
      atomicAdd(&hist[b], 1);
      const int ty = __float_as_int(w.ref[i].w);
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (t == ty) { ts[t] += v; tn[t] += 1.f; }
      high += v >= 9.f ? 1.f : 0.f;
    }
    float cl = 0.f;
    for (int i = lane; i < d.n_atoms; i += 32) {
      const float4 xi = w.pose[i];
      for (int wd = 0; wd < d.n_words; ++wd) {
        uint32_t m = __ldg(p.elig + d.elig_base + i * d.n_words + wd);
        const int lo = i + 1 - 32 * wd;
        if (lo >= 32) m = 0; else if (lo > 0) m &= ~0u << lo;
        while (m) {
          const int j = 32 * wd + __ffs(m) - 1;
          m &= m - 1;
          const float4 xj = w.pose[j];
          const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
          const float t = fmaxf(0.f, fmaf(-fmaf(dx, dx, fmaf(dy, dy, dz * dz)), p.inv_dc2_grid, 1.f));
          cl = fmaf(t, t, cl);
        }
      }
    }
    e = warp_sum(e);
    cl = p.clash_w * warp_sum(cl);
    high = warp_sum(high);
#pragma unroll
    for (int t = 0; t < 8; ++t) { ts[t] = warp_sum(ts[t]); tn[t] = warp_sum(tn[t]); }
    __syncwarp();
    for (int b = lane; b < 64; b += 32) f[b] = log1pf((float)hist[b]);
    if (lane < 8) {
      float m = 0.f;
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (t == lane) m = tn[t] > 0.f ? ts[t] / tn[t] : 0.f;
      f[64 + lane] = m;
    }
    if (lane == 0) {
      f[72] = (e + cl) / (float)d.n_atoms;
      f[73] = cl;
      f[74] = log1pf((float)d.n_atoms);
      f[75] = (float)d.n_rot;
      f[76] = log1pf(high);
    }
    for (int k = 77 + lane; k < 256; k += 32) f[k] = 0.f;
    __syncwarp();
  }
}

cudaError_t launch_pose_features(const DockParams &p, int n_poses, const int32_t *lig_idx,
                                 const int32_t *start_id, const uint8_t *tors, const ligate_pose *poses,
                                 const int32_t *row_lig, float *out, cudaStream_t s) {
  if (n_poses <= 0) return cudaSuccess;
  const int warps = 4;
  const size_t smem = (size_t)warps * smem_bytes_per_warp(p.nmax, 0, 1, 0);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(pose_features_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, occ = 0;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pose_features_kernel, 32 * warps, smem)))
    return e;
  const long long need = (n_poses + warps - 1) / warps;
  const int grid = (int)std::min<long long>(need, (long long)sms * std::max(occ, 1));
  pose_features_kernel<<<grid, 32 * warps, smem, s>>>(p, n_poses, lig_idx, start_id, tors,
                                                      reinterpret_cast<const PoseOut *>(poses), row_lig, out);
  return cudaGetLastError();
}

size_t rescore_smem_bytes(const DockParams &p, const RecParams &r, int warps) {
  const int ncells = r.ncx * r.ncy * r.ncz;
  return (size_t)r.n_rec * 16 + (size_t)((r.n_types * r.n_types + 1) & ~1) * 8 +
         (size_t)((ncells + 1 + 3) & ~3) * 4 + (size_t)warps * smem_bytes_per_warp(p.nmax, 0, 1, 0, 0);
}

cudaError_t launch_rescore(const DockParams &p, const RecParams &r, int n_poses, const int32_t *lig_idx,
                           const int32_t *start_id, const uint8_t *tors, const ligate_pose *poses,
                           const int32_t *row_lig, const StateSrc *states, ligate_rescored *out,
                           cudaStream_t s) {
  if (n_poses <= 0) return cudaSuccess;
  int warps = 8;
  while (warps > 1 && rescore_smem_bytes(p, r, warps) > 227 * 1024) --warps;
  const size_t smem = rescore_smem_bytes(p, r, warps);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(rescore_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, occ = 0;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, rescore_kernel, 32 * warps, smem)))
    return e;
  const long long need = (n_poses + warps - 1) / warps;
  const int grid = (int)std::min<long long>(need, (long long)sms * std::max(occ, 1));
  StateSrc ss;
  memset(&ss, 0, sizeof(ss));
  if (states) ss = *states;
  rescore_kernel<<<grid, 32 * warps, smem, s>>>(p, r, n_poses, lig_idx, start_id, tors,
                                                reinterpret_cast<const PoseOut *>(poses), row_lig, ss, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Coordinates of continuous states as the refinement and the exact
// rescoring build them (build_state): one warp per state, Angstrom, atoms
// written back in the ligand's input order.
__global__ void __launch_bounds__(256) state_coords_kernel(const DockParams p, const uint8_t *__restrict__ order,
                                                           int n, const int32_t *__restrict__ lig_idx,
                                                           const ligate_pose_state *__restrict__ states,
                                                           float *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const WarpSmem w = warp_smem(smem_raw + (size_t)warp * smem_bytes_per_warp(p.nmax, 0, 1, 0), p.nmax, 1);
  const int pi = blockIdx.x * (blockDim.x >> 5) + warp;
  if (pi >= n) return;
  float *o = out + (size_t)pi * LIGATE_MAX_ATOMS * 3;
  const int li = lig_idx[pi];
  if (li < 0 || li >= p.n_ligands) {  // caller's device data
    for (int q = lane; q < LIGATE_MAX_ATOMS * 3; q += 32) o[q] = __int_as_float(0x7fc00000);
    return;
  }
  LigDesc d;
  (void)load_ligand(p, w, li, d, lane);
  const ligate_pose_state &st = states[pi];
  build_state(w.ref, w.pose, w.bonds, d, st.rot, st.trans, st.tors, lane);
  for (int i = lane; i < d.n_atoms; i += 32) {
    const float4 x = w.pose[i];
    float *a = o + 3 * (int)order[d.atom_base + i];
    a[0] = x.x; a[1] = x.y; a[2] = x.z;
  }
}

cudaError_t launch_state_coords(const DockParams &p, const uint8_t *order, int n, const int32_t *lig_idx,
                                const ligate_pose_state *states, float *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int warps = 4;
  const size_t smem = (size_t)warps * smem_bytes_per_warp(p.nmax, 0, 1, 0);
  cudaError_t e = cudaFuncSetAttribute(state_coords_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       227 * 1024);
  if (e != cudaSuccess) return e;
  state_coords_kernel<<<(n + warps - 1) / warps, 32 * warps, smem, s>>>(p, order, n, lig_idx, states, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-ligand result after the filter (paper Sec. 2: docking, then rescoring
// and a filter; a ligand scores as its best surviving pose): one thread per
// row of K rescored poses, the lowest energy among those that pass (ties:
// the smaller slot), or -1 and +inf when none passes.
__global__ void best_passing_kernel(const ligate_rescored *__restrict__ rec, int n, int K,
                                    int32_t *__restrict__ idx, float *__restrict__ energy) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int best = -1;
  float be = __int_as_float(0x7f800000);
  for (int k = 0; k < K; ++k) {
    const ligate_rescored q = rec[(size_t)r * K + k];
    if (q.pass == 1 && (best < 0 || q.energy < be)) { best = k; be = q.energy; }
  }
  idx[r] = best;
  if (energy) energy[r] = be;
}

// Learned pose selector's rule (paper Sec. 3.5: a pose selector that keeps
// one pose per ligand without rescoring them all): per row of K poses in
// docking order, the first live pose (start id >= 0) whose predicted label
// is below pass_below; else the live pose with the lowest prediction (ties:
// the smaller slot); -1 for a row without a live pose.
__global__ void select_poses_kernel(const float *__restrict__ pred, const PoseOut *__restrict__ poses, int n,
                                    int K, float pass_below, int32_t *__restrict__ idx) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int first = -1, low = -1;
  float lp = 0.f;
  for (int k = 0; k < K; ++k) {
    if (poses[(size_t)r * K + k].start_id < 0) continue;
    const float v = pred[(size_t)r * K + k];
    if (first < 0 && v < pass_below) first = k;
    if (low < 0 || v < lp) { low = k; lp = v; }
  }
  idx[r] = first >= 0 ? first : low;
}

// Selector training label of a rescored pose: its energy clipped to
// fail_label when it passes the filter, fail_label when it fails (an empty
// slot too).
__global__ void selector_labels_kernel(const ligate_rescored *__restrict__ rec, long long n, float fail_label,
                                       float *__restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const ligate_rescored q = rec[i];
  out[i] = q.pass == 1 ? fminf(q.energy, fail_label) : fail_label;
}

cudaError_t launch_best_passing(const ligate_rescored *rec, int n, int K, int32_t *idx, float *energy,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  best_passing_kernel<<<(n + 127) / 128, 128, 0, s>>>(rec, n, K, idx, energy);
  return cudaGetLastError();
}

cudaError_t launch_select_poses(const float *pred, const ligate_pose *poses, int n, int K, float pass_below,
                                int32_t *idx, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  select_poses_kernel<<<(n + 127) / 128, 128, 0, s>>>(pred, reinterpret_cast<const PoseOut *>(poses), n, K,
                                                      pass_below, idx);
  return cudaGetLastError();
}

cudaError_t launch_selector_labels(const ligate_rescored *rec, long long n, float fail_label, float *out,
                                   cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  selector_labels_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rec, n, fail_label, out);
  return cudaGetLastError();
}

}  // namespace ligate
