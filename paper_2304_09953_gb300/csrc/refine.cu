// Pose refinement by gradient descent (paper Sec. 2: the docking search is
// a gradient descent from multiple restarts; the greedy sweep's best poses
// are the restarts and a local descent refines each of them).
//
// State q = (R, t, phi): x_i = R (y_i - c) + t, y the input conformation
// after torsion angle phi_b is applied to each rotatable bond in sweep order
// about its current axis u -> v (c the input centroid; t in Angstrom).  The
// energy is the docking score on the FP32 maps.  Its generalised gradient is
//   F = sum_i g_i,  tau = sum_i (x_i - t) x g_i,
//   psi_b = n_b . sum_{i moved by b} (x_i - x_v) x g_i,
// the derivatives along a translation, a rotation about t and a turn of
// bond b, with g_i = dE/dx_i (trilinear derivative in the atom's cell / h,
// zero for penalty atoms; clash -4 w t (x_i - x_j) / d_c^2 per pair with
// t = 1 - d^2/d_c^2 > 0).  Descent: the trial t - eta F / N,
// GS(exp([-eta tau / I_R]x) R), phi - eta psi / I_b (I_R, I_b the moments
// 1 + sum |r|^2 about t and about each bond axis) is accepted when it lowers
// E (eta *= 1.25), else rejected (eta *= 0.5), for a fixed iteration count.
//
// One warp per pose: lanes over atoms for the coordinate build, the
// per-atom gradient (each lane sums the pair forces on its own atoms, so no
// atomics) and the moment sums; warp reductions give the warp-uniform
// energy and gradient, and lane 0 forms each trial state in shared memory.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "dock_device.cuh"

namespace ligate {
namespace {

constexpr unsigned FULLM = 0xffffffffu;
constexpr int NG = 6 + LIGATE_MAX_ROT;  // gradient components
constexpr int NI = 1 + LIGATE_MAX_ROT;  // moments

struct State {
  float R[9], t[3], phi[LIGATE_MAX_ROT];
};
static_assert(sizeof(State) == sizeof(ligate_pose_state), "state layout");
static_assert(sizeof(ligate_refined) == sizeof(State) + 16, "refined layout");

// Per-warp shared memory.
struct RSmem {
  float4 *ref;  // [nmax] input coordinates - centroid (A), .w = atom type (int bits)
  float4 *x;    // [nmax] coordinates of the state being evaluated
  float4 *g;    // [nmax] dE/dx
  BondRec *bonds;
  State *q;     // [2]: current, trial
  float *G;     // [2][NG]
  float *I;     // [2][NI]
};

// Rounded up to 16 bytes: every warp's float4 arrays must stay 16-byte aligned.
__host__ __device__ inline size_t refine_smem_per_warp(int nmax) {
  const size_t b = (size_t)nmax * 48 + sizeof(BondRec) * LIGATE_MAX_ROT + 2 * sizeof(State) +
                   2 * NG * sizeof(float) + 2 * NI * sizeof(float);
  return (b + 15) / 16 * 16;
}

__device__ __forceinline__ RSmem rsmem(unsigned char *base, int nmax) {
  RSmem w;
  w.ref = reinterpret_cast<float4 *>(base);
  w.x = w.ref + nmax;
  w.g = w.x + nmax;
  w.bonds = reinterpret_cast<BondRec *>(w.g + nmax);
  w.q = reinterpret_cast<State *>(w.bonds + LIGATE_MAX_ROT);
  w.G = reinterpret_cast<float *>(w.q + 2);
  w.I = w.G + 2 * NG;
  return w;
}

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULLM, v, o);
  return v;
}

__device__ __forceinline__ void unit_axis(const float4 &a, const float4 &b, float &nx, float &ny,
                                          float &nz) {
  nx = b.x - a.x; ny = b.y - a.y; nz = b.z - a.z;
  const float inv = rsqrtf(nx * nx + ny * ny + nz * nz);
  nx *= inv; ny *= inv; nz *= inv;
}

// Trilinear value of the FP32 plain map at grid coordinates u and its
// derivative with respect to u (zero outside [0, n-1], where the value is
// the penalty).
__device__ __forceinline__ float map_value_grad(const float *__restrict__ maps, int toff, float ux,
                                                float uy, float uz, const GridConst &g, float &dx,
                                                float &dy, float &dz) {
  dx = dy = dz = 0.f;
  if (!((ux >= 0.f) & (ux <= g.fx1) & (uy >= 0.f) & (uy <= g.fy1) & (uz >= 0.f) & (uz <= g.fz1)))
    return g.penalty;
  const int ix = min((int)ux, g.nx - 2), iy = min((int)uy, g.ny - 2), iz = min((int)uz, g.nz - 2);
  const float fx = ux - (float)ix, fy = uy - (float)iy, fz = uz - (float)iz;
  const float *m = maps + toff + (iz * g.ny + iy) * g.nx + ix;
  const int sy = g.nx, sz = g.nx * g.ny;
  const float v0 = __ldg(m), v1 = __ldg(m + 1), v2 = __ldg(m + sy), v3 = __ldg(m + sy + 1);
  const float v4 = __ldg(m + sz), v5 = __ldg(m + sz + 1), v6 = __ldg(m + sz + sy), v7 = __ldg(m + sz + sy + 1);
  const float d0 = v1 - v0, d1 = v3 - v2, d2 = v5 - v4, d3 = v7 - v6;
  const float y0z0 = fmaf(fx, d0, v0), y1z0 = fmaf(fx, d1, v2);
  const float y0z1 = fmaf(fx, d2, v4), y1z1 = fmaf(fx, d3, v6);
  const float z0 = fmaf(fy, y1z0 - y0z0, y0z0), z1 = fmaf(fy, y1z1 - y0z1, y0z1);
  const float e0 = fmaf(fy, d1 - d0, d0), e1 = fmaf(fy, d3 - d2, d2);
  dx = fmaf(fz, e1 - e0, e0);
  const float c0 = y1z0 - y0z0, c1 = y1z1 - y0z1;
  dy = fmaf(fz, c1 - c0, c0);
  dz = z1 - z0;
  return fmaf(fz, z1 - z0, z0);
}

struct RefineArgs {
  DockParams p;
  float ox, oy, oz, h, inv_h;
  int n;
  const int32_t *lig_idx;      // state/eval modes: ligand of each pose
  const State *init;           // state/eval modes
  const PoseOut *poses;        // plan mode: [rows][K]
  const int32_t *row_lig;      // plan mode: ligand of each row
  int iters;
  float eta0;
  ligate_refined *out;         // refine modes
  float *energy, *grad;        // eval mode
};

// Energy and generalised gradient of state w.q[s] into w.G[s], w.I[s].
__device__ float eval_state(const RefineArgs &a, const RSmem &w, const LigDesc &d, int s, int lane) {
  const DockParams &p = a.p;
  const State &q = w.q[s];
  build_state(w.ref, w.x, w.bonds, d, q.R, q.t, q.phi, lane);
  const int ts = p.g.nx * p.g.ny * p.g.nz;
  const float fcl = -4.f * p.clash_w * p.inv_dc2_ang;
  float e = 0.f, cl = 0.f, F0 = 0.f, F1 = 0.f, F2 = 0.f, T0 = 0.f, T1 = 0.f, T2 = 0.f, IR = 0.f;
  for (int i = lane; i < d.n_atoms; i += 32) {
    const float4 xi = w.x[i];
    float dx, dy, dz;
    e += map_value_grad(p.maps_f32, __float_as_int(xi.w) * ts, (xi.x - a.ox) * a.inv_h,
                        (xi.y - a.oy) * a.inv_h, (xi.z - a.oz) * a.inv_h, p.g, dx, dy, dz);
    float gx = dx * a.inv_h, gy = dy * a.inv_h, gz = dz * a.inv_h;
    for (int wd = 0; wd < d.n_words; ++wd) {
      uint32_t m = __ldg(p.elig + d.elig_base + i * d.n_words + wd);
      while (m) {
        const int j = 32 * wd + __ffs(m) - 1;
        m &= m - 1;
        const float4 xj = w.x[j];
        const float rx = xi.x - xj.x, ry = xi.y - xj.y, rz = xi.z - xj.z;
        const float tt = fmaf(-fmaf(rx, rx, fmaf(ry, ry, rz * rz)), p.inv_dc2_ang, 1.f);
        if (tt > 0.f) {
          if (j > i) cl = fmaf(tt, tt, cl);
          const float f = fcl * tt;
          gx = fmaf(f, rx, gx); gy = fmaf(f, ry, gy); gz = fmaf(f, rz, gz);
        }
      }
    }
    w.g[i] = make_float4(gx, gy, gz, 0.f);
    const float rx = xi.x - q.t[0], ry = xi.y - q.t[1], rz = xi.z - q.t[2];
    F0 += gx; F1 += gy; F2 += gz;
    T0 += ry * gz - rz * gy; T1 += rz * gx - rx * gz; T2 += rx * gy - ry * gx;
    IR += rx * rx + ry * ry + rz * rz;
  }
  const float E = wsum(fmaf(p.clash_w, cl, e));
  F0 = wsum(F0); F1 = wsum(F1); F2 = wsum(F2);
  T0 = wsum(T0); T1 = wsum(T1); T2 = wsum(T2);
  IR = wsum(IR);
  float *G = w.G + s * NG, *I = w.I + s * NI;
  __syncwarp();
  for (int b = 0; b < d.n_rot; ++b) {
    const BondRec br = w.bonds[b];
    const float4 pu = w.x[br.u], pv = w.x[br.v];
    float nx, ny, nz;
    unit_axis(pu, pv, nx, ny, nz);
    float ps = 0.f, ib = 0.f;
    for (int i = br.v + 1 + lane; i < br.end; i += 32) {
      const float4 xi = w.x[i], gi = w.g[i];
      const float rx = xi.x - pv.x, ry = xi.y - pv.y, rz = xi.z - pv.z;
      ps += nx * (ry * gi.z - rz * gi.y) + ny * (rz * gi.x - rx * gi.z) + nz * (rx * gi.y - ry * gi.x);
      const float ra = rx * nx + ry * ny + rz * nz;
      ib += rx * rx + ry * ry + rz * rz - ra * ra;
    }
    ps = wsum(ps);
    ib = wsum(ib);
    if (lane == 0) { G[6 + b] = ps; I[1 + b] = 1.f + ib; }
  }
  if (lane == 0) {
    G[0] = F0; G[1] = F1; G[2] = F2; G[3] = T0; G[4] = T1; G[5] = T2;
    for (int b = d.n_rot; b < LIGATE_MAX_ROT; ++b) { G[6 + b] = 0.f; I[1 + b] = 1.f; }
    I[0] = 1.f + IR;
  }
  __syncwarp();
  return E;
}

// Trial state from w.q[0] with gradient w.G[0] and moments w.I[0] into
// w.q[1] (one thread).
__device__ void make_trial(const RSmem &w, int n_atoms, int n_rot, float eta) {
  const State &q = w.q[0];
  State &t = w.q[1];
  const float *G = w.G, *I = w.I;
  const float sN = eta / (float)n_atoms, sR = -eta / I[0];
  for (int k = 0; k < 3; ++k) t.t[k] = q.t[k] - sN * G[k];
  const float wx = sR * G[3], wy = sR * G[4], wz = sR * G[5];
  const float th = sqrtf(wx * wx + wy * wy + wz * wz);
  float M[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
  if (th > 0.f) {
    const float nx = wx / th, ny = wy / th, nz = wz / th;
    float sn, c;
    sincosf(th, &sn, &c);
    const float o = 1.f - c;
    M[0] = c + o * nx * nx;      M[1] = o * nx * ny - sn * nz; M[2] = o * nx * nz + sn * ny;
    M[3] = o * ny * nx + sn * nz; M[4] = c + o * ny * ny;      M[5] = o * ny * nz - sn * nx;
    M[6] = o * nz * nx - sn * ny; M[7] = o * nz * ny + sn * nx; M[8] = c + o * nz * nz;
  }
  float R[9];
  for (int r = 0; r < 3; ++r)
    for (int cc = 0; cc < 3; ++cc)
      R[3 * r + cc] = M[3 * r] * q.R[cc] + M[3 * r + 1] * q.R[3 + cc] + M[3 * r + 2] * q.R[6 + cc];
  // Gram-Schmidt on the rows, r2 = r0 x r1
  const float l0 = rsqrtf(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
  R[0] *= l0; R[1] *= l0; R[2] *= l0;
  const float dp = R[0] * R[3] + R[1] * R[4] + R[2] * R[5];
  R[3] -= dp * R[0]; R[4] -= dp * R[1]; R[5] -= dp * R[2];
  const float l1 = rsqrtf(R[3] * R[3] + R[4] * R[4] + R[5] * R[5]);
  R[3] *= l1; R[4] *= l1; R[5] *= l1;
  R[6] = R[1] * R[5] - R[2] * R[4];
  R[7] = R[2] * R[3] - R[0] * R[5];
  R[8] = R[0] * R[4] - R[1] * R[3];
  for (int k = 0; k < 9; ++k) t.R[k] = R[k];
  for (int b = 0; b < LIGATE_MAX_ROT; ++b)
    t.phi[b] = b < n_rot ? q.phi[b] - eta * G[6 + b] / I[1 + b] : 0.f;
}

// MODE 0: energy + gradient of explicit states; 1: refine explicit states;
// 2: refine the plan's top-K poses.
template <int MODE>
__global__ void __launch_bounds__(128) refine_kernel(const __grid_constant__ RefineArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const DockParams &p = a.p;
  const RSmem w = rsmem(smem_raw + (size_t)warp * refine_smem_per_warp(p.nmax), p.nmax);
  const int pi = blockIdx.x * (blockDim.x >> 5) + warp;
  if (pi >= a.n) return;
  int li;
  if (MODE == 2) {
    const PoseOut po = a.poses[pi];
    li = a.row_lig[pi / p.K];
    if (po.start_id < 0) {  // empty slot: nothing to refine
      if (lane == 0) {
        ligate_refined r;
        memset(&r, 0, sizeof(r));
        r.score_in = r.score = po.score;
        r.ligand = li;
        a.out[pi] = r;
      }
      return;
    }
    if (lane == 0) {  // state of docked pose (start, tors) in Angstrom
      State &q = w.q[0];
      const int o = po.start_id / p.n_anchor, an = po.start_id - o * p.n_anchor;
      for (int k = 0; k < 9; ++k) q.R[k] = p.rot[9 * o + k] * a.h;
      q.t[0] = fmaf(p.anc[3 * an], a.h, a.ox);
      q.t[1] = fmaf(p.anc[3 * an + 1], a.h, a.oy);
      q.t[2] = fmaf(p.anc[3 * an + 2], a.h, a.oz);
      const float step = 6.283185307179586f / (float)p.S;
      for (int b = 0; b < LIGATE_MAX_ROT; ++b) {
        const int kb = (po.tors[b >> 2] >> (8 * (b & 3))) & 0xff;
        q.phi[b] = (float)(kb % p.S) * step;
      }
    }
  } else {
    li = a.lig_idx[pi];
    if (li < 0 || li >= p.n_ligands) {  // caller's device data
      if (lane == 0) {
        if (MODE == 0) a.energy[pi] = __int_as_float(0x7fc00000);
        else { ligate_refined r; memset(&r, 0, sizeof(r)); r.score_in = r.score = __int_as_float(0x7fc00000); r.ligand = li; a.out[pi] = r; }
      }
      return;
    }
    if (lane == 0) w.q[0] = a.init[pi];
  }
  const LigDesc d = p.lig[li];
  // input coordinates about their centroid
  float sx = 0.f, sy = 0.f, sz = 0.f;
  for (int i = lane; i < d.n_atoms; i += 32) {
    const float4 v = __ldg(p.atoms + d.atom_base + i);
    w.ref[i] = v;
    sx += v.x; sy += v.y; sz += v.z;
  }
  sx = wsum(sx); sy = wsum(sy); sz = wsum(sz);
  const float inv_n = 1.f / (float)d.n_atoms;
  const float cx = sx * inv_n, cy = sy * inv_n, cz = sz * inv_n;
  __syncwarp();
  for (int i = lane; i < d.n_atoms; i += 32) {
    float4 v = w.ref[i];
    v.x -= cx; v.y -= cy; v.z -= cz;
    w.ref[i] = v;
  }
  for (int b = lane; b < d.n_rot; b += 32) w.bonds[b] = p.bonds[d.bond_base + b];
  __syncwarp();

  float E = eval_state(a, w, d, 0, lane);
  if (MODE == 0) {
    if (lane == 0) a.energy[pi] = E;
    for (int k = lane; k < NG; k += 32) a.grad[(size_t)pi * NG + k] = w.G[k];
    return;
  }
  const float e_in = E;
  float eta = a.eta0;
  uint32_t mask = 0;
  for (int it = 0; it < a.iters; ++it) {
    if (lane == 0) make_trial(w, d.n_atoms, d.n_rot, eta);
    __syncwarp();
    const float Et = eval_state(a, w, d, 1, lane);
    if (Et < E) {
      if (lane == 0) {
        w.q[0] = w.q[1];
        for (int k = 0; k < NG; ++k) w.G[k] = w.G[NG + k];
        for (int k = 0; k < NI; ++k) w.I[k] = w.I[NI + k];
      }
      E = Et;
      eta *= 1.25f;
      mask |= 1u << it;
    } else {
      eta *= 0.5f;
    }
    __syncwarp();
  }
  if (lane == 0) {
    ligate_refined r;
    memcpy(&r.state, &w.q[0], sizeof(State));
    r.score_in = e_in;
    r.score = E;
    r.accepted = mask;
    r.ligand = li;
    a.out[pi] = r;
  }
}

}  // namespace

size_t refine_smem_bytes(int nmax) { return refine_smem_per_warp(nmax); }

cudaError_t launch_refine(int mode, const DockParams &p, const double origin[3], double h, int n,
                          const int32_t *lig_idx, const ligate_pose_state *init, const ligate_pose *poses,
                          const int32_t *row_lig, int iters, float eta0, ligate_refined *out,
                          float *energy, float *grad, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  RefineArgs a;
  memset(&a, 0, sizeof(a));
  a.p = p;
  a.ox = (float)origin[0]; a.oy = (float)origin[1]; a.oz = (float)origin[2];
  a.h = (float)h; a.inv_h = (float)(1.0 / h);
  a.n = n;
  a.lig_idx = lig_idx;
  a.init = reinterpret_cast<const State *>(init);
  a.poses = reinterpret_cast<const PoseOut *>(poses);
  a.row_lig = row_lig;
  a.iters = iters;
  a.eta0 = eta0;
  a.out = out;
  a.energy = energy;
  a.grad = grad;
  const int warps = 4;
  const size_t smem = refine_smem_per_warp(p.nmax) * warps;
  const void *fn = mode == 0 ? (const void *)refine_kernel<0>
                 : mode == 1 ? (const void *)refine_kernel<1> : (const void *)refine_kernel<2>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void *args[] = {&a};
  return cudaLaunchKernel(fn, dim3((n + warps - 1) / warps), dim3(32 * warps), args, smem, s);
}

}  // namespace ligate
