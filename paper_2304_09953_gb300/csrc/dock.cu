// Persistent docking kernel for sm_103a: rigid starts (orientation x anchor),
// greedy torsion sweep, trilinear grid score + intramolecular clash term,
// warp-shuffle top-K per ligand, last-arriver merge and optional FP32
// rescoring.  Paper Sec. 2 (multi-restart docking with a geometric score;
// ligand score = best pose; optional re-scoring of the generated poses) and
// Sec. 3.3 (one batch of ligand-pocket pairs per device launch).
//
// Work mapping.  A warp takes work items (ligand, range of starts) from a
// global queue.  Inside the warp, lanes form G = 32 / L groups of L lanes
// (L = S rounded up to a power of two); each group runs one start, and lane
// k of a group evaluates torsion step k of the current bond.  Every lane of
// the warp therefore executes the same bond, the same moved atom and the same
// clash partner at the same time: no divergence, and each pose coordinate is
// a shared-memory broadcast.  Only the moved side of the current bond is
// re-scored (the rest of the score is the same for every k); the k = 0 lane
// re-evaluates the current pose, so E += V(k*) - V(0).
//
// Branch and bound: a start whose lower bound on its final energy exceeds
// the K-th best energy already found stops sweeping (bound_setup,
// beyond_bound); the top-K is unchanged.  The two groups of a warp run in
// lockstep, so a work item visits each orientation's anchors in the plan's
// nearest-neighbour pair order (DockParams::visit): partners sweep nearby
// poses and tend to stop together, and then the warp leaves the bond loop.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include <algorithm>

#include "dock_device.cuh"

namespace ligate {

size_t dock_smem_per_warp(int nmax, int S, int G, int rmax) { return smem_bytes_per_warp(nmax, S, G, rmax); }

int dock_memo1_tables(const LigDesc &d, const BondRec *bonds, int) {
  int n = 0;
  for (int b = 2; b < d.n_rot; ++b) n += bonds[b].n_cand1 > 0;
  return n;
}

// Clash part of the sweep of bond br at this lane's torsion step (ck, sk):
// the sum over the bond's crossing candidate pairs of max(0, 1 - d^2/d_c^2)^2
// on the group's conformation `pose` (grid units; axis n through pv).
// Moved atom i travels on a circle about the axis; with
// u = radial vector of i, m = n x u, w = radial vector of fixed atom
// j, P = u.w, Q = m.w and D0 = |x_i - x_j|^2 at the current pose,
//   d^2(theta) = D0 + 2P (1 - cos theta) - 2Q sin theta,
// whose minimum over the circle is D0 + 2P - 2 sqrt(P^2 + Q^2).  A
// pair whose minimum is beyond d_c contributes exactly zero at every
// step and is dropped; the others are evaluated in closed form.
// Warp-collective: every lane calls it, each with its own group's data; a
// group that is not `alive` (its start was pruned) loads and tests nothing.
__device__ __forceinline__ float clash_sweep(const DockParams &p, const WarpSmem &w, const float4 *pose,
                                             const LigDesc &d, const BondRec &br, float nx, float ny,
                                             float nz, const float4 &pv, float ck, float sk, int g,
                                             int k, int L, int G, unsigned &n_test, unsigned &n_pair,
                                             bool alive = true) {
  float ac = 0.f;
  const int cap = PAIR_WARP / G;  // = 6 L
  float4 *list = w.list + g * cap;
  float2 *cab = w.cab + g * p.nmax;  // (axial a, radial distance b) of each atom
  const unsigned lmask = L == 32 ? FULL : ((1u << L) - 1u);
  const unsigned below = (1u << k) - 1u;
  const float omc = 1.f - ck;
  int cnt = 0;
  for (int j = alive ? k : d.n_atoms; j < d.n_atoms; j += L) {
    const float4 xj = pose[j];
    const float fx = xj.x - pv.x, fy = xj.y - pv.y, fz = xj.z - pv.z;
    const float a = fmaf(fx, nx, fmaf(fy, ny, fz * nz));
    const float wx = fmaf(-a, nx, fx), wy = fmaf(-a, ny, fy), wz = fmaf(-a, nz, fz);
    // radial distance by the hardware square-root approximation (relative
    // error ~1e-7): it only feeds the survivor test, whose threshold carries
    // a 1e-4 margin, and the pair coefficients' squared radii
    float rb;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(rb) : "f"(fmaf(wx, wx, fmaf(wy, wy, wz * wz))));
    cab[j] = make_float2(a, rb);
  }
  __syncwarp();
  auto flush = [&]() {
    __syncwarp();
    // the group's lanes turn buffered pair indices into closed-form
    // coefficients, one pair per lane
    for (int q = k; q < cnt; q += L) {
      const unsigned pr = __float_as_uint(list[q].w);
      const int i = pr & 0xffu, j = pr >> 8;
      const float2 hi = cab[i], hj = cab[j];
      const float4 xi = pose[i], xj = pose[j];
      // radial vectors about the axis: w = (x - p) - a n
      const float4 ui = make_float4(fmaf(-hi.x, nx, xi.x - pv.x), fmaf(-hi.x, ny, xi.y - pv.y),
                                    fmaf(-hi.x, nz, xi.z - pv.z), 0.f);
      const float4 wj = make_float4(fmaf(-hj.x, nx, xj.x - pv.x), fmaf(-hj.x, ny, xj.y - pv.y),
                                    fmaf(-hj.x, nz, xj.z - pv.z), 0.f);
      const float da = hi.x - hj.x;
      const float P = fmaf(ui.x, wj.x, fmaf(ui.y, wj.y, ui.z * wj.z));
      const float cx = ui.y * wj.z - ui.z * wj.y, cy = ui.z * wj.x - ui.x * wj.z,
                  cz = ui.x * wj.y - ui.y * wj.x;
      const float Q = fmaf(nx, cx, fmaf(ny, cy, nz * cz));  // (n x u).w
      const float D0 = fmaf(da, da, fmaf(hi.y, hi.y, fmaf(hj.y, hj.y, -2.f * P)));
      list[q] = make_float4(fmaf(-D0, p.inv_dc2_grid, 1.f), -2.f * P * p.inv_dc2_grid,
                            2.f * Q * p.inv_dc2_grid, 0.f);
    }
    __syncwarp();
    const int top = __reduce_max_sync(FULL, (unsigned)cnt);
    for (int q = 0; q < top; ++q) {
      if (q < cnt) {
        const float4 e = list[q];
        const float t = fmaxf(0.f, fmaf(e.z, sk, fmaf(e.y, omc, e.x)));
        ac = fmaf(t, t, ac);
      }
    }
    n_pair += cnt;
    cnt = 0;
    __syncwarp();
  };
  // candidates of this bond, L per pass; with u = radial vector of the
  // moved atom, the minimum distance over its circle is
  // sqrt(da^2 + (b_j - b_i)^2)
  const uint16_t *cand = p.cand + d.cand_base + br.cand_off;
  if (alive) n_test += br.n_cand;
  // PASSES independent passes of L candidates per iteration: their
  // loads and tests overlap, then the survivors are appended in order
  constexpr int PASSES = 4;
  for (int c0 = 0; c0 < br.n_cand; c0 += PASSES * L) {
    unsigned pr[PASSES];
    bool surv[PASSES];
#pragma unroll
    for (int u = 0; u < PASSES; ++u) {
      const int c = c0 + u * L + k;
      pr[u] = alive && c < br.n_cand ? __ldg(cand + c) : 0u;
    }
#pragma unroll
    for (int u = 0; u < PASSES; ++u) {
      const float2 hi = cab[pr[u] & 0xffu], hj = cab[pr[u] >> 8];
      const float da = hi.x - hj.x, db = hj.y - hi.y;
      surv[u] = alive && (c0 + u * L + k < br.n_cand) && fmaf(da, da, db * db) < p.dc2_grid_margin;
    }
#pragma unroll
    for (int u = 0; u < PASSES; ++u) {
      const unsigned gm = (__ballot_sync(FULL, surv[u]) >> (g * L)) & lmask;
      if (surv[u]) list[cnt + __popc(gm & below)].w = __uint_as_float(pr[u]);
      cnt += __popc(gm);
    }
    if (__any_sync(FULL, cnt > cap - PASSES * L)) flush();
  }
  flush();
  return ac;
}

// Clash sums of the first n_memo bonds' sweeps into w.memo: memo[k] for
// bond 0 on the input conformation, memo[S + k0 S + k] for bond 1 after
// bond 0 turned by step k0; and of each later bond b, the sums over its
// first n_cand0 candidates on the input conformation, memo[memo_row0(S) +
// (b - memo_bonds(S)) S + k]; and, when m1 is given, of each bond b >= 2
// with pairs that bond e1 alone separates, the sums over those pairs after
// e1 turned by step t, m1[(slot S + t) S + k] (e1 and slot packed in e1).
// Conformations are posed by start 0's frame (the clash term is invariant
// under the rigid move); group g takes k0 = g, g + G, ...  Warp-collective.
__device__ void build_memo(const DockParams &p, const WarpSmem &w, float4 *pose, const LigDesc &d,
                           int n_memo, float ck, float sk, int g, int k, int L, int G, int S,
                           float *__restrict__ m1) {
  unsigned n_test = 0, n_pair = 0;  // not counted: once per ligand
  float R[9], T[3];
  start_frame(p, 0, R, T);
  if (m1) {
    for (int b = 2; b < d.n_rot; ++b) {
      BondRec bb = w.bonds[b];
      if (bb.n_cand1 == 0) continue;  // warp-uniform
      const int slot = bb.e1 >> 16;
      const BondRec be = w.bonds[bb.e1 & 0xffff];
      bb.cand_off += bb.n_cand0;
      bb.n_cand = bb.n_cand1;
      for (int r = 0; r < (S + G - 1) / G; ++r) {
        const int te = min(r * G + g, S - 1);  // groups past S repeat the last step
        for (int i = k; i < d.n_atoms; i += L) {
          const float4 a = w.ref[i];
          pose[i] = make_float4(fmaf(R[0], a.x, fmaf(R[1], a.y, fmaf(R[2], a.z, T[0]))),
                                fmaf(R[3], a.x, fmaf(R[4], a.y, fmaf(R[5], a.z, T[1]))),
                                fmaf(R[6], a.x, fmaf(R[7], a.y, fmaf(R[8], a.z, T[2]))), 0.f);
        }
        __syncwarp();
        float ex, ey, ez;
        const float4 ev = pose[be.v];
        bond_axis(pose[be.u], ev, ex, ey, ez);
        float ce, se;
        step_cs(p, te, ce, se);
        Rot re;
        re.make(ce, se, ex, ey, ez, ev.x, ev.y, ev.z);
        __syncwarp();
        for (int i = be.v + 1 + k; i < be.end; i += L) {
          float4 q = pose[i];
          re.apply(q.x, q.y, q.z, q.x, q.y, q.z);
          pose[i] = q;
        }
        __syncwarp();
        float mx, my, mz;
        const float4 qv = pose[bb.v];
        bond_axis(pose[bb.u], qv, mx, my, mz);
        const float a1 = clash_sweep(p, w, pose, d, bb, mx, my, mz, qv, ck, sk, g, k, L, G, n_test, n_pair);
        if (r * G + g < S && k < S) {  // kept in L2 ahead of streaming data (evict-last policy)
          uint64_t pol;
          asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
          asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(m1 + (slot * S + te) * S + k), "f"(a1),
                       "l"(pol) : "memory");
        }
        __syncwarp();
      }
    }
  }
  const int rounds = n_memo == 2 ? (S + G - 1) / G : 0;
  for (int r = -1; r < rounds; ++r) {  // r = -1: bond 0 on the input conformation
    for (int i = k; i < d.n_atoms; i += L) {
      const float4 a = w.ref[i];
      pose[i] = make_float4(fmaf(R[0], a.x, fmaf(R[1], a.y, fmaf(R[2], a.z, T[0]))),
                            fmaf(R[3], a.x, fmaf(R[4], a.y, fmaf(R[5], a.z, T[1]))),
                            fmaf(R[6], a.x, fmaf(R[7], a.y, fmaf(R[8], a.z, T[2]))), 0.f);
    }
    __syncwarp();
    const BondRec b0 = w.bonds[0];
    float nx, ny, nz;
    float4 pv = pose[b0.v];
    bond_axis(pose[b0.u], pv, nx, ny, nz);
    if (r < 0) {
      const float ac = clash_sweep(p, w, pose, d, b0, nx, ny, nz, pv, ck, sk, g, k, L, G, n_test, n_pair);
      if (g == 0 && k < S) w.memo[k] = ac;
      __syncwarp();
      for (int b = memo_bonds(S); b < d.n_rot; ++b) {  // the fixed-geometry pairs of later bonds
        BondRec bb = w.bonds[b];
        if (bb.n_cand0 == 0) continue;  // warp-uniform
        bb.n_cand = bb.n_cand0;
        float mx, my, mz;
        const float4 qv = pose[bb.v];
        bond_axis(pose[bb.u], qv, mx, my, mz);
        const float a0 = clash_sweep(p, w, pose, d, bb, mx, my, mz, qv, ck, sk, g, k, L, G, n_test, n_pair);
        if (g == 0 && k < S) w.memo[memo_row0(S) + (b - memo_bonds(S)) * S + k] = a0;
        __syncwarp();
      }
      continue;
    }
    const int k0 = min(r * G + g, S - 1);  // groups past S repeat the last step
    float c0, s0;
    step_cs(p, k0, c0, s0);
    Rot rb;
    rb.make(c0, s0, nx, ny, nz, pv.x, pv.y, pv.z);
    __syncwarp();
    for (int i = b0.v + 1 + k; i < b0.end; i += L) {
      float4 q = pose[i];
      rb.apply(q.x, q.y, q.z, q.x, q.y, q.z);
      pose[i] = q;
    }
    __syncwarp();
    const BondRec b1 = w.bonds[1];
    pv = pose[b1.v];
    bond_axis(pose[b1.u], pv, nx, ny, nz);
    const float ac = clash_sweep(p, w, pose, d, b1, nx, ny, nz, pv, ck, sk, g, k, L, G, n_test, n_pair);
    if (r * G + g < S && k < S) w.memo[S + k0 * S + k] = ac;
    __syncwarp();
  }
}

// Drops the L2 copies of the whole 128-byte lines inside [lo, hi) without
// writing them back to DRAM: for scratch whose contents are dead (a
// ligand's merged partial lists, a warp's clash tables at exit).  Lines that
// reach outside the range may hold another owner's live data and are left
// alone.  Warp-collective over `lane`; the caller has finished its reads.
// A discard acts as a write of undefined data, so the fence and the warp
// barrier order it before any lane's next write to the same lines.
__device__ __forceinline__ void l2_discard(const void *lo, const void *hi, int lane) {
  const uintptr_t a = ((uintptr_t)lo + 127u) & ~(uintptr_t)127u, b = (uintptr_t)hi & ~(uintptr_t)127u;
  for (uintptr_t q = a + (uintptr_t)lane * 128u; q < b; q += 32u * 128u)
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(q) : "memory");
  __threadfence();
  __syncwarp();
}

// Lower bound of a start's final energy (branch and bound on the sweep).
// A bond turns the DFS range (v, end); atom i is moved by no bond after the
// last one whose range holds it.  Before bond b the atoms with lastb <= b are
// fixed for good, the others can still reach any cell, and the clash term is
// never negative, so the final energy is at least
//   A_b + lbc[b],  A_b = grid energy of the fixed atoms at the current pose,
//   lbc[b] = sum over the atoms a bond >= b moves of their type's map minimum.
// lastb[i] = 1 + that last bond (0: no bond moves atom i).  Warp-collective.
__device__ void bound_setup(const DockParams &p, const WarpSmem &w, const LigDesc &d, int lane) {
  for (int i = lane; i < d.n_atoms; i += 32) {
    int last = 0;
    for (int b = 0; b < d.n_rot; ++b) {
      const BondRec &br = w.bonds[b];
      if (i > br.v && i < br.end) last = b + 1;
    }
    w.lastb[i] = (uint8_t)last;
  }
  for (int s = 0; s <= d.n_rot; ++s) {  // each lane reads the lastb entries it wrote
    float a = 0.f;
    for (int i = lane; i < d.n_atoms; i += 32)
      if (w.lastb[i] > s) a += p.gmin[__float_as_int(w.ref[i].w)];
    a = warp_sum(a);
    if (lane == 0) w.lbc[s] = a;
  }
  __syncwarp();
}

// Order-preserving 32-bit key of a float (smaller value, smaller key) and
// its inverse; the argmin of the sweep uses the same map.
__device__ __forceinline__ unsigned value_key(float v) {
  const unsigned b = __float_as_uint(v);
  return b ^ ((unsigned)((int)b >> 31) | 0x80000000u);
}
__device__ __forceinline__ float key_value(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k ^ 0x80000000u) : ~k);
}

// True when a start whose final energy is at least `lb` cannot enter a top-K
// whose K-th best energy is `thr`.  The margin covers the FP32 rounding of
// the running energy and of the bound (sums of at most 128 terms of
// magnitude at most the cap, over at most 16 bonds), so the test holds for
// the kernel's own arithmetic; an empty top-K (thr = inf) prunes nothing.
__device__ __forceinline__ bool beyond_bound(float lb, float thr) {
  return lb > thr + 1.f + (fabsf(thr) + fabsf(lb)) * (1.f / 1024.f);
}

// ---------------------------------------------------------------------------
// CTAs of at most 128 threads; MINB of them must fit on one SM: 4 caps the
// registers at 128 (16 resident warps), 5 at 102 (20 warps), 6 at 85 (24
// warps, a few spills).
// Latency of the map gathers is covered by resident warps, so occupancy
// matters more than per-thread registers here.
template <int MODE, int MINB>
__global__ void __launch_bounds__(128, MINB) dock_kernel(const DockParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const WarpSmem w = warp_smem(smem_raw + (size_t)warp * smem_bytes_per_warp(p.nmax, p.S, p.G, p.rmax),
                               p.nmax, p.G);
  const int L = p.L, G = p.G, S = p.S, K = p.K;
  const int g = lane / L, k = lane - g * L;
  const int glead = g * L;
  float4 *pose = w.pose + (size_t)g * (p.nmax + 1);
  float ck = 1.f, sk = 0.f;
  if (k < S) step_cs(p, k, ck, sk);
  const int ts = type_stride(MODE, p.g);
  const float INF = __int_as_float(0x7f800000);
  float *const m1 = p.memo1 ? p.memo1 + ((size_t)blockIdx.x * (blockDim.x >> 5) + warp) * p.m1max * S * S
                            : nullptr;

  const int n_items = p.n_items_dev ? __ldcg(p.n_items_dev) : p.n_items;
  int cur = -1, n_memo = 0;
  LigDesc d;
  float clash_ref = 0.f;
  TopK top;

  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(p.queue, 1);
    it = __shfl_sync(FULL, it, 0);
    if (it >= n_items) {
      if (m1) {  // this warp's clash tables are dead: no write-back
        __syncwarp();
        l2_discard(m1, m1 + (size_t)p.m1max * S * S, lane);
      }
      break;
    }
    const Item item = p.items[it];
    if (item.ligand != cur) {
      __syncwarp();
      if (m1 && cur >= 0) l2_discard(m1, m1 + (size_t)p.m1max * S * S, lane);  // the last ligand's tables
      clash_ref = load_ligand(p, w, item.ligand, d, lane);
      cur = item.ligand;
      n_memo = min(d.n_rot, memo_bonds(S));
      if (n_memo > 0) build_memo(p, w, pose, d, n_memo, ck, sk, g, k, L, G, S, m1);
      bound_setup(p, w, d, lane);
    }
    top.clear();
    float thr = INF;  // K-th best energy of the item so far: a start bounded above it stops
    float thr_pub = INF;  // the last value this warp shared with the row's other items
    unsigned *const row_thr = p.lig_thr ? p.lig_thr + item.row : nullptr;
    const float cut = p.cut ? __ldcg(p.cut) : INF;  // screening cutoff (the same for every ligand)
    // work counters of this lane's group: atom interpolations, pair tests,
    // pair survivors, candidate pairs of the evaluated sweeps, pruned starts,
    // evaluated bond sweeps
    unsigned n_atom = 0, n_test = 0, n_pair = 0, n_cand = 0, n_prn = 0, n_bsw = 0;

    for (int s0 = item.s0; s0 < item.s1; s0 += G) {
      // visit index (a group past the end repeats the last one) -> start id:
      // each orientation's anchors in the plan's visiting order
      const int vi = min(s0 + g, item.s1 - 1);
      const int sid = p.visit ? vi - vi % p.n_anchor + p.visit[vi % p.n_anchor] : vi;
      const unsigned n_atom0 = n_atom, n_test0 = n_test, n_pair0 = n_pair;
      // the row's shared K-th best (any item's is at least the row's final
      // one, so it bounds as safely as this item's own), loaded now and used
      // after the rigid stage's gathers
      unsigned shared_key = 0;
      if (row_thr && lane == 0) shared_key = __ldcg(row_thr);
      // -- rigid start: pose = R_o (x - c) / h + (a - origin) / h
      float R[9], T[3];
      start_frame(p, sid, R, T);
      float e = 0.f, ef = 0.f;  // ef: the atoms no bond moves
      for (int i = k; i < d.n_atoms; i += L) {
        const float4 r = w.ref[i];
        float4 u;
        u.x = fmaf(R[0], r.x, fmaf(R[1], r.y, fmaf(R[2], r.z, T[0])));
        u.y = fmaf(R[3], r.x, fmaf(R[4], r.y, fmaf(R[5], r.z, T[1])));
        u.z = fmaf(R[6], r.x, fmaf(R[7], r.y, fmaf(R[8], r.z, T[2])));
        const int toff = __float_as_int(r.w) * ts;
        u.w = __int_as_float(toff);
        pose[i] = u;
        const float gi = grid_eval<MODE>(p.maps, toff, u.x, u.y, u.z, p.g);
        e += gi;
        if (w.lastb[i] == 0) ef += gi;
      }
      for (int o = L >> 1; o > 0; o >>= 1) {
        e += __shfl_xor_sync(FULL, e, o);
        ef += __shfl_xor_sync(FULL, ef, o);
      }
      float E = fmaf(p.clash_w, clash_ref, e);
      float A = ef;  // grid energy of the atoms fixed for good (the bound's first part)
      shared_key = __shfl_sync(FULL, shared_key, 0);
      const float thr_use = fminf(fminf(thr, cut), shared_key ? key_value(~shared_key) : INF);
      // a group past the item's end, or a start bounded above the K-th best, sweeps nothing
      bool alive = s0 + g < item.s1 && !beyond_bound(A + w.lbc[0], thr_use);
      if (s0 + g < item.s1 && !alive) ++n_prn;
      n_atom += d.n_atoms;
      uint32_t t0 = 0, t1 = 0, t2 = 0, t3 = 0;
      __syncwarp();

      // -- greedy torsion sweep
      for (int b = 0; b < d.n_rot; ++b) {
        if (!__any_sync(FULL, alive)) break;  // every start of the warp is pruned
        const BondRec br = w.bonds[b];
        const float4 pv = pose[br.v];
        float nx, ny, nz;
        bond_axis(pose[br.u], pv, nx, ny, nz);
        Rot rot;
        rot.make(ck, sk, nx, ny, nz, pv.x, pv.y, pv.z);
        // grid part: every moved atom at this lane's torsion step, two atoms
        // per iteration: two map gathers in flight per lane, and the rotation
        // and interpolation arithmetic of the pair in packed FP32 (FFMA2);
        // agf: the atoms this bond moves for the last time (fixed after it)
        float ag = 0.f, ag2 = 0.f, agf = 0.f;
        const int bb = b + 1, iend = alive ? br.end : 0;  // a pruned group evaluates nothing
        int i = br.v + 1;
        for (; i + 1 < iend; i += 2) {
          const float4 q = pose[i], q2 = pose[i + 1];
          if (MODE == MODE_F32_PLAIN) {  // eight scalar gathers each: registers go to loads in flight
            float yx, yy, yz, zx, zy, zz;
            rot.apply(q.x, q.y, q.z, yx, yy, yz);
            rot.apply(q2.x, q2.y, q2.z, zx, zy, zz);
            const float ga = grid_eval<MODE>(p.maps, __float_as_int(q.w), yx, yy, yz, p.g);
            const float gb = grid_eval<MODE>(p.maps, __float_as_int(q2.w), zx, zy, zz, p.g);
            ag += ga;
            ag2 += gb;
            agf += (w.lastb[i] == bb ? ga : 0.f) + (w.lastb[i + 1] == bb ? gb : 0.f);
            continue;
          }
          const float2 X = make_float2(q.x, q2.x), Y = make_float2(q.y, q2.y), Z = make_float2(q.z, q2.z);
          const float2 ox = __ffma2_rn(make_float2(rot.r00, rot.r00), X, __ffma2_rn(make_float2(rot.r01, rot.r01), Y,
                            __ffma2_rn(make_float2(rot.r02, rot.r02), Z, make_float2(rot.tx, rot.tx))));
          const float2 oy = __ffma2_rn(make_float2(rot.r10, rot.r10), X, __ffma2_rn(make_float2(rot.r11, rot.r11), Y,
                            __ffma2_rn(make_float2(rot.r12, rot.r12), Z, make_float2(rot.ty, rot.ty))));
          const float2 oz = __ffma2_rn(make_float2(rot.r20, rot.r20), X, __ffma2_rn(make_float2(rot.r21, rot.r21), Y,
                            __ffma2_rn(make_float2(rot.r22, rot.r22), Z, make_float2(rot.tz, rot.tz))));
          const float2 v = grid_eval2<MODE>(p.maps, __float_as_int(q.w), ox.x, oy.x, oz.x, __float_as_int(q2.w),
                                            ox.y, oy.y, oz.y, p.g);
          ag += v.x;
          ag2 += v.y;
          agf += (w.lastb[i] == bb ? v.x : 0.f) + (w.lastb[i + 1] == bb ? v.y : 0.f);
        }
        if (i < iend) {
          const float4 q = pose[i];
          float yx, yy, yz;
          rot.apply(q.x, q.y, q.z, yx, yy, yz);
          const float ga = grid_eval<MODE>(p.maps, __float_as_int(q.w), yx, yy, yz, p.g);
          ag += ga;
          if (w.lastb[i] == bb) agf += ga;
        }
        ag += ag2;
        if (alive) {
          n_atom += (unsigned)(br.end - br.v - 1) * (unsigned)S;
          n_cand += (unsigned)br.n_cand;
          ++n_bsw;
        }
        float ac;
        if (b < n_memo) {  // looked up: bond 0, or bond 1 after bond 0's step
          ac = k < S ? w.memo[b == 0 ? k : S + (int)(t0 & 0xffu) * S + k] : 0.f;
        } else {  // pairs whose geometry earlier steps change, swept live, + the memoised rest
          // the pairs bond e1 alone separates: their sums by e1's chosen
          // step, loaded before the live sweep and added after it
          const bool has1 = m1 && b >= 2 && br.n_cand1 > 0;  // warp-uniform
          float c1 = 0.f;
          if (alive && has1 && k < S) {
            const int e1 = br.e1 & 0xffff, q = e1 >> 2;
            const uint32_t tw = q == 0 ? t0 : q == 1 ? t1 : q == 2 ? t2 : t3;
            uint64_t pol;  // the tables stay in L2 ahead of streaming data (evict-last policy)
            asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
            asm volatile("ld.global.cg.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(c1)
                         : "l"(m1 + ((br.e1 >> 16) * S + ((tw >> (8 * (e1 & 3))) & 0xff)) * S + k), "l"(pol));
          }
          BondRec live = br;
          const int skip = br.n_cand0 + (has1 ? br.n_cand1 : 0);
          live.cand_off += skip;
          live.n_cand -= skip;
          ac = clash_sweep(p, w, pose, d, live, nx, ny, nz, pv, ck, sk, g, k, L, G, n_test, n_pair, alive);
          if (br.n_cand0 > 0 && k < S) ac += w.memo[memo_row0(S) + (b - memo_bonds(S)) * S + k];
          ac += c1;
        }
        const float V = (k < S) ? fmaf(p.clash_w, ac, ag) + 0.f : INF;  // + 0: -0 becomes +0
        // argmin over the group's lanes (ties: smaller k) by one min-reduction
        // of an order-preserving integer key and one ballot
        const unsigned vb = __float_as_uint(V);
        const unsigned key = vb ^ ((unsigned)((int)vb >> 31) | 0x80000000u);
        const unsigned gmask = L == 32 ? FULL : (((1u << L) - 1u) << glead);
        const unsigned kmin = __reduce_min_sync(gmask, key);
        const int bk1 = __ffs(__ballot_sync(FULL, key == kmin) & gmask) - 1 - glead;
        const int bk = alive ? bk1 : 0;  // a pruned group keeps its pose
        const float best = __uint_as_float((kmin & 0x80000000u) ? (kmin ^ 0x80000000u) : ~kmin);
        const float V0 = __shfl_sync(FULL, V, glead);
        const float cb = __shfl_sync(FULL, ck, glead + bk);
        const float sb = __shfl_sync(FULL, sk, glead + bk);
        E += best - V0;
        // the atoms fixed from now on at the chosen step join the bound's
        // first part; the rest may still reach their map minimum
        A += __shfl_sync(FULL, agf, glead + bk);
        if (alive && bb < d.n_rot && beyond_bound(A + w.lbc[bb], thr_use)) { alive = false; ++n_prn; }
        const uint32_t bits = (uint32_t)bk << (8 * (b & 3));
        switch (b >> 2) { case 0: t0 |= bits; break; case 1: t1 |= bits; break;
                          case 2: t2 |= bits; break; default: t3 |= bits; }
        __syncwarp();
        if (__any_sync(FULL, bk != 0)) {  // a group whose step is 0 applies the identity exactly
          Rot rb;
          rb.make(cb, sb, nx, ny, nz, pv.x, pv.y, pv.z);
          for (int i = br.v + 1 + k; i < br.end; i += L) {
            float4 q = pose[i];
            rb.apply(q.x, q.y, q.z, q.x, q.y, q.z);
            pose[i] = q;
          }
        }
        __syncwarp();
      }

      if (s0 + g >= item.s1) { n_atom = n_atom0; n_test = n_test0; n_pair = n_pair0; }

      // -- candidates of this start group into the warp's top-K (a pruned
      // start's energy exceeds the K-th best: it could not enter)
      for (int gg = 0; gg < G; ++gg) {
        const int src = gg * L;
        const float ce = __shfl_sync(FULL, E, src);
        const uint32_t c0 = __shfl_sync(FULL, t0, src), c1 = __shfl_sync(FULL, t1, src),
                       c2 = __shfl_sync(FULL, t2, src), c3 = __shfl_sync(FULL, t3, src);
        const bool live = __shfl_sync(FULL, alive, src);
        const int cs = __shfl_sync(FULL, sid, src);
        if (live) top.insert(ce, cs, c0, c1, c2, c3, K, lane);
      }
      thr = __shfl_sync(FULL, top.e, K - 1);
      if (row_thr && thr < thr_pub) {  // share an improved K-th best with the row's other items
        if (lane == 0) atomicMax(row_thr, ~value_key(thr));
        thr_pub = thr;
      }
    }

    if (p.stats) {  // one count per start group (its lane 0)
      unsigned long long a = k == 0 ? n_atom : 0, t = k == 0 ? n_test : 0, q = k == 0 ? n_pair : 0,
                         c = k == 0 ? n_cand : 0, r = k == 0 ? n_prn : 0, v = k == 0 ? n_bsw : 0;
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(FULL, a, o);
        t += __shfl_xor_sync(FULL, t, o);
        q += __shfl_xor_sync(FULL, q, o);
        c += __shfl_xor_sync(FULL, c, o);
        r += __shfl_xor_sync(FULL, r, o);
        v += __shfl_xor_sync(FULL, v, o);
      }
      if (lane == 0) {
        atomicAdd(p.stats + 0, a);
        atomicAdd(p.stats + 1, t);
        atomicAdd(p.stats + 2, q);
        atomicAdd(p.stats + 3, c);
        atomicAdd(p.stats + 4, r);
        atomicAdd(p.stats + 5, v);
      }
    }

    // -- publish this item's list; the last item of the ligand merges
    if (lane < K) {
      PoseOut o;
      o.score = top.e; o.start_id = top.s;
      o.tors[0] = top.t0; o.tors[1] = top.t1; o.tors[2] = top.t2; o.tors[3] = top.t3;
      p.partial[(size_t)item.slot * K + lane] = o;
    }
    __threadfence();
    __syncwarp();
    int prev = 0;
    if (lane == 0) prev = atomicAdd(p.done + item.row, 1);
    prev = __shfl_sync(FULL, prev, 0);
    if (prev != p.lig_items[item.row] - 1) continue;
    __threadfence();

    top.clear();
    const int slot0 = p.lig_slot0[item.row], nit = p.lig_items[item.row];
    for (int c = 0; c < nit; ++c) {
      const PoseOut *src = p.partial + (size_t)(slot0 + c) * K;
      float pe = INF;
      int ps = EMPTY_SID;
      uint32_t q0 = 0, q1 = 0, q2 = 0, q3 = 0;
      if (lane < K) {
        pe = __ldcg(&src[lane].score); ps = __ldcg(&src[lane].start_id);
        q0 = __ldcg(&src[lane].tors[0]); q1 = __ldcg(&src[lane].tors[1]);
        q2 = __ldcg(&src[lane].tors[2]); q3 = __ldcg(&src[lane].tors[3]);
      }
      for (int j = 0; j < K; ++j) {
        const float ce = __shfl_sync(FULL, pe, j);
        const int cs = __shfl_sync(FULL, ps, j);
        const uint32_t c0 = __shfl_sync(FULL, q0, j), c1 = __shfl_sync(FULL, q1, j),
                       c2 = __shfl_sync(FULL, q2, j), c3 = __shfl_sync(FULL, q3, j);
        if (cs != EMPTY_SID) top.insert(ce, cs, c0, c1, c2, c3, K, lane);
      }
    }
    __syncwarp();  // the ligand's partial lists are merged and dead: no write-back
    l2_discard(p.partial + (size_t)slot0 * K, p.partial + (size_t)(slot0 + nit) * K, lane);
    int rank = lane;
    if (p.rescore) {
      for (int j = 0; j < K; ++j) {
        const int cs = __shfl_sync(FULL, top.s, j);
        if (cs == EMPTY_SID) break;
        uint32_t tt[4];
        tt[0] = __shfl_sync(FULL, top.t0, j); tt[1] = __shfl_sync(FULL, top.t1, j);
        tt[2] = __shfl_sync(FULL, top.t2, j); tt[3] = __shfl_sync(FULL, top.t3, j);
        const float en = full_score<MODE_F32_PLAIN>(p, p.maps_f32, w, w.pose, d, cs, tt, lane);
        if (lane == j) top.e = en;
      }
      rank = 0;  // equal keys (empty slots) keep their lane order
      for (int j = 0; j < K; ++j) {
        const float oe = __shfl_sync(FULL, top.e, j);
        const int os = __shfl_sync(FULL, top.s, j);
        if (pose_less(oe, os, top.e, top.s) || (j < lane && !pose_less(top.e, top.s, oe, os))) ++rank;
      }
    }
    if (lane < K) {
      PoseOut o;
      o.score = top.e;
      o.start_id = top.s == EMPTY_SID ? -1 : top.s;
      o.tors[0] = top.t0; o.tors[1] = top.t1; o.tors[2] = top.t2; o.tors[3] = top.t3;
      p.out[(size_t)item.row * K + rank] = o;
    }
  }
}

// ---------------------------------------------------------------------------
// Explicit poses: one warp per pose.
template <int MODE>
__global__ void __launch_bounds__(256) score_poses_kernel(const DockParams p, int n_poses,
                                                          const int32_t *__restrict__ lig_idx,
                                                          const int32_t *__restrict__ start_id,
                                                          const uint8_t *__restrict__ tors,
                                                          float *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const WarpSmem w = warp_smem(smem_raw + (size_t)warp * smem_bytes_per_warp(p.nmax, 0, 1, 0), p.nmax, 1);
  const int pi = blockIdx.x * (blockDim.x >> 5) + warp;
  if (pi >= n_poses) return;
  const int li = lig_idx[pi], sid = start_id[pi];
  if (li < 0 || li >= p.n_ligands || sid < 0 || sid >= p.n_starts) {  // caller's device data
    if (lane == 0) out[pi] = __int_as_float(0x7fc00000);
    return;
  }
  LigDesc d;
  (void)load_ligand(p, w, li, d, lane);
  uint32_t tt[4];
  for (int q = 0; q < 4; ++q) {
    const uint8_t *t = tors + (size_t)pi * LIGATE_MAX_ROT + 4 * q;
    tt[q] = (uint32_t)t[0] | ((uint32_t)t[1] << 8) | ((uint32_t)t[2] << 16) | ((uint32_t)t[3] << 24);
  }
  const float e = full_score<MODE>(p, p.maps, w, w.pose, d, sid, tt, lane);
  if (lane == 0) out[pi] = e;
}

// ---------------------------------------------------------------------------
// Explicit poses' coordinates as every kernel builds them: one warp per pose,
// grid units, atoms written back in the ligand's input order.
__global__ void __launch_bounds__(256) pose_coords_kernel(const DockParams p, const uint8_t *__restrict__ order,
                                                          int n_poses, const int32_t *__restrict__ lig_idx,
                                                          const int32_t *__restrict__ start_id,
                                                          const uint8_t *__restrict__ tors,
                                                          float *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const WarpSmem w = warp_smem(smem_raw + (size_t)warp * smem_bytes_per_warp(p.nmax, 0, 1, 0), p.nmax, 1);
  const int pi = blockIdx.x * (blockDim.x >> 5) + warp;
  if (pi >= n_poses) return;
  float *o = out + (size_t)pi * LIGATE_MAX_ATOMS * 3;
  const int li = lig_idx[pi], sid = start_id[pi];
  if (li < 0 || li >= p.n_ligands || sid < 0 || sid >= p.n_starts) {  // caller's device data
    for (int q = lane; q < LIGATE_MAX_ATOMS * 3; q += 32) o[q] = __int_as_float(0x7fc00000);
    return;
  }
  LigDesc d;
  (void)load_ligand(p, w, li, d, lane);
  uint32_t tt[4];
  for (int q = 0; q < 4; ++q) {
    const uint8_t *t = tors + (size_t)pi * LIGATE_MAX_ROT + 4 * q;
    tt[q] = (uint32_t)t[0] | ((uint32_t)t[1] << 8) | ((uint32_t)t[2] << 16) | ((uint32_t)t[3] << 24);
  }
  build_pose<MODE_F32_PLAIN>(p, w, w.pose, d, sid, tt, lane);
  for (int i = lane; i < d.n_atoms; i += 32) {
    const float4 x = w.pose[i];
    float *a = o + 3 * (int)order[d.atom_base + i];
    a[0] = x.x; a[1] = x.y; a[2] = x.z;
  }
}

cudaError_t launch_pose_coords(const DockParams &p, const uint8_t *order, int n_poses, const int32_t *lig_idx,
                               const int32_t *start_id, const uint8_t *tors, float *out, cudaStream_t s) {
  if (n_poses <= 0) return cudaSuccess;
  const int warps = 4;
  const size_t smem = (size_t)warps * smem_bytes_per_warp(p.nmax, 0, 1, 0);
  cudaError_t e = cudaFuncSetAttribute(pose_coords_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       227 * 1024);
  if (e != cudaSuccess) return e;
  pose_coords_kernel<<<(n_poses + warps - 1) / warps, 32 * warps, smem, s>>>(p, order, n_poses, lig_idx,
                                                                            start_id, tors, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Start frames: rotation of each orientation quaternion (normalised, rows
// re-orthonormalised by Gram-Schmidt in FP32) scaled by 1/h, and anchors in
// grid units.
__global__ void start_frames_kernel(const float4 *__restrict__ quat, int n_orient,
                                    const float *__restrict__ anchors, int n_anchor, float ox,
                                    float oy, float oz, float inv_h, float *__restrict__ rot,
                                    float *__restrict__ anc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_orient) quat_frame(quat[i], inv_h, rot + 9 * i);
  if (i < n_anchor) {
    anc[3 * i] = (anchors[3 * i] - ox) * inv_h;
    anc[3 * i + 1] = (anchors[3 * i + 1] - oy) * inv_h;
    anc[3 * i + 2] = (anchors[3 * i + 2] - oz) * inv_h;
  }
}

// ---------------------------------------------------------------------------
// Kernel instance of a mode and register cap: reg_cap 1 = at most 85
// registers (6 CTAs of 128 threads per SM), 2 = at most 102 (5 CTAs), 3 = at
// most 128 (4 CTAs), 0 = the mode's default: 128 for the plain FP32 layout
// (eight scalar gathers per interpolation want registers for loads in
// flight), 102 for the corner layouts (one vector gather; occupancy wins).
static const void *dock_fn(int mode, int reg_cap) {
  const int minb = reg_cap == 1 ? 6 : reg_cap == 2 ? 5 : reg_cap == 3 ? 4 : (mode == MODE_F32_PLAIN ? 4 : 5);
  switch (mode * 3 + (minb - 4)) {
    case 0: return (const void *)dock_kernel<MODE_F32_PLAIN, 4>;
    case 1: return (const void *)dock_kernel<MODE_F32_PLAIN, 5>;
    case 2: return (const void *)dock_kernel<MODE_F32_PLAIN, 6>;
    case 3: return (const void *)dock_kernel<MODE_F32_CORNER, 4>;
    case 4: return (const void *)dock_kernel<MODE_F32_CORNER, 5>;
    case 5: return (const void *)dock_kernel<MODE_F32_CORNER, 6>;
    case 6: return (const void *)dock_kernel<MODE_BF16_CORNER, 4>;
    case 7: return (const void *)dock_kernel<MODE_BF16_CORNER, 5>;
    case 8: return (const void *)dock_kernel<MODE_BF16_CORNER, 6>;
    case 9: return (const void *)dock_kernel<MODE_F16_CORNER, 4>;
    case 10: return (const void *)dock_kernel<MODE_F16_CORNER, 5>;
    default: return (const void *)dock_kernel<MODE_F16_CORNER, 6>;
  }
}

cudaError_t launch_dock(int mode, int reg_cap, const DockParams &p, int grid, int block, size_t smem,
                        cudaStream_t s) {
  void *args[] = {(void *)&p};
  return cudaLaunchKernel(dock_fn(mode, reg_cap), dim3(grid), dim3(block), args, smem, s);
}

size_t dock_kernel_local_bytes(int mode, int reg_cap) {
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, dock_fn(mode, reg_cap)) != cudaSuccess) return 0;
  return a.localSizeBytes;
}

int dock_kernel_max_ctas_per_sm(int mode, int reg_cap, int block, size_t smem) {
  int n = 0;
  const void *f = dock_fn(mode, reg_cap);
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, block, smem) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_start_frames(const double *, const float *quat_f32_dev, int n_orient,
                                const float *anchors_dev, int n_anchor, const double origin[3],
                                double h, float *rot_out, float *anc_out, cudaStream_t s) {
  const int n = n_orient > n_anchor ? n_orient : n_anchor;
  start_frames_kernel<<<(n + 127) / 128, 128, 0, s>>>(
      reinterpret_cast<const float4 *>(quat_f32_dev), n_orient, anchors_dev, n_anchor,
      (float)origin[0], (float)origin[1], (float)origin[2], (float)(1.0 / h), rot_out, anc_out);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_score_t(const DockParams &p, int n_poses, const int32_t *lig_idx,
                                  const int32_t *start_id, const uint8_t *tors, float *out,
                                  cudaStream_t s) {
  const int warps = 4;
  const size_t smem = (size_t)warps * smem_bytes_per_warp(p.nmax, 0, 1, 0);
  cudaError_t e = cudaFuncSetAttribute(score_poses_kernel<MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e != cudaSuccess) return e;
  score_poses_kernel<MODE><<<(n_poses + warps - 1) / warps, 32 * warps, smem, s>>>(
      p, n_poses, lig_idx, start_id, tors, out);
  return cudaGetLastError();
}

cudaError_t launch_score_poses(int mode, const DockParams &p, int n_poses, const int32_t *lig_idx,
                               const int32_t *start_id, const uint8_t *tors, float *out,
                               cudaStream_t s) {
  if (n_poses <= 0) return cudaSuccess;
  switch (mode) {
    case MODE_F32_PLAIN: return launch_score_t<MODE_F32_PLAIN>(p, n_poses, lig_idx, start_id, tors, out, s);
    case MODE_F32_CORNER: return launch_score_t<MODE_F32_CORNER>(p, n_poses, lig_idx, start_id, tors, out, s);
    case MODE_BF16_CORNER: return launch_score_t<MODE_BF16_CORNER>(p, n_poses, lig_idx, start_id, tors, out, s);
    default: return launch_score_t<MODE_F16_CORNER>(p, n_poses, lig_idx, start_id, tors, out, s);
  }
}

}  // namespace ligate
