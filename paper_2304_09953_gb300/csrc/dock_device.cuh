// Device building blocks shared by the docking kernel (dock.cu) and the
// rescoring and pose-feature kernels (rescore.cu): trilinear map reads in
// every layout, rotations about a bond, the warp-distributed top-K list,
// the per-warp shared-memory slot, ligand loading, start frames and the
// construction and full scoring of a pose (paper Sec. 2: rigid start x
// torsion steps, geometric score = grid terms + intramolecular clash).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "ligate_internal.h"

namespace ligate {

constexpr unsigned FULL = 0xffffffffu;  // full-warp mask
constexpr int EMPTY_SID = 0x7fffffff;   // start id of an empty top-K slot

// ---------------------------------------------------------------------------
// Trilinear interpolation at grid coordinates (ux, uy, uz) of the map whose
// first element (plain) or cell (corner layouts) is at `toff`.  Outside
// [0, n-1] on any axis the atom scores the penalty.  Cell = min(floor, n-2),
// then successive linear interpolation along x, y, z.
//
// The cell index is taken without float/integer conversions (a slow pipe):
// for 0 <= u < 2^22, u + 2^23 rounded toward minus infinity is exactly
// 2^23 + floor(u) (FP32 spacing is 1 there), so its bit pattern minus that
// of 2^23 is floor(u), and (u + 2^23) - 2^23 is floor(u) as a float; the
// clamp to n - 2 is an FP32 min against 2^23 + n - 2 (GridConst cx, cy, cz).
// Inside the box the cell and the fraction equal those of (int)u exactly.
template <int MODE>
__device__ __forceinline__ float grid_eval(const void *__restrict__ maps, int toff, float ux,
                                           float uy, float uz, const GridConst &g) {
  if (!((ux >= 0.f) & (ux <= g.fx1) & (uy >= 0.f) & (uy <= g.fy1) & (uz >= 0.f) &
        (uz <= g.fz1)))
    return g.penalty;
  const float M23 = 8388608.f;
  const float tx = fminf(__fadd_rd(ux, M23), g.cx), ty = fminf(__fadd_rd(uy, M23), g.cy),
              tz = fminf(__fadd_rd(uz, M23), g.cz);
  const int ix = __float_as_int(tx) - 0x4B000000, iy = __float_as_int(ty) - 0x4B000000,
            iz = __float_as_int(tz) - 0x4B000000;
  const float fx = ux - (tx - M23), fy = uy - (ty - M23), fz = uz - (tz - M23);
  float v0, v1, v2, v3, v4, v5, v6, v7;
  if (MODE == MODE_F32_PLAIN) {
    const float *m = (const float *)maps + toff + (iz * g.ny + iy) * g.nx + ix;
    const int sy = g.nx, sz = g.nx * g.ny;
    v0 = __ldg(m); v1 = __ldg(m + 1); v2 = __ldg(m + sy); v3 = __ldg(m + sy + 1);
    v4 = __ldg(m + sz); v5 = __ldg(m + sz + 1); v6 = __ldg(m + sz + sy); v7 = __ldg(m + sz + sy + 1);
  } else {
    const int cell = toff + (iz * (g.ny - 1) + iy) * (g.nx - 1) + ix;  // < 2^28: host limit
    if (MODE == MODE_F32_CORNER) {
      const float4 *m = (const float4 *)maps + 2 * cell;
      const float4 a = __ldg(m), b = __ldg(m + 1);
      v0 = a.x; v1 = a.y; v2 = a.z; v3 = a.w; v4 = b.x; v5 = b.y; v6 = b.z; v7 = b.w;
    } else {
      const uint4 w = __ldg((const uint4 *)maps + cell);
      if (MODE == MODE_BF16_CORNER) {
        v0 = __uint_as_float(w.x << 16); v1 = __uint_as_float(w.x & 0xffff0000u);
        v2 = __uint_as_float(w.y << 16); v3 = __uint_as_float(w.y & 0xffff0000u);
        v4 = __uint_as_float(w.z << 16); v5 = __uint_as_float(w.z & 0xffff0000u);
        v6 = __uint_as_float(w.w << 16); v7 = __uint_as_float(w.w & 0xffff0000u);
      } else {
        float2 f;
        f = __half22float2(*reinterpret_cast<const __half2 *>(&w.x)); v0 = f.x; v1 = f.y;
        f = __half22float2(*reinterpret_cast<const __half2 *>(&w.y)); v2 = f.x; v3 = f.y;
        f = __half22float2(*reinterpret_cast<const __half2 *>(&w.z)); v4 = f.x; v5 = f.y;
        f = __half22float2(*reinterpret_cast<const __half2 *>(&w.w)); v6 = f.x; v7 = f.y;
      }
    }
  }
  const float y0z0 = fmaf(fx, v1 - v0, v0);
  const float y1z0 = fmaf(fx, v3 - v2, v2);
  const float y0z1 = fmaf(fx, v5 - v4, v4);
  const float y1z1 = fmaf(fx, v7 - v6, v6);
  const float z0 = fmaf(fy, y1z0 - y0z0, y0z0);
  const float z1 = fmaf(fy, y1z1 - y0z1, y0z1);
  return fmaf(fz, z1 - z0, z0);
}


// Two atoms at once with packed FP32 (FFMA2 / FADD2: per component the same
// rounding as fmaf / the scalar add, so each value equals grid_eval's).
template <int MODE>
__device__ __forceinline__ void load_corners(const void *__restrict__ maps, int toff, int ix, int iy, int iz,
                                             const GridConst &g, float (&v)[8]) {
  if (MODE == MODE_F32_PLAIN) {
    const float *m = (const float *)maps + toff + (iz * g.ny + iy) * g.nx + ix;
    const int sy = g.nx, sz = g.nx * g.ny;
    v[0] = __ldg(m); v[1] = __ldg(m + 1); v[2] = __ldg(m + sy); v[3] = __ldg(m + sy + 1);
    v[4] = __ldg(m + sz); v[5] = __ldg(m + sz + 1); v[6] = __ldg(m + sz + sy); v[7] = __ldg(m + sz + sy + 1);
  } else {
    const int cell = toff + (iz * (g.ny - 1) + iy) * (g.nx - 1) + ix;
    if (MODE == MODE_F32_CORNER) {
      const float4 *m = (const float4 *)maps + 2 * cell;
      const float4 a = __ldg(m), b = __ldg(m + 1);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
      const uint4 w = __ldg((const uint4 *)maps + cell);
      if (MODE == MODE_BF16_CORNER) {
        v[0] = __uint_as_float(w.x << 16); v[1] = __uint_as_float(w.x & 0xffff0000u);
        v[2] = __uint_as_float(w.y << 16); v[3] = __uint_as_float(w.y & 0xffff0000u);
        v[4] = __uint_as_float(w.z << 16); v[5] = __uint_as_float(w.z & 0xffff0000u);
        v[6] = __uint_as_float(w.w << 16); v[7] = __uint_as_float(w.w & 0xffff0000u);
      } else {
        float2 f;
        f = __half22float2(*reinterpret_cast<const __half2 *>(&w.x)); v[0] = f.x; v[1] = f.y;
        f = __half22float2(*reinterpret_cast<const __half2 *>(&w.y)); v[2] = f.x; v[3] = f.y;
        f = __half22float2(*reinterpret_cast<const __half2 *>(&w.z)); v[4] = f.x; v[5] = f.y;
        f = __half22float2(*reinterpret_cast<const __half2 *>(&w.w)); v[6] = f.x; v[7] = f.y;
      }
    }
  }
}

__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

template <int MODE>
__device__ __forceinline__ float2 grid_eval2(const void *__restrict__ maps, int toffa, float ax, float ay, float az,
                                             int toffb, float bx, float by, float bz, const GridConst &g) {
  const bool ina = (ax >= 0.f) & (ax <= g.fx1) & (ay >= 0.f) & (ay <= g.fy1) & (az >= 0.f) & (az <= g.fz1);
  const bool inb = (bx >= 0.f) & (bx <= g.fx1) & (by >= 0.f) & (by <= g.fy1) & (bz >= 0.f) & (bz <= g.fz1);
  const float M23 = 8388608.f;
  const float txa = fminf(__fadd_rd(ax, M23), g.cx), tya = fminf(__fadd_rd(ay, M23), g.cy),
              tza = fminf(__fadd_rd(az, M23), g.cz);
  const float txb = fminf(__fadd_rd(bx, M23), g.cx), tyb = fminf(__fadd_rd(by, M23), g.cy),
              tzb = fminf(__fadd_rd(bz, M23), g.cz);
  const int ixa = ina ? __float_as_int(txa) - 0x4B000000 : 0, iya = ina ? __float_as_int(tya) - 0x4B000000 : 0,
            iza = ina ? __float_as_int(tza) - 0x4B000000 : 0;
  const int ixb = inb ? __float_as_int(txb) - 0x4B000000 : 0, iyb = inb ? __float_as_int(tyb) - 0x4B000000 : 0,
            izb = inb ? __float_as_int(tzb) - 0x4B000000 : 0;
  const float2 m23 = make_float2(M23, M23);
  const float2 fx = sub2(make_float2(ax, bx), sub2(make_float2(txa, txb), m23));
  const float2 fy = sub2(make_float2(ay, by), sub2(make_float2(tya, tyb), m23));
  const float2 fz = sub2(make_float2(az, bz), sub2(make_float2(tza, tzb), m23));
  float va[8], vb[8];
  load_corners<MODE>(maps, ina ? toffa : 0, ixa, iya, iza, g, va);
  load_corners<MODE>(maps, inb ? toffb : 0, ixb, iyb, izb, g, vb);
  const float2 v0 = make_float2(va[0], vb[0]), v1 = make_float2(va[1], vb[1]), v2 = make_float2(va[2], vb[2]),
               v3 = make_float2(va[3], vb[3]), v4 = make_float2(va[4], vb[4]), v5 = make_float2(va[5], vb[5]),
               v6 = make_float2(va[6], vb[6]), v7 = make_float2(va[7], vb[7]);
  const float2 y0z0 = __ffma2_rn(fx, sub2(v1, v0), v0);
  const float2 y1z0 = __ffma2_rn(fx, sub2(v3, v2), v2);
  const float2 y0z1 = __ffma2_rn(fx, sub2(v5, v4), v4);
  const float2 y1z1 = __ffma2_rn(fx, sub2(v7, v6), v6);
  const float2 z0 = __ffma2_rn(fy, sub2(y1z0, y0z0), y0z0);
  const float2 z1 = __ffma2_rn(fy, sub2(y1z1, y0z1), y0z1);
  const float2 r = __ffma2_rn(fz, sub2(z1, z0), z0);
  return make_float2(ina ? r.x : g.penalty, inb ? r.y : g.penalty);
}

// Element stride of one atom type's map in a given mode (plain: nodes;
// corner: cells).
__host__ __device__ inline int type_stride(int mode, const GridConst &g) {
  return mode == MODE_F32_PLAIN ? g.nx * g.ny * g.nz : (g.nx - 1) * (g.ny - 1) * (g.nz - 1);
}

// Rotation by angle (c = cos, s = sin) about unit axis n through point p:
// y = R x + t, with R = c I + s [n]x + (1 - c) n n^T and t = p - R p.
struct Rot {
  float r00, r01, r02, r10, r11, r12, r20, r21, r22, tx, ty, tz;
  __device__ __forceinline__ void make(float c, float s, float nx, float ny, float nz, float px,
                                       float py, float pz) {
    const float o = 1.f - c;
    r00 = fmaf(o * nx, nx, c);       r01 = fmaf(o * nx, ny, -s * nz); r02 = fmaf(o * nx, nz, s * ny);
    r10 = fmaf(o * ny, nx, s * nz);  r11 = fmaf(o * ny, ny, c);       r12 = fmaf(o * ny, nz, -s * nx);
    r20 = fmaf(o * nz, nx, -s * ny); r21 = fmaf(o * nz, ny, s * nx);  r22 = fmaf(o * nz, nz, c);
    tx = px - fmaf(r00, px, fmaf(r01, py, r02 * pz));
    ty = py - fmaf(r10, px, fmaf(r11, py, r12 * pz));
    tz = pz - fmaf(r20, px, fmaf(r21, py, r22 * pz));
  }
  __device__ __forceinline__ void apply(float x, float y, float z, float &ox, float &oy,
                                        float &oz) const {
    ox = fmaf(r00, x, fmaf(r01, y, fmaf(r02, z, tx)));
    oy = fmaf(r10, x, fmaf(r11, y, fmaf(r12, z, ty)));
    oz = fmaf(r20, x, fmaf(r21, y, fmaf(r22, z, tz)));
  }
};

// Unit axis from atom u to atom v of a pose.
__device__ __forceinline__ void bond_axis(const float4 &pu, const float4 &pv, float &nx, float &ny,
                                          float &nz) {
  nx = pv.x - pu.x; ny = pv.y - pu.y; nz = pv.z - pu.z;
  const float inv = rsqrtf(fmaf(nx, nx, fmaf(ny, ny, nz * nz)));
  nx *= inv; ny *= inv; nz *= inv;
}

// (E, s) lexicographic order; an empty slot is (+inf, EMPTY_SID).
__device__ __forceinline__ bool pose_less(float e1, int s1, float e2, int s2) {
  return e1 < e2 || (e1 == e2 && s1 < s2);
}

// Warp-distributed sorted top-K list: lane j < K holds entry j.
struct TopK {
  float e;
  int s;
  uint32_t t0, t1, t2, t3;
  __device__ __forceinline__ void clear() {
    e = __int_as_float(0x7f800000); s = EMPTY_SID; t0 = t1 = t2 = t3 = 0;
  }
  // Insert a warp-uniform candidate (all lanes pass the same values).
  __device__ __forceinline__ void insert(float ce, int cs, uint32_t c0, uint32_t c1, uint32_t c2,
                                         uint32_t c3, int K, int lane) {
    const float ke = __shfl_sync(FULL, e, K - 1);
    const int ks = __shfl_sync(FULL, s, K - 1);
    if (!pose_less(ce, cs, ke, ks)) return;  // warp-uniform
    const bool before = lane < K && pose_less(e, s, ce, cs);
    const int pos = __popc(__ballot_sync(FULL, before));
    const float ue = __shfl_up_sync(FULL, e, 1);
    const int us = __shfl_up_sync(FULL, s, 1);
    const uint32_t u0 = __shfl_up_sync(FULL, t0, 1), u1 = __shfl_up_sync(FULL, t1, 1),
                   u2 = __shfl_up_sync(FULL, t2, 1), u3 = __shfl_up_sync(FULL, t3, 1);
    if (lane > pos && lane < K) { e = ue; s = us; t0 = u0; t1 = u1; t2 = u2; t3 = u3; }
    if (lane == pos) { e = ce; s = cs; t0 = c0; t1 = c1; t2 = c2; t3 = c3; }
  }
};

// Per-warp shared-memory slot.
struct WarpSmem {
  float4 *ref;     // [nmax]  (x - c, y - c, z - c) Angstrom, .w = atom type (int bits)
  float4 *pose;    // [G][nmax + 1] current pose, grid units, .w = map offset (int bits)
  float4 *list;    // [PAIR_WARP] clash pairs that survive the circle bound of a bond
  float2 *cab;     // [G][nmax] (axial coordinate, radial distance) about the bond axis
  BondRec *bonds;  // [LIGATE_MAX_ROT]
  float *lbc;      // [LBC_FLOATS] per sweep stage b: sum of the map minima of the atoms bonds >= b move
  uint8_t *lastb;  // [nmax] 1 + the last bond that moves each atom (0: no bond moves it)
  float *memo;     // [memo_floats(S, rmax)] clash sums that every start shares
};

// floats of WarpSmem::lbc (LIGATE_MAX_ROT + 1 stages, padded to 16 bytes)
constexpr int LBC_FLOATS = (LIGATE_MAX_ROT + 1 + 3) / 4 * 4;

// Surviving clash pairs buffered per warp before they are evaluated for
// every torsion step: 192 entries, 192 / G = 6 L per start group (the
// buffer is flushed whenever a group may overflow).
constexpr int PAIR_WARP = 192;

// The clash term of a bond's sweep depends only on the ligand's internal
// conformation, which before bond b is set by the steps chosen at bonds
// 0 .. b-1.  Bond 0 therefore sweeps the same conformation for every start
// and bond 1 one of S conformations: their clash sums are computed once per
// ligand (S values for bond 0, S x S for bond 1 when S <= 16) and looked up
// by every start.  Of a later bond b, the pairs no earlier bond separates
// (the first n_cand0 candidates) have the same geometry in every start's
// sweep too: their sums are one row of S values per bond, the rest of the
// pairs are swept live.
__host__ __device__ inline int memo_bonds(int S) { return S <= 16 ? 2 : 1; }
__host__ __device__ inline int memo_rows(int S, int rmax) { return rmax > memo_bonds(S) ? rmax - memo_bonds(S) : 0; }
// first float of the rows of bonds memo_bonds(S), memo_bonds(S) + 1, ...
__host__ __device__ inline int memo_row0(int S) { return S + (memo_bonds(S) == 2 ? S * S : 0); }
__host__ __device__ inline int memo_floats(int S, int rmax) {
  return S <= 0 ? 0 : (memo_row0(S) + memo_rows(S, rmax) * S + 3) / 4 * 4;
}

// `list` pair-list entries (PAIR_WARP for kernels that sweep clash pairs or
// keep a histogram there, 0 for those that need neither).
__host__ __device__ inline size_t smem_bytes_per_warp(int nmax, int S, int G, int rmax, int list = PAIR_WARP) {
  return (size_t)nmax * 16 + (size_t)G * (nmax + 1) * 16 + (size_t)list * 16 +
         (size_t)G * nmax * 8 + sizeof(BondRec) * LIGATE_MAX_ROT + (size_t)LBC_FLOATS * 4 +
         (size_t)((nmax + 15) & ~15) + (size_t)memo_floats(S, rmax) * 4;
}


__device__ __forceinline__ WarpSmem warp_smem(unsigned char *base, int nmax, int G, int list = PAIR_WARP) {
  WarpSmem w;
  w.ref = reinterpret_cast<float4 *>(base);
  w.pose = w.ref + nmax;
  w.list = w.pose + (size_t)G * (nmax + 1);
  w.cab = reinterpret_cast<float2 *>(w.list + list);
  w.bonds = reinterpret_cast<BondRec *>(w.cab + (size_t)G * nmax);
  w.lbc = reinterpret_cast<float *>(w.bonds + LIGATE_MAX_ROT);
  w.lastb = reinterpret_cast<uint8_t *>(w.lbc + LBC_FLOATS);
  w.memo = reinterpret_cast<float *>(w.lastb + ((nmax + 15) & ~15));
  return w;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Load ligand `li` into the warp's slot: reference coordinates centred on
// their centroid, bond table, clash masks.  Returns the clash sum (without
// the weight) of the input conformation, which every pose shares up to the
// torsion-dependent part.
__device__ inline float load_ligand(const DockParams &p, const WarpSmem &w, int li, LigDesc &d,
                             int lane) {
  d = p.lig[li];
  float sx = 0.f, sy = 0.f, sz = 0.f;
  for (int i = lane; i < d.n_atoms; i += 32) {
    const float4 a = __ldg(p.atoms + d.atom_base + i);
    w.ref[i] = a;
    sx += a.x; sy += a.y; sz += a.z;
  }
  sx = warp_sum(sx); sy = warp_sum(sy); sz = warp_sum(sz);
  const float inv_n = 1.f / (float)d.n_atoms;
  const float cx = sx * inv_n, cy = sy * inv_n, cz = sz * inv_n;
  __syncwarp();
  for (int i = lane; i < d.n_atoms; i += 32) {
    float4 a = w.ref[i];
    a.x -= cx; a.y -= cy; a.z -= cz;
    w.ref[i] = a;
  }
  for (int b = lane; b < d.n_rot; b += 32) w.bonds[b] = p.bonds[d.bond_base + b];
  __syncwarp();
  float cl = 0.f;
  for (int i = lane; i < d.n_atoms; i += 32) {
    const float4 xi = w.ref[i];
    for (int wd = 0; wd < d.n_words; ++wd) {
      uint32_t m = __ldg(p.elig + d.elig_base + i * d.n_words + wd);
      const int lo = i + 1 - 32 * wd;  // keep only j > i
      if (lo >= 32) m = 0; else if (lo > 0) m &= ~0u << lo;
      while (m) {
        const int j = 32 * wd + __ffs(m) - 1;
        m &= m - 1;
        const float4 xj = w.ref[j];
        const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
        const float t = fmaxf(0.f, fmaf(-fmaf(dx, dx, fmaf(dy, dy, dz * dz)), p.inv_dc2_ang, 1.f));
        cl = fmaf(t, t, cl);
      }
    }
  }
  return warp_sum(cl);
}

// Rigid start frame: rows of R_o / h and (anchor - origin) / h.
__device__ __forceinline__ void start_frame(const DockParams &p, int sid, float (&R)[9],
                                            float (&T)[3]) {
  const int o = sid / p.n_anchor, a = sid - o * p.n_anchor;
#pragma unroll
  for (int q = 0; q < 9; ++q) R[q] = __ldg(p.rot + 9 * o + q);
#pragma unroll
  for (int q = 0; q < 3; ++q) T[q] = __ldg(p.anc + 3 * a + q);
}

// Start frame of one orientation: quaternion (w, x, y, z) normalised, the
// rows of its rotation re-orthonormalised by Gram-Schmidt in FP32, scaled by
// 1/h (row-major into rot[9]).
__device__ __forceinline__ void quat_frame(float4 q, float inv_h, float *__restrict__ rot) {
  const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
  float r0[3] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)};
  float r1[3] = {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)};
  float n0 = rsqrtf(r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]);
  for (int a = 0; a < 3; ++a) r0[a] *= n0;
  const float dp = r0[0] * r1[0] + r0[1] * r1[1] + r0[2] * r1[2];
  for (int a = 0; a < 3; ++a) r1[a] -= dp * r0[a];
  const float n1 = rsqrtf(r1[0] * r1[0] + r1[1] * r1[1] + r1[2] * r1[2]);
  for (int a = 0; a < 3; ++a) r1[a] *= n1;
  const float r2[3] = {r0[1] * r1[2] - r0[2] * r1[1], r0[2] * r1[0] - r0[0] * r1[2],
                       r0[0] * r1[1] - r0[1] * r1[0]};
  for (int a = 0; a < 3; ++a) {
    rot[a] = r0[a] * inv_h;
    rot[3 + a] = r1[a] * inv_h;
    rot[6 + a] = r2[a] * inv_h;
  }
}

// cos/sin of 2 pi k / S from the run's table (FP64 on the host, rounded).
__device__ __forceinline__ void step_cs(const DockParams &p, int k, float &c, float &s) {
  c = p.cs_tab[2 * k];
  s = p.cs_tab[2 * k + 1];
}

// Coordinates (grid units, .w = map offset of the atom's type for map
// layout MODE) of pose (sid, tors) of the loaded ligand into buf:
// rigid start frame, then each bond's step about its current axis.
// Warp-cooperative.
template <int MODE>
__device__ void build_pose(const DockParams &p, const WarpSmem &w, float4 *buf, const LigDesc &d, int sid,
                           const uint32_t (&tors)[4], int lane) {
  float R[9], T[3];
  start_frame(p, sid, R, T);
  const int ts = type_stride(MODE, p.g);
  for (int i = lane; i < d.n_atoms; i += 32) {
    const float4 r = w.ref[i];
    float4 u;
    u.x = fmaf(R[0], r.x, fmaf(R[1], r.y, fmaf(R[2], r.z, T[0])));
    u.y = fmaf(R[3], r.x, fmaf(R[4], r.y, fmaf(R[5], r.z, T[1])));
    u.z = fmaf(R[6], r.x, fmaf(R[7], r.y, fmaf(R[8], r.z, T[2])));
    u.w = __int_as_float(__float_as_int(r.w) * ts);
    buf[i] = u;
  }
  __syncwarp();
  for (int b = 0; b < d.n_rot; ++b) {
    const int kb = (tors[b >> 2] >> (8 * (b & 3))) & 0xff;
    if (kb % p.S == 0) continue;
    const BondRec br = w.bonds[b];
    float nx, ny, nz;
    const float4 pv = buf[br.v];
    bond_axis(buf[br.u], pv, nx, ny, nz);
    float c, s;
    step_cs(p, kb % p.S, c, s);
    Rot rot;
    rot.make(c, s, nx, ny, nz, pv.x, pv.y, pv.z);
    __syncwarp();
    for (int i = br.v + 1 + lane; i < br.end; i += 32) {
      float4 q = buf[i];
      rot.apply(q.x, q.y, q.z, q.x, q.y, q.z);
      buf[i] = q;
    }
    __syncwarp();
  }
}

// Angstrom coordinates of continuous state (R, t, phi) of the loaded ligand
// into buf: starting from its centred input coordinates `ref` (.w kept),
// each rotatable bond in sweep order turns its subtree by phi_b (radians,
// skipped when exactly 0) about its current axis u -> v, then x = R y + t.
// The refinement, the exact rescoring of states and ligate_state_coords all
// build states with this function, so they see the same FP32 geometry.
// Warp-cooperative.
__device__ inline void build_state(const float4 *ref, float4 *buf, const BondRec *bonds, const LigDesc &d,
                                   const float *R, const float *T, const float *phi, int lane) {
  for (int i = lane; i < d.n_atoms; i += 32) buf[i] = ref[i];
  __syncwarp();
  for (int b = 0; b < d.n_rot; ++b) {
    const float ang = phi[b];
    if (ang == 0.f) continue;
    const BondRec br = bonds[b];
    float nx, ny, nz;
    const float4 pv = buf[br.v];
    bond_axis(buf[br.u], pv, nx, ny, nz);
    float sn, cs;
    sincosf(ang, &sn, &cs);
    Rot rot;
    rot.make(cs, sn, nx, ny, nz, pv.x, pv.y, pv.z);
    __syncwarp();
    for (int i = br.v + 1 + lane; i < br.end; i += 32) {
      float4 q = buf[i];
      rot.apply(q.x, q.y, q.z, q.x, q.y, q.z);
      buf[i] = q;
    }
    __syncwarp();
  }
  for (int i = lane; i < d.n_atoms; i += 32) {
    const float4 y = buf[i];
    float4 x;
    x.x = fmaf(R[0], y.x, fmaf(R[1], y.y, fmaf(R[2], y.z, T[0])));
    x.y = fmaf(R[3], y.x, fmaf(R[4], y.y, fmaf(R[5], y.z, T[1])));
    x.z = fmaf(R[6], y.x, fmaf(R[7], y.y, fmaf(R[8], y.z, T[2])));
    x.w = y.w;
    buf[i] = x;
  }
  __syncwarp();
}

// Full FP32 score of pose (sid, tors) of the loaded ligand, warp-cooperative,
// using the map `maps` read in mode MODE (scratch: pose slot `buf`).
template <int MODE>
__device__ float full_score(const DockParams &p, const void *maps, const WarpSmem &w, float4 *buf,
                            const LigDesc &d, int sid, const uint32_t (&tors)[4], int lane) {
  build_pose<MODE>(p, w, buf, d, sid, tors, lane);
  float e = 0.f, cl = 0.f;
  for (int i = lane; i < d.n_atoms; i += 32) {
    const float4 xi = buf[i];
    e += grid_eval<MODE>(maps, __float_as_int(xi.w), xi.x, xi.y, xi.z, p.g);
    for (int wd = 0; wd < d.n_words; ++wd) {
      uint32_t m = __ldg(p.elig + d.elig_base + i * d.n_words + wd);
      const int lo = i + 1 - 32 * wd;
      if (lo >= 32) m = 0; else if (lo > 0) m &= ~0u << lo;
      while (m) {
        const int j = 32 * wd + __ffs(m) - 1;
        m &= m - 1;
        const float4 xj = buf[j];
        const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
        const float t = fmaxf(0.f, fmaf(-fmaf(dx, dx, fmaf(dy, dy, dz * dz)), p.inv_dc2_grid, 1.f));
        cl = fmaf(t, t, cl);
      }
    }
  }
  e = warp_sum(e);
  cl = warp_sum(cl);
  __syncwarp();
  return fmaf(p.clash_w, cl, e);
}

}  // namespace ligate
