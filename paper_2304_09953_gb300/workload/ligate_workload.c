/*
 * Seeded synthetic workload generator for ligand docking (host, FP64).
 *
 * This file produces INPUTS only: ligand trees with 3D coordinates, receptor
 * atoms, per-atom-type grid maps computed from them, pocket anchor points and
 * orientation quaternions.  It holds none of the docking method's arithmetic
 * (no pose construction, no interpolation, no scoring), so both the FP64
 * oracle and the CUDA path can consume what it writes without sharing code.
 *
 * Every random draw comes from SplitMix64 (Steele, Lea & Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014), one independent
 * stream per ligand / per object, so any ligand of a library can be
 * regenerated alone.  Only IEEE-exact operations (+ - * / sqrt) are used on
 * values that reach an output, and the file is compiled with
 * -ffp-contract=off, so x86-64 and aarch64 hosts write identical bytes.
 *
 * The workload recipe (tree growth rules, receptor shell, Lennard-Jones-like
 * map with a cap) stands in for the paper's real chemical libraries and PDB
 * targets (Sec. 2: SMILES library, 3D preparation, PDB target), which are not
 * available; the recipe itself is fixed by the synthetic benchmark definition.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define LW_EXPORT __attribute__((visibility("default")))

/* ---- SplitMix64 --------------------------------------------------------- */
static inline uint64_t sm64_next(uint64_t *s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
/* Independent stream for (seed, tag, index). */
static inline uint64_t sm64_stream(uint64_t seed, uint64_t tag, uint64_t index) {
  uint64_t s = seed ^ (tag * 0xD1B54A32D192ED03ULL);
  (void)sm64_next(&s);
  s ^= index * 0x8CB92BA72F3D8DD7ULL;
  (void)sm64_next(&s);
  return s;
}
/* Uniform double in [0, 1) with 53 random bits. */
static inline double u01(uint64_t *s) { return (double)(sm64_next(s) >> 11) * 0x1.0p-53; }
/* Uniform integer in [0, n). */
static inline int uint_below(uint64_t *s, int n) {
  int v = (int)(u01(s) * (double)n);
  return v < n ? v : n - 1;
}
/* Uniform point in the unit ball (rejection from the cube). */
static void unit_ball(uint64_t *s, double v[3]) {
  for (;;) {
    double x = 2.0 * u01(s) - 1.0, y = 2.0 * u01(s) - 1.0, z = 2.0 * u01(s) - 1.0;
    double r2 = x * x + y * y + z * z;
    if (r2 <= 1.0) { v[0] = x; v[1] = y; v[2] = z; return; }
  }
}
/* Uniform direction on the unit sphere. */
static void unit_dir(uint64_t *s, double v[3]) {
  for (;;) {
    double b[3];
    unit_ball(s, b);
    double r2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    if (r2 > 1e-6) {
      double r = sqrt(r2);
      v[0] = b[0] / r; v[1] = b[1] / r; v[2] = b[2] / r;
      return;
    }
  }
}

enum { TAG_SIZES = 1, TAG_LIGAND = 2, TAG_RECEPTOR = 3, TAG_TYPES = 4, TAG_ANCHORS = 5,
       TAG_ORIENT = 6, TAG_NORMAL = 7 };

/* ---- ligand sizes --------------------------------------------------------
 * kind 0: N uniform on {nmin..nmax}; kind 1: P(N) proportional to 1/N on
 * {nmin..nmax} (discrete log-uniform).  Requested rotatable-bond counts are
 * uniform on {rmin..rmax}; the generator caps them at what the tree offers. */
LW_EXPORT int lw_ligand_sizes(uint64_t seed, int n, int kind, int nmin, int nmax, int rmin,
                              int rmax, int *n_atoms, int *n_rot_req) {
  if (n < 0 || nmin < 1 || nmax < nmin || rmin < 0 || rmax < rmin) return -1;
  int span = nmax - nmin + 1;
  double *cdf = NULL;
  if (kind == 1) {
    cdf = (double *)malloc(sizeof(double) * (size_t)span);
    if (!cdf) return -2;
    double acc = 0.0;
    for (int k = 0; k < span; ++k) { acc += 1.0 / (double)(nmin + k); cdf[k] = acc; }
    for (int k = 0; k < span; ++k) cdf[k] /= acc;
  }
  for (int i = 0; i < n; ++i) {
    uint64_t s = sm64_stream(seed, TAG_SIZES, (uint64_t)i);
    if (kind == 1) {
      double u = u01(&s);
      int k = 0;
      while (k < span - 1 && u >= cdf[k]) ++k;
      n_atoms[i] = nmin + k;
    } else {
      n_atoms[i] = nmin + uint_below(&s, span);
    }
    n_rot_req[i] = rmin + uint_below(&s, rmax - rmin + 1);
  }
  free(cdf);
  return 0;
}

/* ---- one ligand tree -----------------------------------------------------
 * Atom 0 sits at the origin; atom i > 0 bonds to a random earlier atom of
 * degree < 4, at 1.5 A, along a direction making at least 100 degrees with
 * the parent's existing bonds and keeping every non-bonded atom at least
 * 2.0 A away.  After 100 failed draws for one atom the whole ligand is drawn
 * again.  Rotatable bonds are picked uniformly among non-terminal bonds (both
 * ends of degree >= 2); if fewer exist than requested, all are used.
 * Writes xyz[n][3] (FP32), type[n], bonds[n-1][2] (parent, child),
 * rotatable[n-1]; returns the realised rotatable count, or -1. */
static int gen_one_ligand(uint64_t s, int n, int r_req, int n_types, float *xyz_out,
                          uint8_t *type_out, int *bonds_out, uint8_t *rot_out) {
  const double bond = 1.5, min_nb2 = 2.0 * 2.0;
  const double cos_max = -0.17364817766693033; /* cos(100 deg) */
  double *pos = (double *)malloc(sizeof(double) * 3 * (size_t)n);
  int *deg = (int *)malloc(sizeof(int) * (size_t)n);
  int *par = (int *)malloc(sizeof(int) * (size_t)n);
  int *cand = (int *)malloc(sizeof(int) * (size_t)n);
  int *nb = (int *)malloc(sizeof(int) * 4 * (size_t)n);
  int realised = -1;
  if (!pos || !deg || !par || !cand || !nb) goto done;
  for (int whole = 0; whole < 1000; ++whole) {
    int ok_all = 1;
    pos[0] = pos[1] = pos[2] = 0.0;
    deg[0] = 0; par[0] = -1;
    for (int i = 1; i < n && ok_all; ++i) {
      int placed = 0;
      for (int attempt = 0; attempt < 100 && !placed; ++attempt) {
        int nc = 0;
        for (int j = 0; j < i; ++j) if (deg[j] < 4) cand[nc++] = j;
        int p = cand[uint_below(&s, nc)];
        double d[3];
        unit_dir(&s, d);
        int ok = 1;
        for (int q = 0; q < deg[p] && ok; ++q) {
          int o = nb[4 * p + q];
          double e[3] = {pos[3 * o] - pos[3 * p], pos[3 * o + 1] - pos[3 * p + 1],
                         pos[3 * o + 2] - pos[3 * p + 2]};
          double el = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
          double c = (d[0] * e[0] + d[1] * e[1] + d[2] * e[2]) / el;
          if (c > cos_max) ok = 0;
        }
        double x[3] = {pos[3 * p] + bond * d[0], pos[3 * p + 1] + bond * d[1],
                       pos[3 * p + 2] + bond * d[2]};
        for (int j = 0; j < i && ok; ++j) {
          if (j == p) continue;
          double dx = x[0] - pos[3 * j], dy = x[1] - pos[3 * j + 1], dz = x[2] - pos[3 * j + 2];
          if (dx * dx + dy * dy + dz * dz < min_nb2) ok = 0;
        }
        if (!ok) continue;
        pos[3 * i] = x[0]; pos[3 * i + 1] = x[1]; pos[3 * i + 2] = x[2];
        par[i] = p; deg[i] = 1; nb[4 * i] = p;
        nb[4 * p + deg[p]] = i; deg[p] += 1;
        placed = 1;
      }
      if (!placed) ok_all = 0;
    }
    if (!ok_all) continue;
    for (int i = 0; i < n; ++i) {
      xyz_out[3 * i] = (float)pos[3 * i];
      xyz_out[3 * i + 1] = (float)pos[3 * i + 1];
      xyz_out[3 * i + 2] = (float)pos[3 * i + 2];
      type_out[i] = (uint8_t)uint_below(&s, n_types);
    }
    int nnt = 0;
    for (int i = 1; i < n; ++i) {
      bonds_out[2 * (i - 1)] = par[i];
      bonds_out[2 * (i - 1) + 1] = i;
      rot_out[i - 1] = 0;
      if (deg[par[i]] >= 2 && deg[i] >= 2) cand[nnt++] = i - 1;
    }
    int r = r_req < nnt ? r_req : nnt;
    for (int k = 0; k < r; ++k) { /* partial Fisher-Yates */
      int j = k + uint_below(&s, nnt - k);
      int t = cand[k]; cand[k] = cand[j]; cand[j] = t;
      rot_out[cand[k]] = 1;
    }
    realised = r;
    break;
  }
done:
  free(pos); free(deg); free(par); free(cand); free(nb);
  return realised;
}

/* Library of n ligands; ligand i uses stream (seed, LIGAND, first_index + i).
 * atom_offset[n+1] and bond_offset[n+1] must already hold prefix sums of
 * n_atoms and n_atoms-1 (see lw_offsets).  r_real[i] receives the realised
 * rotatable count.  Returns 0 or the negative index-1 of a failed ligand. */
LW_EXPORT int lw_ligands(uint64_t seed, int64_t first_index, int n, int n_types,
                         const int *n_atoms, const int *n_rot_req, const int64_t *atom_offset,
                         const int64_t *bond_offset, float *xyz, uint8_t *type, int *bonds,
                         uint8_t *rotatable, int *r_real) {
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16)
  for (int i = 0; i < n; ++i) {
    uint64_t s = sm64_stream(seed, TAG_LIGAND, (uint64_t)(first_index + i));
    int64_t a0 = atom_offset[i], b0 = bond_offset[i];
    int r = gen_one_ligand(s, n_atoms[i], n_rot_req[i], n_types, xyz + 3 * a0, type + a0,
                           bonds + 2 * b0, rotatable + b0);
    r_real[i] = r;
    if (r < 0) {
#pragma omp critical
      bad = -(i + 1);
    }
  }
  return bad;
}

/* Per-type radius r_t in [1.5, 2.1] A and well depth eps_t in [0.1, 0.3]. */
LW_EXPORT void lw_type_params(uint64_t seed, int n_types, double *radius, double *eps) {
  uint64_t s = sm64_stream(seed, TAG_TYPES, 0);
  for (int t = 0; t < n_types; ++t) {
    radius[t] = 1.5 + 0.6 * u01(&s);
    eps[t] = 0.1 + 0.2 * u01(&s);
  }
}

/* Receptor atoms uniform in the shell r_in <= |x - c| <= r_out, random types. */
LW_EXPORT void lw_receptor(uint64_t seed, int n, int n_types, const double center[3],
                           double r_in, double r_out, double *xyz, int *type) {
  uint64_t s = sm64_stream(seed, TAG_RECEPTOR, 0);
  for (int i = 0; i < n; ++i) {
    for (;;) {
      double v[3];
      unit_ball(&s, v);
      double r2 = (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * r_out * r_out;
      if (r2 < r_in * r_in) continue;
      xyz[3 * i] = center[0] + r_out * v[0];
      xyz[3 * i + 1] = center[1] + r_out * v[1];
      xyz[3 * i + 2] = center[2] + r_out * v[2];
      break;
    }
    type[i] = uint_below(&s, n_types);
  }
}

/* Anchor points uniform in the ball of the given radius about center (FP32). */
LW_EXPORT void lw_anchors(uint64_t seed, int n, const double center[3], double radius,
                          float *out) {
  uint64_t s = sm64_stream(seed, TAG_ANCHORS, 0);
  for (int i = 0; i < n; ++i) {
    double v[3];
    unit_ball(&s, v);
    out[3 * i] = (float)(center[0] + radius * v[0]);
    out[3 * i + 1] = (float)(center[1] + radius * v[1]);
    out[3 * i + 2] = (float)(center[2] + radius * v[2]);
  }
}

/* Uniform random unit quaternions (w, x, y, z) by Marsaglia's method
 * (Ann. Math. Stat. 43, 1972): two points in the unit disk. */
LW_EXPORT void lw_orientations(uint64_t seed, int n, double *quat) {
  uint64_t s = sm64_stream(seed, TAG_ORIENT, 0);
  for (int i = 0; i < n; ++i) {
    double x1, y1, s1, x2, y2, s2;
    do { x1 = 2.0 * u01(&s) - 1.0; y1 = 2.0 * u01(&s) - 1.0; s1 = x1 * x1 + y1 * y1; } while (s1 >= 1.0);
    do { x2 = 2.0 * u01(&s) - 1.0; y2 = 2.0 * u01(&s) - 1.0; s2 = x2 * x2 + y2 * y2; } while (s2 >= 1.0 || s2 == 0.0);
    double f = sqrt((1.0 - s1) / s2);
    quat[4 * i] = x1; quat[4 * i + 1] = y1; quat[4 * i + 2] = x2 * f; quat[4 * i + 3] = y2 * f;
  }
}

/* Standard normal draws (Box-Muller); used only for network initial weights,
 * which are always passed to both sides explicitly. */
LW_EXPORT void lw_normal(uint64_t seed, uint64_t tag, int64_t n, double *out) {
  uint64_t s = sm64_stream(seed, TAG_NORMAL, tag);
  for (int64_t i = 0; i < n; i += 2) {
    double u1 = u01(&s), u2 = u01(&s);
    if (u1 < 1e-300) u1 = 1e-300;
    double r = sqrt(-2.0 * log(u1));
    out[i] = r * cos(6.283185307179586 * u2);
    if (i + 1 < n) out[i + 1] = r * sin(6.283185307179586 * u2);
  }
}

/* Uniform doubles in [0,1) from stream (seed, tag). */
LW_EXPORT void lw_uniform(uint64_t seed, uint64_t tag, int64_t n, double *out) {
  uint64_t s = sm64_stream(seed, TAG_NORMAL + 1, tag);
  for (int64_t i = 0; i < n; ++i) out[i] = u01(&s);
}

/* ---- grid maps -----------------------------------------------------------
 * V_t(g) = min(cap, sum_j eps_tj [ (r0/r)^12 - 2 (r0/r)^6 ]) over receptor
 * atoms j within `cutoff` of node g, r clamped below at rmin, with
 * r0 = r_t + r_tau(j) and eps_tj = sqrt(eps_t * eps_tau(j)).  Node (ix,iy,iz)
 * sits at origin + h*(ix,iy,iz); maps[t][iz][iy][ix] (FP32, rounded from
 * FP64).  Each node sums its atoms in index order, so the result does not
 * depend on threading. */
LW_EXPORT int lw_grid_maps(int n_types, const double *radius, const double *eps, int n_rec,
                           const double *rec_xyz, const int *rec_type, const double origin[3],
                           double h, int nx, int ny, int nz, double cutoff, double cap,
                           double rmin, float *maps) {
  double *r0 = (double *)malloc(sizeof(double) * (size_t)n_types * n_types);
  double *et = (double *)malloc(sizeof(double) * (size_t)n_types * n_types);
  if (!r0 || !et) { free(r0); free(et); return -2; }
  for (int t = 0; t < n_types; ++t)
    for (int u = 0; u < n_types; ++u) {
      r0[t * n_types + u] = radius[t] + radius[u];
      et[t * n_types + u] = sqrt(eps[t] * eps[u]);
    }
  const double c2 = cutoff * cutoff;
  const size_t plane = (size_t)nx * ny * nz;
  int err = 0;
#pragma omp parallel
  {
    int *row = (int *)malloc(sizeof(int) * (size_t)(n_rec > 0 ? n_rec : 1));
    double *acc = (double *)malloc(sizeof(double) * (size_t)n_types);
    if (!row || !acc) {
#pragma omp critical
      err = -2;
    } else {
#pragma omp for schedule(dynamic, 1) collapse(2)
      for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy) {
          double gy = origin[1] + h * iy, gz = origin[2] + h * iz;
          int nr = 0; /* atoms within the cutoff of this row's line */
          for (int j = 0; j < n_rec; ++j) {
            double dy = rec_xyz[3 * j + 1] - gy, dz = rec_xyz[3 * j + 2] - gz;
            if (dy * dy + dz * dz <= c2) row[nr++] = j;
          }
          for (int ix = 0; ix < nx; ++ix) {
            double gx = origin[0] + h * ix;
            for (int t = 0; t < n_types; ++t) acc[t] = 0.0;
            for (int q = 0; q < nr; ++q) {
              int j = row[q];
              double dx = rec_xyz[3 * j] - gx, dy = rec_xyz[3 * j + 1] - gy,
                     dz = rec_xyz[3 * j + 2] - gz;
              double d2 = dx * dx + dy * dy + dz * dz;
              if (d2 > c2) continue;
              double r = sqrt(d2);
              if (r < rmin) r = rmin;
              int tau = rec_type[j];
              for (int t = 0; t < n_types; ++t) {
                double q1 = r0[t * n_types + tau] / r;
                double q2 = q1 * q1;
                double q6 = q2 * q2 * q2;
                acc[t] += et[t * n_types + tau] * (q6 * q6 - 2.0 * q6);
              }
            }
            size_t g = ((size_t)iz * ny + iy) * nx + ix;
            for (int t = 0; t < n_types; ++t) {
              double v = acc[t] < cap ? acc[t] : cap;
              maps[(size_t)t * plane + g] = (float)v;
            }
          }
        }
    }
    free(row); free(acc);
  }
  free(r0); free(et);
  return err;
}
