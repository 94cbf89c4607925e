/*
 * FP64 CPU oracle for the ligand dock+score hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed
 * CPU baseline of the benchmark may load this file's library.  It shares no
 * code, header, table or constant generator with the CUDA path, and it never
 * touches a GPU.
 *
 * What it computes (paper Sec. 2: each ligand is docked in the binding site
 * by a search with multiple restarts, scored with a geometry-only function,
 * and the ligand's score is the score of its best pose; Sec. 3.3 batches
 * many ligand-pocket pairs).  The paper names the method but gives no
 * formula; the concrete readings taken here are:
 *
 *   pose(s, tors) : start s = o*A + a (orientation o, anchor a).  From the
 *       input (reference) coordinates, each rotatable bond b, in ascending
 *       DFS pre-order of its child atom v (root = atom 0, children visited
 *       in ascending atom index), rotates the subtree of v (the side not
 *       holding the root) about the axis u->v through the CURRENT positions
 *       of u and v by theta = 2*pi*tors[b]/S (right-hand rule, Rodrigues).
 *       Then x' = R_o (x - c) + anchor_a with c the centroid of the input
 *       conformation and R_o the rotation of unit quaternion q_o.
 *   score(x')    : E = sum_i G_{type(i)}(x'_i)
 *                      + w * sum_{(i,j) in P} max(0, 1 - d_ij^2/d_c^2)^2
 *       with P the atom pairs at least 4 bonds apart in the tree.
 *   G_t(x)       : trilinear interpolation of map t at u = (x - origin)/h.
 *       If any component of u lies outside [0, n-1] the atom scores the
 *       out-of-grid penalty instead.  Cell index min(floor(u), n-2), so
 *       every node, the upper faces included, returns its node value.
 *       Written as successive linear interpolations along x, then y, then z.
 *   greedy(s)    : tors = 0; for each bond b in order, try k = 0..S-1
 *       (other torsions fixed), score each pose in full from the reference
 *       coordinates, keep the smallest score (ties -> smaller k).
 *   top-K        : the K starts with the smallest (E, s) pairs; the ligand
 *       score is the first entry's E.
 *   descriptor   : per ligand, counts of each atom type, 8-bin histograms
 *       (edges 1.5, 3, ..., 10.5 A, last bin open) of intramolecular
 *       distances for each unordered pair of DISTINCT types, and the
 *       rotatable-bond count; every count goes through log1p; 233 used
 *       entries zero-padded to 256.  The bin decision is taken in FP32
 *       (d^2 = (dx*dx + dy*dy) + dz*dz with FP32 rounding at each step,
 *       compared with the exactly representable squared edges), the
 *       precision of the GPU kernel, so both sides pick the same bin.
 *
 * Parity pins for every function live in tests/test_oracle_*.py.
 * Compile with -ffp-contract=off.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_EXPORT __attribute__((visibility("default")))
#define OR_MAXA 256

/* ------------------------------------------------------------------------ */
/* Ligand topology, computed from the plain tree definition.                 */
typedef struct {
  int n;                  /* atoms */
  double ref[OR_MAXA][3]; /* input coordinates */
  int type[OR_MAXA];
  int nadj[OR_MAXA];
  int adj[OR_MAXA][8];
  int parent[OR_MAXA];    /* rooted at atom 0 */
  int preorder[OR_MAXA];  /* DFS pre-order position of each atom */
  int nrot;
  int rot_u[64], rot_v[64]; /* rotatable bonds, sorted by preorder[v] */
  unsigned char *moved;     /* nrot x n flags: atom in subtree(v) */
  int *topo;                /* n x n bond distances */
  double centroid[3];
} or_lig;

static void dfs(or_lig *L, int a, int *counter) {
  L->preorder[a] = (*counter)++;
  /* children in ascending atom index */
  int kids[8], nk = 0;
  for (int q = 0; q < L->nadj[a]; ++q) {
    int b = L->adj[a][q];
    if (b != L->parent[a]) kids[nk++] = b;
  }
  for (int i = 1; i < nk; ++i)
    for (int j = i; j > 0 && kids[j - 1] > kids[j]; --j) {
      int t = kids[j]; kids[j] = kids[j - 1]; kids[j - 1] = t;
    }
  for (int i = 0; i < nk; ++i) {
    L->parent[kids[i]] = a;
    dfs(L, kids[i], counter);
  }
}

static int in_subtree(const or_lig *L, int root, int a) {
  while (a >= 0) {
    if (a == root) return 1;
    a = L->parent[a];
  }
  return 0;
}

/* Build the topology; returns 0 or -1 if the bonds do not form a tree. */
static int lig_init(or_lig *L, int n, const float *xyz, const uint8_t *type, int nb,
                    const int *bonds, const uint8_t *rot) {
  L->moved = NULL;
  L->topo = NULL;
  if (n < 1 || n > OR_MAXA || nb != n - 1) return -1;
  memset(L->nadj, 0, sizeof(L->nadj));
  L->n = n;
  for (int i = 0; i < n; ++i) {
    for (int d = 0; d < 3; ++d) L->ref[i][d] = (double)xyz[3 * i + d];
    L->type[i] = type[i];
    L->parent[i] = -2;
  }
  for (int b = 0; b < nb; ++b) {
    int x = bonds[2 * b], y = bonds[2 * b + 1];
    if (x < 0 || y < 0 || x >= n || y >= n || x == y) return -1;
    if (L->nadj[x] >= 8 || L->nadj[y] >= 8) return -1;
    L->adj[x][L->nadj[x]++] = y;
    L->adj[y][L->nadj[y]++] = x;
  }
  L->parent[0] = -1;
  int visited = 0;
  dfs(L, 0, &visited);
  if (visited != n) return -1;
  /* rotatable bonds: child = endpoint whose parent is the other */
  L->nrot = 0;
  for (int b = 0; b < nb; ++b) {
    if (!rot[b]) continue;
    int x = bonds[2 * b], y = bonds[2 * b + 1];
    int u = (L->parent[y] == x) ? x : y;
    int v = (u == x) ? y : x;
    if (L->nrot >= 64) return -1;
    L->rot_u[L->nrot] = u; L->rot_v[L->nrot] = v; L->nrot++;
  }
  for (int i = 1; i < L->nrot; ++i) /* sort by preorder of child */
    for (int j = i; j > 0 && L->preorder[L->rot_v[j - 1]] > L->preorder[L->rot_v[j]]; --j) {
      int t = L->rot_u[j]; L->rot_u[j] = L->rot_u[j - 1]; L->rot_u[j - 1] = t;
      t = L->rot_v[j]; L->rot_v[j] = L->rot_v[j - 1]; L->rot_v[j - 1] = t;
    }
  L->moved = (unsigned char *)malloc((size_t)(L->nrot > 0 ? L->nrot : 1) * n);
  L->topo = (int *)malloc(sizeof(int) * (size_t)n * n);
  if (!L->moved || !L->topo) return -1;
  for (int b = 0; b < L->nrot; ++b)
    for (int a = 0; a < n; ++a) L->moved[b * n + a] = (unsigned char)in_subtree(L, L->rot_v[b], a);
  /* all-pairs bond distance by BFS from each atom */
  int *queue = (int *)malloc(sizeof(int) * (size_t)n);
  for (int s = 0; s < n; ++s) {
    int *d = L->topo + (size_t)s * n;
    for (int a = 0; a < n; ++a) d[a] = -1;
    int h = 0, t = 0;
    queue[t++] = s; d[s] = 0;
    while (h < t) {
      int a = queue[h++];
      for (int q = 0; q < L->nadj[a]; ++q) {
        int b = L->adj[a][q];
        if (d[b] < 0) { d[b] = d[a] + 1; queue[t++] = b; }
      }
    }
  }
  free(queue);
  for (int d = 0; d < 3; ++d) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += L->ref[i][d];
    L->centroid[d] = s / n;
  }
  return 0;
}
static void lig_free(or_lig *L) { free(L->moved); free(L->topo); L->moved = NULL; L->topo = NULL; }

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */

/* Rotation matrix of the unit quaternion q = (w, x, y, z) (normalised here):
 * R v equals the vector part of q v q*. */
OR_EXPORT void or_quat_to_matrix(const double q_in[4], double R[9]) {
  double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
  double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Rodrigues rotation of point p about the axis through a with unit
 * direction n, by angle theta (right-hand rule). */
static void rodrigues(const double a[3], const double n[3], double c, double s, double p[3]) {
  double v[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
  double kv[3] = {n[1] * v[2] - n[2] * v[1], n[2] * v[0] - n[0] * v[2], n[0] * v[1] - n[1] * v[0]};
  double kd = n[0] * v[0] + n[1] * v[1] + n[2] * v[2];
  for (int d = 0; d < 3; ++d) p[d] = a[d] + v[d] * c + kv[d] * s + n[d] * kd * (1.0 - c);
}

/* Rotate the subtree of bond b of L in coords x by angle theta about the
 * current axis u->v. */
static void apply_torsion(const or_lig *L, int b, double theta, double (*x)[3]) {
  int u = L->rot_u[b], v = L->rot_v[b];
  double n[3] = {x[v][0] - x[u][0], x[v][1] - x[u][1], x[v][2] - x[u][2]};
  double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  for (int d = 0; d < 3; ++d) n[d] /= len;
  double c = cos(theta), s = sin(theta);
  double axis_pt[3] = {x[v][0], x[v][1], x[v][2]};
  for (int a = 0; a < L->n; ++a)
    if (L->moved[b * L->n + a]) rodrigues(axis_pt, n, c, s, x[a]);
}

static const double OR_TWO_PI = 6.283185307179586476925286766559;

/* Pose coordinates for rigid part (R, anchor) and torsion indices tors[nrot]
 * with S steps per turn. */
static void build_pose(const or_lig *L, const double R[9], const double anchor[3],
                       const int *tors, int S, double (*out)[3]) {
  for (int a = 0; a < L->n; ++a)
    for (int d = 0; d < 3; ++d) out[a][d] = L->ref[a][d];
  for (int b = 0; b < L->nrot; ++b)
    if (tors[b] % S != 0) apply_torsion(L, b, OR_TWO_PI * (double)tors[b] / (double)S, out);
  for (int a = 0; a < L->n; ++a) {
    double v[3] = {out[a][0] - L->centroid[0], out[a][1] - L->centroid[1], out[a][2] - L->centroid[2]};
    for (int d = 0; d < 3; ++d)
      out[a][d] = R[3 * d] * v[0] + R[3 * d + 1] * v[1] + R[3 * d + 2] * v[2] + anchor[d];
  }
}

/* ------------------------------------------------------------------------ */
/* Pocket and score                                                          */
typedef struct {
  const float *maps; /* [T][nz][ny][nx] */
  int n_types, nx, ny, nz;
  double origin[3], h;
  double penalty;   /* out-of-grid per-atom score */
} or_pocket;

static double lerp(double a, double b, double f) { return a + f * (b - a); }

static double trilinear(const or_pocket *P, int t, const double x[3]) {
  int dims[3] = {P->nx, P->ny, P->nz};
  double u[3];
  int c[3];
  for (int d = 0; d < 3; ++d) {
    u[d] = (x[d] - P->origin[d]) / P->h;
    if (!(u[d] >= 0.0 && u[d] <= (double)(dims[d] - 1))) return P->penalty;
    int f = (int)floor(u[d]);
    c[d] = f < dims[d] - 2 ? f : dims[d] - 2;
  }
  double fx = u[0] - c[0], fy = u[1] - c[1], fz = u[2] - c[2];
  const float *m = P->maps + (size_t)t * P->nx * P->ny * P->nz;
#define V(i, j, k) ((double)m[((size_t)(c[2] + (k)) * P->ny + (c[1] + (j))) * P->nx + (c[0] + (i))])
  double y0z0 = lerp(V(0, 0, 0), V(1, 0, 0), fx);
  double y1z0 = lerp(V(0, 1, 0), V(1, 1, 0), fx);
  double y0z1 = lerp(V(0, 0, 1), V(1, 0, 1), fx);
  double y1z1 = lerp(V(0, 1, 1), V(1, 1, 1), fx);
#undef V
  double z0 = lerp(y0z0, y1z0, fy);
  double z1 = lerp(y0z1, y1z1, fy);
  return lerp(z0, z1, fz);
}

typedef struct {
  double w;      /* clash weight */
  double dc;     /* clash distance (A) */
  int min_sep;   /* pairs at least this many bonds apart */
} or_clash;

/* Score of coordinates x; *mag (optional) receives the sum of the absolute
 * values of its terms, the scale against which rounding error of the sum is
 * measured. */
static double score_coords_mag(const or_lig *L, const or_pocket *P, const or_clash *C,
                               double (*x)[3], double *mag) {
  double e = 0.0, m = 0.0;
  for (int a = 0; a < L->n; ++a) {
    double g = trilinear(P, L->type[a], x[a]);
    e += g;
    m += fabs(g);
  }
  double cl = 0.0, inv = 1.0 / (C->dc * C->dc);
  for (int i = 0; i < L->n; ++i)
    for (int j = i + 1; j < L->n; ++j) {
      if (L->topo[(size_t)i * L->n + j] < C->min_sep) continue;
      double dx = x[i][0] - x[j][0], dy = x[i][1] - x[j][1], dz = x[i][2] - x[j][2];
      double t = 1.0 - (dx * dx + dy * dy + dz * dz) * inv;
      if (t > 0.0) cl += t * t;
    }
  if (mag) *mag = m + fabs(C->w) * cl;
  return e + C->w * cl;
}

static double score_coords(const or_lig *L, const or_pocket *P, const or_clash *C,
                           double (*x)[3]) {
  return score_coords_mag(L, P, C, x, NULL);
}

/* ------------------------------------------------------------------------ */
/* Exported API                                                              */

/* Ligand input (one ligand). */
typedef struct {
  int n_atoms;
  const float *xyz;      /* [n][3] */
  const uint8_t *type;   /* [n] */
  int n_bonds;           /* n-1 */
  const int *bonds;      /* [n-1][2] */
  const uint8_t *rot;    /* [n-1] */
} or_ligand_in;

typedef struct {
  int n_orient, n_anchor, S;
  const double *quat;     /* [n_orient][4] */
  const float *anchors;   /* [n_anchor][3] */
  double clash_w, clash_dc;
  int clash_min_sep;
  double penalty;
} or_sampling;

typedef struct {
  const float *maps;
  int n_types, nx, ny, nz;
  double origin[3];
  double h;
} or_pocket_in;

static void make_pocket(const or_pocket_in *pi, double penalty, or_pocket *P) {
  P->maps = pi->maps; P->n_types = pi->n_types;
  P->nx = pi->nx; P->ny = pi->ny; P->nz = pi->nz;
  for (int d = 0; d < 3; ++d) P->origin[d] = pi->origin[d];
  P->h = pi->h; P->penalty = penalty;
}

static void start_frame(const or_sampling *sp, int s, double R[9], double anc[3]) {
  int o = s / sp->n_anchor, a = s % sp->n_anchor;
  or_quat_to_matrix(sp->quat + 4 * o, R);
  for (int d = 0; d < 3; ++d) anc[d] = (double)sp->anchors[3 * a + d];
}

/* Realised rotatable-bond count of a ligand in the oracle's order, with the
 * (u, v) atoms of each bond; returns nrot or -1. */
OR_EXPORT int or_ligand_bonds(const or_ligand_in *li, int *u_out, int *v_out) {
  or_lig L;
  if (lig_init(&L, li->n_atoms, li->xyz, li->type, li->n_bonds, li->bonds, li->rot)) { lig_free(&L); return -1; }
  for (int b = 0; b < L.nrot; ++b) { if (u_out) u_out[b] = L.rot_u[b]; if (v_out) v_out[b] = L.rot_v[b]; }
  int r = L.nrot;
  lig_free(&L);
  return r;
}

/* Topological (bond-count) distance matrix n x n. */
OR_EXPORT int or_topo_distance(const or_ligand_in *li, int *out) {
  or_lig L;
  if (lig_init(&L, li->n_atoms, li->xyz, li->type, li->n_bonds, li->bonds, li->rot)) { lig_free(&L); return -1; }
  memcpy(out, L.topo, sizeof(int) * (size_t)L.n * L.n);
  lig_free(&L);
  return 0;
}

/* Coordinates of n_poses poses: start ids s[i], torsions tors[i][nrot]
 * (stride tors_stride); out [n_poses][n][3]. */
OR_EXPORT int or_pose_coords(const or_ligand_in *li, const or_sampling *sp, int n_poses,
                             const int *starts, const int *tors, int tors_stride, double *out) {
  or_lig L;
  if (lig_init(&L, li->n_atoms, li->xyz, li->type, li->n_bonds, li->bonds, li->rot)) { lig_free(&L); return -1; }
  for (int p = 0; p < n_poses; ++p) {
    double R[9], anc[3];
    start_frame(sp, starts[p], R, anc);
    build_pose(&L, R, anc, tors + (size_t)p * tors_stride, sp->S, (double(*)[3])(out + (size_t)p * L.n * 3));
  }
  lig_free(&L);
  return 0;
}

/* Apply torsions to the input coordinates in a caller-given bond order,
 * each about the current axis, without the rigid part (pins torsion-order
 * independence). angles[nrot] in radians; order[nrot] permutes bonds. */
OR_EXPORT int or_torsions_in_order(const or_ligand_in *li, const double *angles, const int *order,
                                   double *out) {
  or_lig L;
  if (lig_init(&L, li->n_atoms, li->xyz, li->type, li->n_bonds, li->bonds, li->rot)) { lig_free(&L); return -1; }
  double (*x)[3] = (double(*)[3])out;
  for (int a = 0; a < L.n; ++a)
    for (int d = 0; d < 3; ++d) x[a][d] = L.ref[a][d];
  for (int q = 0; q < L.nrot; ++q) apply_torsion(&L, order[q], angles[order[q]], x);
  lig_free(&L);
  return 0;
}

/* Trilinear value of map t at n points (pins interpolation). */
OR_EXPORT void or_trilinear(const or_pocket_in *pi, double penalty, int t, int n,
                            const double *pts, double *out) {
  or_pocket P;
  make_pocket(pi, penalty, &P);
  for (int i = 0; i < n; ++i) out[i] = trilinear(&P, t, pts + 3 * i);
}

/* Score of arbitrary coordinates [n][3] for the ligand's types/topology. */
OR_EXPORT int or_score_coords(const or_ligand_in *li, const or_pocket_in *pi, const or_sampling *sp,
                              const double *coords, double *out) {
  or_lig L;
  if (lig_init(&L, li->n_atoms, li->xyz, li->type, li->n_bonds, li->bonds, li->rot)) { lig_free(&L); return -1; }
  or_pocket P;
  make_pocket(pi, sp->penalty, &P);
  or_clash C = {sp->clash_w, sp->clash_dc, sp->clash_min_sep};
  double (*x)[3] = (double(*)[3])malloc(sizeof(double) * 3 * (size_t)L.n);
  memcpy(x, coords, sizeof(double) * 3 * (size_t)L.n);
  *out = score_coords(&L, &P, &C, x);
  free(x);
  lig_free(&L);
  return 0;
}

/* Scores of n_poses (start, tors) poses, parallel over poses; mag_out
 * (optional) receives each score's sum of absolute term values. */
OR_EXPORT int or_score_poses(const or_ligand_in *li, const or_pocket_in *pi, const or_sampling *sp,
                             int n_poses, const int *starts, const int *tors, int tors_stride,
                             double *out, double *mag_out) {
  or_lig L;
  if (lig_init(&L, li->n_atoms, li->xyz, li->type, li->n_bonds, li->bonds, li->rot)) { lig_free(&L); return -1; }
  or_pocket P;
  make_pocket(pi, sp->penalty, &P);
  or_clash C = {sp->clash_w, sp->clash_dc, sp->clash_min_sep};
#pragma omp parallel
  {
    double (*x)[3] = (double(*)[3])malloc(sizeof(double) * 3 * (size_t)L.n);
#pragma omp for schedule(dynamic, 8)
    for (int p = 0; p < n_poses; ++p) {
      double R[9], anc[3];
      start_frame(sp, starts[p], R, anc);
      build_pose(&L, R, anc, tors + (size_t)p * tors_stride, sp->S, x);
      out[p] = score_coords_mag(&L, &P, &C, x, mag_out ? mag_out + p : NULL);
    }
    free(x);
  }
  lig_free(&L);
  return 0;
}

/* Greedy torsion sweep for the listed starts (parallel over starts).
 * e_out[i] = final score, tors_out[i][nrot] (stride tors_stride) = chosen
 * step per bond in bond order; trial_out (optional, [i][nrot][S]) = every
 * trial score. */
OR_EXPORT int or_greedy(const or_ligand_in *li, const or_pocket_in *pi, const or_sampling *sp,
                        int n_starts, const int *starts, double *e_out, int *tors_out,
                        int tors_stride, double *trial_out) {
  or_lig L;
  if (lig_init(&L, li->n_atoms, li->xyz, li->type, li->n_bonds, li->bonds, li->rot)) { lig_free(&L); return -1; }
  or_pocket P;
  make_pocket(pi, sp->penalty, &P);
  or_clash C = {sp->clash_w, sp->clash_dc, sp->clash_min_sep};
  const int S = sp->S;
#pragma omp parallel
  {
    double (*x)[3] = (double(*)[3])malloc(sizeof(double) * 3 * (size_t)L.n);
    int tors[64];
#pragma omp for schedule(dynamic, 4)
    for (int i = 0; i < n_starts; ++i) {
      double R[9], anc[3];
      start_frame(sp, starts[i], R, anc);
      for (int b = 0; b < L.nrot; ++b) tors[b] = 0;
      double best = 0.0;
      if (L.nrot == 0) {
        build_pose(&L, R, anc, tors, S, x);
        best = score_coords(&L, &P, &C, x);
      }
      for (int b = 0; b < L.nrot; ++b) {
        int bk = 0;
        for (int k = 0; k < S; ++k) {
          tors[b] = k;
          build_pose(&L, R, anc, tors, S, x);
          double e = score_coords(&L, &P, &C, x);
          if (trial_out) trial_out[((size_t)i * L.nrot + b) * S + k] = e;
          if (k == 0 || e < best) { best = e; bk = k; }
        }
        tors[b] = bk;
      }
      e_out[i] = best;
      for (int b = 0; b < L.nrot; ++b) tors_out[(size_t)i * tors_stride + b] = tors[b];
    }
    free(x);
  }
  lig_free(&L);
  return 0;
}

/* Exhaustive enumeration of all S^nrot torsion combinations for each listed
 * start; e_out[i][c] with c the odometer index (bond 0 fastest). */
OR_EXPORT int or_exhaustive(const or_ligand_in *li, const or_pocket_in *pi, const or_sampling *sp,
                            int n_starts, const int *starts, double *e_out) {
  or_lig L;
  if (lig_init(&L, li->n_atoms, li->xyz, li->type, li->n_bonds, li->bonds, li->rot)) { lig_free(&L); return -1; }
  or_pocket P;
  make_pocket(pi, sp->penalty, &P);
  or_clash C = {sp->clash_w, sp->clash_dc, sp->clash_min_sep};
  const int S = sp->S;
  long long combos = 1;
  for (int b = 0; b < L.nrot; ++b) combos *= S;
#pragma omp parallel
  {
    double (*x)[3] = (double(*)[3])malloc(sizeof(double) * 3 * (size_t)L.n);
    int tors[64];
#pragma omp for schedule(dynamic, 1) collapse(2)
    for (int i = 0; i < n_starts; ++i)
      for (long long c = 0; c < combos; ++c) {
        double R[9], anc[3];
        start_frame(sp, starts[i], R, anc);
        long long r = c;
        for (int b = 0; b < L.nrot; ++b) { tors[b] = (int)(r % S); r /= S; }
        build_pose(&L, R, anc, tors, S, x);
        e_out[(size_t)i * combos + c] = score_coords(&L, &P, &C, x);
      }
    free(x);
  }
  lig_free(&L);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Pose refinement by gradient descent (paper Sec. 2: the docking search is  */
/* a gradient descent from multiple restarts; here the greedy sweep supplies */
/* the restarts and a local descent refines the best poses).  Readings:      */
/*                                                                           */
/*   state q = (R, t, phi): x_i = R (y_i - c) + t, with y the input          */
/*       conformation after torsion angle phi_b (radians) is applied to each */
/*       rotatable bond b in sweep order about its current axis u->v (as in  */
/*       pose(s, tors), with continuous angles; phi_b = 0 leaves the bond),  */
/*       c the input centroid, R a rotation matrix, t in Angstrom.           */
/*   E(q)    : the docking score of x (grid terms, penalty, clash term).     */
/*   g_i     : dE/dx_i.  Grid: derivative of the trilinear interpolant in    */
/*       the atom's cell (the cell the value uses), divided by h; zero for   */
/*       an atom scoring the penalty.  Clash: -4 w t (x_i - x_j) / d_c^2     */
/*       for every pair with t = 1 - d_ij^2/d_c^2 > 0.                       */
/*   generalised gradient: the derivatives of E along a translation, a       */
/*       rotation exp([w]x) R about t, and a turn of bond b:                 */
/*         F = sum_i g_i,   tau = sum_i (x_i - t) x g_i,                     */
/*         psi_b = n_b . sum_{i moved by b} (x_i - x_v) x g_i,               */
/*       n_b the unit axis u->v of bond b at the pose.                       */
/*   descent : scaled steepest descent with step control.  The trial from q  */
/*       is t' = t - eta F / N, R' = GS(Rot(-eta tau / I_R) R) and           */
/*       phi'_b = phi_b - eta psi_b / I_b, with I_R = 1 + sum_i |x_i - t|^2  */
/*       and I_b = 1 + sum_{i moved by b} |(x_i - x_v) minus its component   */
/*       along n_b|^2 (A^2, the moments that turn a unit angle into atom     */
/*       displacement); GS re-orthonormalises the rows (r0 normalised, r1    */
/*       made orthogonal to r0 and normalised, r2 = r0 x r1).  The trial is  */
/*       accepted if E(trial) < E(q), and eta grows by 1.25; otherwise it is */
/*       rejected and eta halves.  A fixed number of iterations.             */

typedef struct {
  double R[9], t[3], phi[64];
} or_state;

static void state_coords(const or_lig *L, const or_state *q, double (*x)[3]) {
  for (int a = 0; a < L->n; ++a)
    for (int d = 0; d < 3; ++d) x[a][d] = L->ref[a][d];
  for (int b = 0; b < L->nrot; ++b)
    if (q->phi[b] != 0.0) apply_torsion(L, b, q->phi[b], x);
  for (int a = 0; a < L->n; ++a) {
    double v[3] = {x[a][0] - L->centroid[0], x[a][1] - L->centroid[1], x[a][2] - L->centroid[2]};
    for (int d = 0; d < 3; ++d)
      x[a][d] = q->R[3 * d] * v[0] + q->R[3 * d + 1] * v[1] + q->R[3 * d + 2] * v[2] + q->t[d];
  }
}

/* Trilinear value of map t at x (same arithmetic as trilinear()) and its
 * gradient with respect to x; *face = distance (grid units) of u to the
 * nearest face of its cell, or a large value for a penalty atom. */
static double trilinear_grad(const or_pocket *P, int t, const double x[3], double g[3],
                             double *face) {
  int dims[3] = {P->nx, P->ny, P->nz};
  double u[3];
  int c[3];
  g[0] = g[1] = g[2] = 0.0;
  *face = 1e30;
  for (int d = 0; d < 3; ++d) {
    u[d] = (x[d] - P->origin[d]) / P->h;
    if (!(u[d] >= 0.0 && u[d] <= (double)(dims[d] - 1))) return P->penalty;
    int f = (int)floor(u[d]);
    c[d] = f < dims[d] - 2 ? f : dims[d] - 2;
  }
  double fx = u[0] - c[0], fy = u[1] - c[1], fz = u[2] - c[2];
  for (int d = 0; d < 3; ++d) {
    double fr = u[d] - floor(u[d]);
    double dd = fr < 1.0 - fr ? fr : 1.0 - fr;
    if (dd < *face) *face = dd;
  }
  const float *m = P->maps + (size_t)t * P->nx * P->ny * P->nz;
#define V(i, j, k) ((double)m[((size_t)(c[2] + (k)) * P->ny + (c[1] + (j))) * P->nx + (c[0] + (i))])
  double v000 = V(0, 0, 0), v100 = V(1, 0, 0), v010 = V(0, 1, 0), v110 = V(1, 1, 0);
  double v001 = V(0, 0, 1), v101 = V(1, 0, 1), v011 = V(0, 1, 1), v111 = V(1, 1, 1);
#undef V
  double y0z0 = lerp(v000, v100, fx), y1z0 = lerp(v010, v110, fx);
  double y0z1 = lerp(v001, v101, fx), y1z1 = lerp(v011, v111, fx);
  double z0 = lerp(y0z0, y1z0, fy), z1 = lerp(y0z1, y1z1, fy);
  /* d/dfx, d/dfy, d/dfz of the interpolant */
  double dx = lerp(lerp(v100 - v000, v110 - v010, fy), lerp(v101 - v001, v111 - v011, fy), fz);
  double dy = lerp(y1z0 - y0z0, y1z1 - y0z1, fz);
  double dz = z1 - z0;
  g[0] = dx / P->h; g[1] = dy / P->h; g[2] = dz / P->h;
  return lerp(z0, z1, fz);
}

static void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

/* E and generalised gradient G[6 + nrot] = (F, tau, psi) at state q;
 * scale[1 + 6 + nrot]: sum of absolute term values of E, then for each
 * gradient component the sum of the absolute values of its contributions
 * (the scale of its rounding error); inert[1 + nrot] = (I_R, I_b);
 * *face = smallest cell-face distance of any in-grid atom. */
static double energy_grad(const or_lig *L, const or_pocket *P, const or_clash *C, const or_state *q,
                          double (*x)[3], double (*g)[3], double *a_abs, double *G, double *scale,
                          double *inert, double *face) {
  const int n = L->n, nr = L->nrot;
  state_coords(L, q, x);
  double e = 0.0, mag = 0.0, inv = 1.0 / (C->dc * C->dc);
  *face = 1e30;
  for (int i = 0; i < n; ++i) {
    double fc;
    double v = trilinear_grad(P, L->type[i], x[i], g[i], &fc);
    if (fc < *face) *face = fc;
    e += v;
    mag += fabs(v);
    a_abs[i] = fabs(g[i][0]) + fabs(g[i][1]) + fabs(g[i][2]);
  }
  double cl = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      if (L->topo[(size_t)i * n + j] < C->min_sep) continue;
      double d[3] = {x[i][0] - x[j][0], x[i][1] - x[j][1], x[i][2] - x[j][2]};
      double tt = 1.0 - (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * inv;
      if (!(tt > 0.0)) continue;
      cl += tt * tt;
      double f = -4.0 * C->w * tt * inv;
      for (int k = 0; k < 3; ++k) {
        g[i][k] += f * d[k];
        g[j][k] -= f * d[k];
      }
      double fa = fabs(f) * (fabs(d[0]) + fabs(d[1]) + fabs(d[2]));
      a_abs[i] += fa;
      a_abs[j] += fa;
    }
  e += C->w * cl;
  scale[0] = mag + fabs(C->w) * cl;
  for (int k = 0; k < 6 + nr; ++k) { G[k] = 0.0; scale[1 + k] = 0.0; }
  inert[0] = 1.0;
  for (int i = 0; i < n; ++i) {
    double r[3] = {x[i][0] - q->t[0], x[i][1] - q->t[1], x[i][2] - q->t[2]}, c[3];
    cross3(r, g[i], c);
    double rl = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int k = 0; k < 3; ++k) {
      G[k] += g[i][k];
      G[3 + k] += c[k];
      scale[1 + k] += a_abs[i];
      scale[4 + k] += rl * a_abs[i];
    }
    inert[0] += r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  }
  for (int b = 0; b < nr; ++b) {
    int u = L->rot_u[b], v = L->rot_v[b];
    double nb[3] = {x[v][0] - x[u][0], x[v][1] - x[u][1], x[v][2] - x[u][2]};
    double len = sqrt(nb[0] * nb[0] + nb[1] * nb[1] + nb[2] * nb[2]);
    for (int d = 0; d < 3; ++d) nb[d] /= len;
    double psi = 0.0, sc = 0.0, in = 1.0;
    for (int i = 0; i < n; ++i) {
      if (!L->moved[b * n + i] || i == v) continue;
      double r[3] = {x[i][0] - x[v][0], x[i][1] - x[v][1], x[i][2] - x[v][2]}, c[3];
      cross3(r, g[i], c);
      psi += nb[0] * c[0] + nb[1] * c[1] + nb[2] * c[2];
      double rl = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
      sc += rl * a_abs[i];
      double ra = r[0] * nb[0] + r[1] * nb[1] + r[2] * nb[2];
      in += rl * rl - ra * ra;
    }
    G[6 + b] = psi;
    scale[7 + b] = sc;
    inert[1 + b] = in;
  }
  return e;
}

/* Rotation matrix exp([w]x) (Rodrigues; identity for w = 0). */
static void rot_exp(const double w[3], double M[9]) {
  double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  if (th == 0.0) {
    for (int k = 0; k < 9; ++k) M[k] = (k % 4 == 0) ? 1.0 : 0.0;
    return;
  }
  double n[3] = {w[0] / th, w[1] / th, w[2] / th}, c = cos(th), s = sin(th), o = 1.0 - c;
  M[0] = c + o * n[0] * n[0];        M[1] = o * n[0] * n[1] - s * n[2]; M[2] = o * n[0] * n[2] + s * n[1];
  M[3] = o * n[1] * n[0] + s * n[2]; M[4] = c + o * n[1] * n[1];        M[5] = o * n[1] * n[2] - s * n[0];
  M[6] = o * n[2] * n[0] - s * n[1]; M[7] = o * n[2] * n[1] + s * n[0]; M[8] = c + o * n[2] * n[2];
}

/* Rows re-orthonormalised by Gram-Schmidt, r2 = r0 x r1. */
static void gram_schmidt(double R[9]) {
  double *r0 = R, *r1 = R + 3;
  double l0 = sqrt(r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]);
  for (int k = 0; k < 3; ++k) r0[k] /= l0;
  double dp = r0[0] * r1[0] + r0[1] * r1[1] + r0[2] * r1[2];
  for (int k = 0; k < 3; ++k) r1[k] -= dp * r0[k];
  double l1 = sqrt(r1[0] * r1[0] + r1[1] * r1[1] + r1[2] * r1[2]);
  for (int k = 0; k < 3; ++k) r1[k] /= l1;
  cross3(r0, r1, R + 6);
}

static void trial_state(const or_lig *L, const or_state *q, const double *G, const double *inert,
                        double eta, or_state *out) {
  double w[3], M[9];
  for (int k = 0; k < 3; ++k) {
    out->t[k] = q->t[k] - eta * G[k] / L->n;
    w[k] = -eta * G[3 + k] / inert[0];
  }
  rot_exp(w, M);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      out->R[3 * r + c] = M[3 * r] * q->R[c] + M[3 * r + 1] * q->R[3 + c] + M[3 * r + 2] * q->R[6 + c];
  gram_schmidt(out->R);
  for (int b = 0; b < L->nrot; ++b) out->phi[b] = q->phi[b] - eta * G[6 + b] / inert[1 + b];
}

static void state_in(const or_lig *L, const double *s, or_state *q) {
  memcpy(q->R, s, 9 * sizeof(double));
  memcpy(q->t, s + 9, 3 * sizeof(double));
  for (int b = 0; b < L->nrot; ++b) q->phi[b] = s[12 + b];
}

static void state_out(const or_lig *L, const or_state *q, double *s) {
  memcpy(s, q->R, 9 * sizeof(double));
  memcpy(s + 9, q->t, 3 * sizeof(double));
  for (int b = 0; b < L->nrot; ++b) s[12 + b] = q->phi[b];
}

/* Coordinates [n][n_atoms][3] of n states (rows [12 + nrot]). */
OR_EXPORT int or_state_coords(const or_ligand_in *li, int n_states, const double *states, double *out) {
  or_lig L;
  if (lig_init(&L, li->n_atoms, li->xyz, li->type, li->n_bonds, li->bonds, li->rot)) { lig_free(&L); return -1; }
  for (int p = 0; p < n_states; ++p) {
    or_state q;
    state_in(&L, states + (size_t)p * (12 + L.nrot), &q);
    state_coords(&L, &q, (double(*)[3])(out + (size_t)p * L.n * 3));
  }
  lig_free(&L);
  return 0;
}

/* E, generalised gradient and scales at n states.  states: [n][12 + nrot]
 * (R row-major, t, phi); g_out [n][6 + nrot]; scale_out [n][7 + nrot];
 * inert_out [n][1 + nrot]; face_out [n]. */
OR_EXPORT int or_pose_grad(const or_ligand_in *li, const or_pocket_in *pi, const or_sampling *sp,
                           int n_states, const double *states, double *e_out, double *g_out,
                           double *scale_out, double *inert_out, double *face_out) {
  or_lig L;
  if (lig_init(&L, li->n_atoms, li->xyz, li->type, li->n_bonds, li->bonds, li->rot)) { lig_free(&L); return -1; }
  or_pocket P;
  make_pocket(pi, sp->penalty, &P);
  or_clash C = {sp->clash_w, sp->clash_dc, sp->clash_min_sep};
  const int nr = L.nrot;
#pragma omp parallel
  {
    double (*x)[3] = (double(*)[3])malloc(sizeof(double) * 3 * (size_t)L.n);
    double (*g)[3] = (double(*)[3])malloc(sizeof(double) * 3 * (size_t)L.n);
    double *aa = (double *)malloc(sizeof(double) * (size_t)L.n);
#pragma omp for schedule(dynamic, 4)
    for (int p = 0; p < n_states; ++p) {
      or_state q;
      state_in(&L, states + (size_t)p * (12 + nr), &q);
      e_out[p] = energy_grad(&L, &P, &C, &q, x, g, aa, g_out + (size_t)p * (6 + nr),
                             scale_out + (size_t)p * (7 + nr), inert_out + (size_t)p * (1 + nr),
                             face_out + p);
    }
    free(x); free(g); free(aa);
  }
  lig_free(&L);
  return 0;
}

/* Descent from n states for `iters` iterations (see above).  follow
 * (optional, [n]): bit it = the decision to take at iteration it instead of
 * the oracle's own; a decision that differs from the oracle's own by more
 * than a near-tie (|E(trial) - E| > tie_rel * max(scale, 1)) is counted in
 * n_disagree[p].  Outputs: final states [n][12 + nrot], e_in/e_out [n],
 * own_mask [n] (the oracle's own decisions along the path it took),
 * n_disagree [n] (optional), scale_out [n] (sum of |terms| of the final E). */
OR_EXPORT int or_refine(const or_ligand_in *li, const or_pocket_in *pi, const or_sampling *sp,
                        int n_states, const double *states, int iters, double eta0,
                        const uint32_t *follow, double tie_rel, double *states_out, double *e_in,
                        double *e_out, uint32_t *own_mask, int *n_disagree, double *scale_out) {
  if (iters < 0 || iters > 32) return -2;
  or_lig L;
  if (lig_init(&L, li->n_atoms, li->xyz, li->type, li->n_bonds, li->bonds, li->rot)) { lig_free(&L); return -1; }
  or_pocket P;
  make_pocket(pi, sp->penalty, &P);
  or_clash C = {sp->clash_w, sp->clash_dc, sp->clash_min_sep};
  const int nr = L.nrot;
#pragma omp parallel
  {
    double (*x)[3] = (double(*)[3])malloc(sizeof(double) * 3 * (size_t)L.n);
    double (*g)[3] = (double(*)[3])malloc(sizeof(double) * 3 * (size_t)L.n);
    double *aa = (double *)malloc(sizeof(double) * (size_t)L.n);
    double G[70], G2[70], sc[71], sc2[71], in[65], in2[65], face;
#pragma omp for schedule(dynamic, 2)
    for (int p = 0; p < n_states; ++p) {
      or_state q, tq;
      state_in(&L, states + (size_t)p * (12 + nr), &q);
      double e = energy_grad(&L, &P, &C, &q, x, g, aa, G, sc, in, &face);
      e_in[p] = e;
      double eta = eta0;
      uint32_t mask = 0;
      int dis = 0;
      for (int it = 0; it < iters; ++it) {
        trial_state(&L, &q, G, in, eta, &tq);
        double et = energy_grad(&L, &P, &C, &tq, x, g, aa, G2, sc2, in2, &face);
        int own = et < e;
        int take = follow ? (int)((follow[p] >> it) & 1u) : own;
        if (take != own) {
          double s = sc[0] > sc2[0] ? sc[0] : sc2[0];
          if (fabs(et - e) > tie_rel * (s > 1.0 ? s : 1.0)) ++dis;
        }
        if (own) mask |= 1u << it;
        if (take) {
          q = tq; e = et;
          memcpy(G, G2, sizeof(double) * (6 + nr));
          memcpy(sc, sc2, sizeof(double) * (7 + nr));
          memcpy(in, in2, sizeof(double) * (1 + nr));
          eta *= 1.25;
        } else {
          eta *= 0.5;
        }
      }
      state_out(&L, &q, states_out + (size_t)p * (12 + nr));
      e_out[p] = e;
      own_mask[p] = mask;
      if (n_disagree) n_disagree[p] = dis;
      if (scale_out) scale_out[p] = sc[0];
    }
    free(x); free(g); free(aa);
  }
  lig_free(&L);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Exact rescoring and pose filter (paper Sec. 2: a more accurate scoring of */
/* the generated poses, then a filter).  Readings:                           */
/*   e_inter : sum over ligand atoms i of min(cap, sum_j eps_ij [(r0/r)^12   */
/*       - 2 (r0/r)^6]) over receptor atoms j within `cutoff` of x_i, r      */
/*       clamped below at rmin, r0 = r_t + r_tau, eps_ij = sqrt(eps_t eps_tau)*/
/*       -- the function the grid maps tabulate, evaluated at the atom       */
/*       itself instead of interpolated, everywhere (no box penalty).        */
/*   e_clash : the docking score's intramolecular clash term.                */
/*   filter  : a pose passes when no atom lies outside the map box           */
/*       ([0, n-1] in grid units on every axis) and no atom's receptor sum   */
/*       reaches the cap.                                                    */
typedef struct {
  int n;
  const float *xyz;     /* [n][3] */
  const int *type;      /* [n] */
  int n_types;
  const double *radius; /* [n_types] */
  const double *eps;    /* [n_types] */
  double cutoff, cap, rmin;
} or_receptor_in;

/* Receptor sum at ligand atom x of type t (uncapped, FP64) and the sum of
 * the magnitudes of its pair terms. */
static void receptor_sum(const or_receptor_in *rc, int t, const double x[3], double *acc_out, double *mag_out) {
  const double c2 = rc->cutoff * rc->cutoff;
  double acc = 0.0, am = 0.0;
  for (int j = 0; j < rc->n; ++j) {
    double dx = (double)rc->xyz[3 * j] - x[0], dy = (double)rc->xyz[3 * j + 1] - x[1],
           dz = (double)rc->xyz[3 * j + 2] - x[2];
    double d2 = dx * dx + dy * dy + dz * dz;
    if (d2 > c2) continue;
    double r = sqrt(d2);
    if (r < rc->rmin) r = rc->rmin;
    int tau = rc->type[j];
    double q = (rc->radius[t] + rc->radius[tau]) / r;
    double q2 = q * q, q6 = q2 * q2 * q2;
    double v = sqrt(rc->eps[t] * rc->eps[tau]) * (q6 * q6 - 2.0 * q6);
    acc += v;
    am += fabs(v);
  }
  *acc_out = acc;
  *mag_out = am;
}

/* Signed distance (grid units) of x to the nearest face of the map box
 * [0, n-1]^3: positive inside, negative outside. */
static double face_distance(const or_pocket_in *pi, const double x[3]) {
  const int dims[3] = {pi->nx, pi->ny, pi->nz};
  double in = 1e300, out = 0.0;
  for (int d = 0; d < 3; ++d) {
    double u = (x[d] - pi->origin[d]) / pi->h, hi = (double)(dims[d] - 1);
    double m = u < hi - u ? u : hi - u;
    if (m < in) in = m;
    if (m < 0.0 && -m > out) out = -m;
  }
  return in >= 0.0 ? in : -out;
}

/* Per atom of n_poses coordinate sets: the uncapped receptor sum, the sum
 * of its pair-term magnitudes and the signed distance to the box faces
 * (outputs [n_poses][n]).  The filter's per-atom inputs, for checks of the
 * decisions near their thresholds. */
OR_EXPORT int or_rescore_atoms(const or_ligand_in *li, const or_pocket_in *pi, const or_receptor_in *rc,
                               int n_poses, const double *coords, double *atom_sum, double *atom_mag,
                               double *atom_face) {
  or_lig L;
  if (lig_init(&L, li->n_atoms, li->xyz, li->type, li->n_bonds, li->bonds, li->rot)) { lig_free(&L); return -1; }
  const int n = L.n;
#pragma omp parallel for schedule(dynamic, 4)
  for (int p = 0; p < n_poses; ++p) {
    const double (*x)[3] = (const double(*)[3])(coords + (size_t)p * n * 3);
    for (int i = 0; i < n; ++i) {
      receptor_sum(rc, L.type[i], x[i], atom_sum + (size_t)p * n + i, atom_mag + (size_t)p * n + i);
      atom_face[(size_t)p * n + i] = face_distance(pi, x[i]);
    }
  }
  lig_free(&L);
  return 0;
}

/* For n_poses coordinate sets [n_poses][n][3]: e_inter, e_clash, n_outside,
 * n_capped and scale (sum of absolute values of the per-atom and clash terms,
 * each per-atom term itself counted by the sum of its pair magnitudes when
 * it is not capped). */
OR_EXPORT int or_rescore_coords(const or_ligand_in *li, const or_pocket_in *pi, const or_sampling *sp,
                                const or_receptor_in *rc, int n_poses, const double *coords,
                                double *e_inter, double *e_clash, int *n_out, int *n_capped,
                                double *scale) {
  or_lig L;
  if (lig_init(&L, li->n_atoms, li->xyz, li->type, li->n_bonds, li->bonds, li->rot)) { lig_free(&L); return -1; }
  or_clash C = {sp->clash_w, sp->clash_dc, sp->clash_min_sep};
  const int n = L.n;
  const int dims[3] = {pi->nx, pi->ny, pi->nz};
#pragma omp parallel for schedule(dynamic, 4)
  for (int p = 0; p < n_poses; ++p) {
    const double (*x)[3] = (const double(*)[3])(coords + (size_t)p * n * 3);
    double ei = 0.0, mag = 0.0;
    int nout = 0, ncap = 0;
    for (int i = 0; i < n; ++i) {
      int outside = 0;
      for (int d = 0; d < 3; ++d) {
        double u = (x[i][d] - pi->origin[d]) / pi->h;
        if (!(u >= 0.0 && u <= (double)(dims[d] - 1))) outside = 1;
      }
      nout += outside;
      double acc, am;
      receptor_sum(rc, L.type[i], x[i], &acc, &am);
      if (acc >= rc->cap) { acc = rc->cap; am = rc->cap; ++ncap; }
      ei += acc;
      mag += am;
    }
    double cl = 0.0, inv = 1.0 / (C.dc * C.dc);
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) {
        if (L.topo[(size_t)i * n + j] < C.min_sep) continue;
        double dx = x[i][0] - x[j][0], dy = x[i][1] - x[j][1], dz = x[i][2] - x[j][2];
        double t = 1.0 - (dx * dx + dy * dy + dz * dz) * inv;
        if (t > 0.0) cl += t * t;
      }
    e_inter[p] = ei;
    e_clash[p] = C.w * cl;
    n_out[p] = nout;
    n_capped[p] = ncap;
    if (scale) scale[p] = mag + fabs(C.w) * cl;
  }
  lig_free(&L);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Pose features for the learned pose selector (paper Sec. 3.5: a           */
/* high-throughput pose selector trading a little accuracy for much         */
/* throughput).  Per pose, 256 entries:                                      */
/*   [0, 64)   log1p of the count of atoms whose grid value v (trilinear, or  */
/*             the penalty) falls in bin min(63, max(0, floor(4 (v + 4))))   */
/*             -- 0.25-wide bins over [-4, 12);                              */
/*   [64, 72)  mean grid value of the atoms of each type 0..7 (0 if none);   */
/*   [72]      the docking score divided by the atom count;                  */
/*   [73]      the clash term (weight included);                             */
/*   [74]      log1p(atom count);  [75] rotatable-bond count;                */
/*   [76]      log1p of the count of atoms with v >= 9;                      */
/*   [77, 256) zero.                                                         */
/* The bin of v is decided in FP32: v is rounded to FP32 first (the GPU's    */
/* precision), so both sides bin the same value unless their values differ */
/* across an edge.                                                           */
OR_EXPORT int or_pose_features(const or_ligand_in *li, const or_pocket_in *pi, const or_sampling *sp,
                               int n_poses, const double *coords, double *out) {
  or_lig L;
  if (lig_init(&L, li->n_atoms, li->xyz, li->type, li->n_bonds, li->bonds, li->rot)) { lig_free(&L); return -1; }
  or_pocket P;
  make_pocket(pi, sp->penalty, &P);
  or_clash C = {sp->clash_w, sp->clash_dc, sp->clash_min_sep};
  const int n = L.n;
#pragma omp parallel for schedule(dynamic, 8)
  for (int p = 0; p < n_poses; ++p) {
    const double (*x)[3] = (const double(*)[3])(coords + (size_t)p * n * 3);
    double *f = out + (size_t)p * 256;
    for (int k = 0; k < 256; ++k) f[k] = 0.0;
    double cnt[64] = {0}, tsum[8] = {0}, tn[8] = {0}, e = 0.0, high = 0.0;
    for (int i = 0; i < n; ++i) {
      double v = trilinear(&P, L.type[i], x[i]);
      e += v;
      volatile float vf = (float)v;
      volatile float sc = (vf + 4.0f) * 4.0f;
      int b = (int)floorf(sc);
      b = b < 0 ? 0 : (b > 63 ? 63 : b);
      cnt[b] += 1.0;
      if (L.type[i] < 8) { tsum[L.type[i]] += v; tn[L.type[i]] += 1.0; }
      if (vf >= 9.0f) high += 1.0;
    }
    double cl = 0.0, inv = 1.0 / (C.dc * C.dc);
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) {
        if (L.topo[(size_t)i * n + j] < C.min_sep) continue;
        double dx = x[i][0] - x[j][0], dy = x[i][1] - x[j][1], dz = x[i][2] - x[j][2];
        double t = 1.0 - (dx * dx + dy * dy + dz * dz) * inv;
        if (t > 0.0) cl += t * t;
      }
    for (int b = 0; b < 64; ++b) f[b] = log1p(cnt[b]);
    for (int t = 0; t < 8; ++t) f[64 + t] = tn[t] > 0.0 ? tsum[t] / tn[t] : 0.0;
    f[72] = (e + C.w * cl) / n;
    f[73] = C.w * cl;
    f[74] = log1p((double)n);
    f[75] = (double)L.nrot;
    f[76] = log1p(high);
  }
  lig_free(&L);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Descriptor (256 entries, 233 used).                                       */
OR_EXPORT int or_descriptor(const or_ligand_in *li, int n_types, double *out) {
  if (n_types != 8) return -1;
  for (int k = 0; k < 256; ++k) out[k] = 0.0;
  int n = li->n_atoms;
  double counts[8] = {0};
  double hist[28][8];
  memset(hist, 0, sizeof(hist));
  for (int i = 0; i < n; ++i) counts[li->type[i]] += 1.0;
  static const float edge2[7] = {2.25f, 9.0f, 20.25f, 36.0f, 56.25f, 81.0f, 110.25f};
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      int a = li->type[i], b = li->type[j];
      if (a == b) continue;
      if (a > b) { int t = a; a = b; b = t; }
      /* pair index of (a, b), a < b, in lexicographic order */
      int p = a * 8 - a * (a + 1) / 2 + (b - a - 1);
      volatile float dx = li->xyz[3 * i] - li->xyz[3 * j];
      volatile float dy = li->xyz[3 * i + 1] - li->xyz[3 * j + 1];
      volatile float dz = li->xyz[3 * i + 2] - li->xyz[3 * j + 2];
      volatile float xx = dx * dx, yy = dy * dy, zz = dz * dz;
      volatile float s1 = xx + yy;
      volatile float d2 = s1 + zz;
      int bin = 0;
      for (int k = 0; k < 7; ++k) if (d2 >= edge2[k]) bin = k + 1;
      hist[p][bin] += 1.0;
    }
  int nrot = 0;
  for (int b = 0; b < li->n_bonds; ++b) nrot += li->rot[b] ? 1 : 0;
  for (int t = 0; t < 8; ++t) out[t] = log1p(counts[t]);
  for (int p = 0; p < 28; ++p)
    for (int k = 0; k < 8; ++k) out[8 + 8 * p + k] = log1p(hist[p][k]);
  out[232] = log1p((double)nrot);
  return 0;
}
