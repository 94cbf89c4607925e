// Internal declarations shared by the library's translation units.
// Device data layouts of the packed ligand batch, the pocket and the
// docking run, plus the host-side launch wrappers the C ABI calls.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ligate.h"

namespace ligate {

// ---------------------------------------------------------------------------
// Packed ligand batch (device).  Atoms of each ligand are renumbered in DFS
// pre-order from atom 0 (children by ascending input index), so the subtree
// moved by rotatable bond (u, v) is the contiguous range [v, end).
struct LigDesc {
  int atom_base;   // first atom in `atoms`
  int n_atoms;
  int n_rot;       // rotatable bonds, in sweep order at bond_base
  int bond_base;   // first record in `bonds`
  int elig_base;   // first word of the n_atoms x n_words clash-pair bit matrix
  int n_words;     // (n_atoms + 31) / 32
  long long cand_base;  // first clash candidate of this ligand in `cand`
};

// One rotatable bond: u (fixed-side atom), v (child atom), end (one past the
// subtree of v), and its clash candidates: the pairs (i, j) with i moved by
// the bond (v < i < end), j on the fixed side (outside [v, end), j != u) and
// at least 4 bonds apart, stored as i | j << 8 at cand[cand_base + cand_off].
// Only these pairs change distance while the bond turns.  An earlier bond
// (in sweep order) separates j from the moved subtree when exactly one of
// them lies in its subtree; only separating bonds' steps change a pair's
// geometry in this bond's sweep.  The list holds first the n_cand0 pairs no
// earlier bond separates (the same clash sums for every start), then the
// n_cand1 pairs that earlier bond e1 alone separates (sums that depend on
// e1's step only), then the rest.  e1 holds that bond's index in bits 0-15
// and, from bond 2 on, the ligand's running count of such bonds before this
// one in bits 16-31 (the bond's table slot); -1 when n_cand1 = 0.
struct BondRec {
  int u, v, end, n_cand;
  int cand_off;
  int n_cand0;
  int n_cand1;
  int e1;
};

struct BatchDev {
  int n_ligands = 0;
  int max_atoms = 0;
  int max_rot = 0;
  int64_t total_atoms = 0;
  LigDesc *lig = nullptr;    // [n_ligands]
  float4 *atoms = nullptr;   // [total_atoms] (x, y, z, type as int bits) DFS order
  BondRec *bonds = nullptr;  // [total_rot]
  uint32_t *elig = nullptr;  // clash-pair masks (topological distance >= 4)
  uint16_t *cand = nullptr;  // per-bond clash candidates (see BondRec)
  uint8_t *order = nullptr;  // [total_atoms] input index of the atom at each DFS position
  // host copies used for planning
  std::vector<LigDesc> h_lig;
  std::vector<BondRec> h_bonds;
  std::vector<uint32_t> h_elig;
  std::vector<uint16_t> h_cand;
  std::vector<uint8_t> h_types;   // per atom, DFS order
  std::vector<int32_t> h_rot;     // realised rotatable count per ligand
  std::vector<uint8_t> h_order;   // per atom, DFS order: input index within its ligand
};

// ---------------------------------------------------------------------------
struct PocketDev {
  int n_types = 0, nx = 0, ny = 0, nz = 0;
  double origin[3] = {0, 0, 0};
  double spacing = 0;
  int n_anchors = 0;
  float *anchors = nullptr;        // device [n_anchors][3] Angstrom
  std::vector<float> h_anchors;
  float *map_f32 = nullptr;        // plain [T][nz][ny][nx]
  float *map_f32c = nullptr;       // corner [T][cells][8]
  uint16_t *map_bf16c = nullptr;   // corner [T][cells][8]
  uint16_t *map_f16c = nullptr;    // corner [T][cells][8]
  float h_min[LIGATE_MAX_TYPES] = {};  // least value of each type's map (FP32)
  size_t n_nodes() const { return (size_t)nx * ny * nz; }
  size_t n_cells() const { return (size_t)(nx - 1) * (ny - 1) * (nz - 1); }
  // receptor for exact rescoring (ligate_pocket_set_receptor), grid units,
  // sorted by cell of a uniform grid whose cells are at least the cutoff
  // wide (x fastest), so the atoms within the cutoff of any point lie in
  // its 3 x 3 x 3 cell neighbourhood and each of its 9 rows of 3 cells is one
  // contiguous range
  float4 *rec = nullptr;           // [n_rec] (u, type bits)
  float2 *rec_pair = nullptr;      // [rec_types][rec_types] (r0^2 / h^2, eps)
  int *rec_cell = nullptr;         // [ncells + 1] first atom of each cell
  int n_rec = 0, rec_types = 0;
  float rec_cut2 = 0.f, rec_cap = 0.f, rec_rmin2 = 0.f;  // cutoff^2 / h^2, cap, rmin^2 / h^2
  int rec_nc[3] = {1, 1, 1};       // cells per axis (at most 16)
  float rec_lo[3] = {0, 0, 0};     // cell grid origin, grid units
  float rec_inv[3] = {0, 0, 0};    // 1 / cell width
};

// Receptor term of the exact rescoring, device view.
struct RecParams {
  const float4 *rec;
  const float2 *pair;
  const int *cell;          // [ncx ncy ncz + 1] first atom of each cell
  int n_rec, n_types;
  float cut2, cap, rmin2;
  float ox, oy, oz, inv_h;  // Angstrom -> grid units, for poses given as states
  int ncx, ncy, ncz;
  float lox, loy, loz, icx, icy, icz;
};

// Poses given as continuous states (ligate_pose_state at base + i * stride);
// the ligand index comes from lig_idx[i] or, with lig_idx NULL, from the
// int32 at base + i * stride + lig_offset (ligate_refined records, whose
// float at score_offset is not finite for an empty slot; -1: no such field).
struct StateSrc {
  const unsigned char *base;
  int stride, lig_offset, score_offset;
  const int32_t *lig_idx;
};

// Map-read modes of the docking kernel.
enum MapMode { MODE_F32_PLAIN = 0, MODE_F32_CORNER = 1, MODE_BF16_CORNER = 2, MODE_F16_CORNER = 3 };

// Geometry constants of one run (grid units: u = (x - origin) / h).
struct GridConst {
  int nx, ny, nz;
  float fx1, fy1, fz1;  // n - 1 as float (inclusive upper bound)
  float penalty;
  float cx, cy, cz;     // 2^23 + n - 2: the largest cell index in FP32 floor form
};

// One result slot in device memory (same bytes as ligate_pose).
struct PoseOut {
  float score;
  int32_t start_id;
  uint32_t tors[4];
};
static_assert(sizeof(PoseOut) == sizeof(ligate_pose), "pose layout");

// Work item: ligand of the batch, output row of the run (the ligand itself,
// or its position in a subset), start range, slot of its partial top-K list.
struct Item {
  int ligand;
  int row;
  int s0, s1;
  int slot;
  int pad[3];
};

// Work counters of a docking run (DockParams::stats): atom interpolations,
// clash candidates tested against the circle bound, surviving pairs,
// candidate pairs of the evaluated sweeps (memoised ones included; times S
// gives the pair trials), starts bounded out of the top-K, evaluated bond
// sweeps (each S trial poses, one of them the current pose).
constexpr int N_STATS = 6;

struct DockParams {
  // batch
  const LigDesc *lig;
  const float4 *atoms;
  const BondRec *bonds;
  const uint32_t *elig;
  const uint16_t *cand;
  int n_ligands;
  // pocket
  const void *maps;        // map read by the sweep (mode)
  const float *maps_f32;   // FP32 map for rescoring (plain)
  GridConst g;
  // start frames
  const float *rot;        // [n_orient][9] rotation / h (grid units)
  const float *anc;        // [n_anchor][3] (anchor - origin) / h
  int n_anchor;
  int n_starts;
  // sampling
  int S, L, G;             // torsion steps, lanes per start (pow2 >= S), groups per warp
  int K;
  float cs_tab[2 * LIGATE_MAX_STEPS];  // cos, sin of 2 pi k / S (host FP64, rounded)
  float clash_w;
  float inv_dc2_grid;      // h^2 / d_c^2
  float inv_dc2_ang;       // 1 / d_c^2
  float dc2_grid_margin;   // (d_c / h)^2 (1 + 1e-4): pairs beyond it never clash
  unsigned long long *stats;  // optional [N_STATS]: see N_STATS
  int rescore;
  // work queue
  const Item *items;
  int n_items;
  const int *n_items_dev;  // optional: the run's item count in device memory (subset runs); else n_items
  const int *lig_items;    // [n_ligands] items per ligand
  const int *lig_slot0;    // [n_ligands] first partial slot of each ligand
  int *queue;              // [1] next item
  int *done;               // [n_ligands] finished items per ligand
  unsigned *lig_thr;       // optional [n_ligands]: least K-th best energy any item of the row has
                           // reached, as ~(order-preserving key); 0 (reset value) = none yet
  const float *cut;        // optional [1], device: screening cutoff; a start stops once its bound
                           // exceeds it (null: none; see ligate_plan_set_cutoff)
  PoseOut *partial;        // [n_items][K]
  PoseOut *out;            // [n_ligands][K]
  // shared-memory shape
  int nmax;                // atoms capacity per warp slot (multiple of 32)
  int wmax;                // words per clash-mask row
  int rmax;                // rotatable bonds of the batch's largest ligand (memo rows)
  float *memo1;            // [resident warps][m1max][S][S] clash sums of the pairs one earlier bond
                           // separates, by that bond's step (null: those pairs are swept live)
  int m1max;               // tables per warp (bonds with such pairs, largest ligand)
  // optional [n_anchor]: the order a work item visits each orientation's
  // anchors in (consecutive entries are spatially close anchors, so the
  // start groups of a warp sweep similar poses); null: anchor order (plans
  // with more than 1,024 anchors, the allocation-free entry point)
  const uint16_t *visit;
  // smallest value an atom of each type can score: the least stored map
  // value (in the sweep map's precision) or the out-of-box penalty
  float gmin[LIGATE_MAX_TYPES];
};

// gmin of DockParams for the sweep map of layout `mode`.
void set_map_minima(DockParams &p, const PocketDev &d, int mode);

// Visiting order of the first n of the pocket's anchors (DockParams::visit):
// anchors paired greedily with their nearest remaining neighbour (Euclidean
// distance, ties to the smaller index), pairs in the order of their first
// anchor; deterministic.
std::vector<uint16_t> anchor_visit_order(const float *anchors_xyz, int n);

// cos/sin of the S torsion steps 2 pi k / S (k = 0 exactly (1, 0)), FP64
// rounded to FP32, into tab[2k], tab[2k + 1].
inline void fill_step_table(int S, float *tab) {
  for (int k = 0; k < LIGATE_MAX_STEPS; ++k) {
    const double a = 6.283185307179586476925286766559 * (double)k / (double)S;
    tab[2 * k] = k < S ? (float)(k == 0 ? 1.0 : std::cos(a)) : 1.f;
    tab[2 * k + 1] = k < S ? (float)(k == 0 ? 0.0 : std::sin(a)) : 0.f;
  }
}

// Exact rescoring (dock.cu): explicit poses (lig_idx, start_id, tors) or,
// with poses != NULL, a plan's output [n_poses / K][K] with row_lig.
size_t rescore_smem_bytes(const DockParams &p, const RecParams &r, int warps);
cudaError_t launch_rescore(const DockParams &p, const RecParams &r, int n_poses, const int32_t *lig_idx,
                           const int32_t *start_id, const uint8_t *tors, const ligate_pose *poses,
                           const int32_t *row_lig, const StateSrc *states, ligate_rescored *out,
                           cudaStream_t s);

// Per-pose selector features (dock.cu), [n_poses][256] FP32; explicit
// poses or a plan's output as for launch_rescore.
cudaError_t launch_pose_features(const DockParams &p, int n_poses, const int32_t *lig_idx,
                                 const int32_t *start_id, const uint8_t *tors, const ligate_pose *poses,
                                 const int32_t *row_lig, float *out, cudaStream_t s);

// Angstrom coordinates of continuous states, [n][LIGATE_MAX_ATOMS][3],
// atoms in input order (rescore.cu).
cudaError_t launch_state_coords(const DockParams &p, const uint8_t *order, int n, const int32_t *lig_idx,
                                const ligate_pose_state *states, float *out, cudaStream_t s);

// Per-ligand selection after rescoring (rescore.cu).
cudaError_t launch_best_passing(const ligate_rescored *rec, int n, int K, int32_t *idx, float *energy,
                                cudaStream_t s);
cudaError_t launch_select_poses(const float *pred, const ligate_pose *poses, int n, int K, float pass_below,
                                int32_t *idx, cudaStream_t s);
cudaError_t launch_selector_labels(const ligate_rescored *rec, long long n, float fail_label, float *out,
                                   cudaStream_t s);

// Pose refinement (refine.cu): mode 0 energy + gradient of explicit
// states, 1 refine explicit states, 2 refine a plan's poses.
size_t refine_smem_bytes(int nmax);
cudaError_t launch_refine(int mode, const DockParams &p, const double origin[3], double h, int n,
                          const int32_t *lig_idx, const ligate_pose_state *init, const ligate_pose *poses,
                          const int32_t *row_lig, int iters, float eta0, ligate_refined *out,
                          float *energy, float *grad, cudaStream_t s);

// Host launch wrappers (dock.cu).
size_t dock_smem_per_warp(int nmax, int S, int G, int rmax);
// Clash tables of ligand d the docking kernel keeps in memo1 (its swept
// bonds with pairs a single earlier bond separates).
int dock_memo1_tables(const LigDesc &d, const BondRec *bonds, int S);
cudaError_t launch_dock(int mode, int reg_cap, const DockParams &p, int grid, int block, size_t smem,
                        cudaStream_t s);
cudaError_t launch_start_frames(const double *quat_unused, const float *quat_f32_dev,
                                int n_orient, const float *anchors_dev, int n_anchor,
                                const double origin[3], double h, float *rot_out,
                                float *anc_out, cudaStream_t s);
cudaError_t launch_score_poses(int mode, const DockParams &p, int n_poses, const int32_t *lig_idx,
                               const int32_t *start_id, const uint8_t *tors, float *out,
                               cudaStream_t s);
// Grid-unit coordinates of explicit poses, [n_poses][LIGATE_MAX_ATOMS][3],
// atoms in input order (order: the batch's DFS-to-input map).
cudaError_t launch_pose_coords(const DockParams &p, const uint8_t *order, int n_poses, const int32_t *lig_idx,
                               const int32_t *start_id, const uint8_t *tors, float *out, cudaStream_t s);
int dock_kernel_max_ctas_per_sm(int mode, int reg_cap, int block, size_t smem);
// Local (spill) memory per thread of a kernel instance, in bytes.
size_t dock_kernel_local_bytes(int mode, int reg_cap);

// Pocket kernels (pocket.cu).
cudaError_t launch_corner_pack(const float *plain, int n_types, int nx, int ny, int nz,
                               int out_kind, void *out, cudaStream_t s);

// Random corner-cell gathers over a whole corner-packed map (words = 16-byte
// loads per cell): best time of three timed passes after a warm-up, and the
// bytes one pass reads (pocket.cu).
cudaError_t probe_gather(const void *cells, size_t n_cells, int words, int sms, double *ms_out,
                         double *bytes_out);

// Descriptor + surrogate kernels (surrogate.cu): declared there.

// Error helpers (api.cu).
// NVTX range over a scope (a named span on the profiler's timeline; free
// when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

void set_error(const char *fmt, ...);
ligate_status cuda_fail(cudaError_t e, const char *what);

}  // namespace ligate

// Opaque handles of the C ABI.
struct ligate_pocket {
  ligate::PocketDev d;
};
struct ligate_batch {
  ligate::BatchDev d;
  int max_type = 0;
};

