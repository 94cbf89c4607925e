/*
 * ligate.h - C ABI of the GB300 ligand dock+score library (libligate.so).
 *
 * What the library computes (paper Sec. 2, "LIGATE CADD workflow"): every
 * ligand of a chemical library is docked into a prepared target binding
 * site by a search with multiple restarts, each pose is scored by a
 * geometry-only function, and the ligand's score is the score of its best
 * pose; poses may then be re-scored.  Sec. 3.3 processes a BATCH of
 * ligand-pocket pairs per device, with ligands grouped by size (atom count,
 * rotatable-bond count) and batch shapes tuned per size.  Sec. 3.5 proposes
 * an affinity-prediction model on ligand features to speed the screening.
 *
 * The paper gives no formula for any of these steps; the concrete method
 * implemented here is:
 *   start s = o * n_anchor + a   : orientation o (unit quaternion) x pocket
 *                                  anchor a; x' = R_o (x - c) + anchor_a,
 *                                  c = centroid of the input conformation.
 *   torsion sweep (greedy)       : rotatable bonds in ascending DFS pre-order
 *                                  of their child atom (root = atom 0,
 *                                  children by ascending input index); for
 *                                  each bond try theta_k = 2 pi k / S,
 *                                  k = 0..S-1, rotating the child's subtree
 *                                  about the current u->v axis (right-hand
 *                                  rule), keep the best k (ties: smaller k).
 *   score E                      : sum_i G_type(i)(x'_i)  (trilinear
 *                                  interpolation of the type's grid map,
 *                                  out-of-grid atoms score `penalty`)
 *                                  + w sum_{pairs >= 4 bonds apart}
 *                                        max(0, 1 - d^2 / d_c^2)^2.
 *   top-K                        : the K starts with smallest (E, s).
 * Lower scores are better.
 *
 * Conventions (every entry point):
 *  - Returns LIGATE_OK or a negative ligate_status; no call aborts or exits.
 *    The text of the last error of the calling thread is available from
 *    ligate_last_error().
 *  - Input arrays are borrowed for the duration of the call; the library
 *    copies what it keeps.  Handles are owned by the caller and released
 *    with the matching *_destroy (NULL is accepted and ignored).
 *  - "host" pointers are ordinary CPU memory; "device" pointers are memory
 *    of the current CUDA device.  Calls are made on the current device.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls that return results to host memory synchronise the
 *    stream before returning; calls that write device memory only enqueue.
 */
#ifndef LIGATE_H
#define LIGATE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif
#if defined(__GNUC__)
#pragma GCC visibility push(default) /* the library builds with hidden default visibility */
#endif

typedef enum {
  LIGATE_OK = 0,
  LIGATE_ERR_INVALID = -1,     /* bad argument or malformed input */
  LIGATE_ERR_OOM = -2,         /* device or host allocation failed */
  LIGATE_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  LIGATE_ERR_TIMEOUT = -4,     /* a bounded wait ran out */
  LIGATE_ERR_UNSUPPORTED = -5  /* input beyond the documented limits */
} ligate_status;

/* Storage precision of the grid maps read by the docking kernel.  Every
 * precision interpolates and accumulates in FP32. */
typedef enum { LIGATE_FP32 = 0, LIGATE_BF16 = 1, LIGATE_FP16 = 2 } ligate_precision;

/* Map layouts.  PLAIN: [type][z][y][x] node values.  CORNER: for each cell
 * the 8 corner values stored contiguously (x fastest, then y, then z), so
 * one interpolation reads one 32 B (FP32) or 16 B (BF16/FP16) vector. */
typedef enum { LIGATE_LAYOUT_PLAIN = 0, LIGATE_LAYOUT_CORNER = 1 } ligate_layout;

/* Limits: atoms per ligand, rotatable bonds per ligand, torsion steps,
 * top-K, atom types. Larger inputs return LIGATE_ERR_UNSUPPORTED. */
#define LIGATE_MAX_ATOMS 128
#define LIGATE_MAX_ROT 16
#define LIGATE_MAX_STEPS 32
#define LIGATE_MAX_TOPK 32
#define LIGATE_MAX_TYPES 16

/* Pocket precision-mask bits for ligate_pocket_create. */
#define LIGATE_POCKET_FP32_CORNER (1u << 0)
#define LIGATE_POCKET_BF16_CORNER (1u << 1)
#define LIGATE_POCKET_FP16_CORNER (1u << 2)

const char *ligate_last_error(void); /* thread-local text, never NULL */
const char *ligate_version(void);

/* ------------------------------------------------------------------------
 * Prepared target pocket (paper Sec. 2: the target structure every docking
 * step needs).  maps: host FP32 [n_types][nz][ny][nx], node (ix,iy,iz) at
 * origin + spacing*(ix,iy,iz) Angstrom.  anchors: host FP32 [n_anchors][3]
 * Angstrom, the rigid-start translation points.  The FP32 plain layout is
 * always uploaded; `precision_mask` (LIGATE_POCKET_* bits) adds the
 * corner-packed copies, converted on the device (BF16/FP16 round to
 * nearest even).  Errors: INVALID (NULL, dims < 2, n_types outside
 * 1..LIGATE_MAX_TYPES, spacing <= 0, non-finite map value), OOM, CUDA. */
typedef struct ligate_pocket ligate_pocket;
ligate_status ligate_pocket_create(const float *maps, int n_types, int nx, int ny, int nz,
                                   const double origin[3], double spacing, const float *anchors,
                                   int n_anchors, unsigned precision_mask, ligate_pocket **out);
void ligate_pocket_destroy(ligate_pocket *pocket);

/* Measured ceiling of the docking kernel's map reads on this device (the
 * gather half of its roofline; the paper's Sec. 3.1 compares devices by
 * docking throughput): uniformly random corner-cell gathers over the whole
 * corner-packed map of `precision` (16 B per cell for BF16/FP16, 32 B for
 * FP32), four independent loads in flight per thread, all SMs, after one
 * warm-up pass; *gbs_out = bytes gathered / best time of three passes
 * (CUDA events), in GB/s.  Synchronous, on the legacy default stream.
 * Errors: INVALID, UNSUPPORTED (no such map in the pocket), CUDA. */
ligate_status ligate_probe_gather(const ligate_pocket *pocket, ligate_precision precision, double *gbs_out);

/* ------------------------------------------------------------------------
 * Ligand library (paper Sec. 2: ligands after 3D preparation; Sec. 3.3:
 * processed as a batch).  All host arrays, concatenated over ligands:
 *   atom_offset[n_ligands+1], xyz[atoms][3] (Angstrom, the input
 *   conformation), type[atoms] (< pocket n_types), bond_offset[n_ligands+1]
 *   with exactly n_atoms-1 bonds per ligand, bonds[bonds][2] (atom indices
 *   local to the ligand; the bonds must form a tree), rotatable[bonds] (0/1).
 * ligate_batch_create validates, renumbers every ligand in DFS pre-order,
 * builds its bond table and clash-pair masks on the host, and uploads the
 * packed batch to the device, where it stays until destroyed.
 * Errors: INVALID (not a tree, bad index or type, non-finite coordinate),
 * UNSUPPORTED (more than LIGATE_MAX_ATOMS atoms or LIGATE_MAX_ROT rotatable
 * bonds in a ligand), OOM, CUDA.  n_ligands == 0 is valid. */
typedef struct {
  int n_ligands;
  const int32_t *atom_offset;
  const float *xyz;
  const uint8_t *type;
  const int32_t *bond_offset;
  const int32_t *bonds;
  const uint8_t *rotatable;
} ligate_ligands;

typedef struct ligate_batch ligate_batch;
ligate_status ligate_batch_create(const ligate_ligands *ligands, ligate_batch **out);
void ligate_batch_destroy(ligate_batch *batch);

typedef struct {
  int n_ligands;
  int max_atoms;
  int max_rot;
  int64_t total_atoms;
} ligate_batch_info;
ligate_status ligate_batch_get_info(const ligate_batch *batch, ligate_batch_info *out);

/* How ligand li of L is packed for the docking kernel, on the host only (no
 * device work; usable without a GPU).  Paper Sec. 2: the torsion sweep turns
 * the rotatable bonds one by one; the clash term of a bond's sweep only
 * involves pairs across it, grouped here by the earlier bonds that separate
 * them (the kernel memoises the first two groups).
 *   *n_atoms_out, order_out (host int32[n_atoms], optional): the input index
 *     of the atom at each DFS pre-order position (children by ascending
 *     input index).
 *   *n_rot_out, bonds_out (host int32[n_rot][8], optional), in sweep order:
 *     u, v, end (DFS positions of the fixed-side atom, the child, and one
 *     past the child's subtree), n_cand, cand_off, n_cand0 (pairs no earlier
 *     bond separates), n_cand1 (pairs earlier bond e1 alone separates), e1
 *     (that bond's index in bits 0-15 and, from bond 2 on, its table slot in
 *     bits 16-31; -1 when n_cand1 = 0).
 *   cand_out (host uint16[cand_cap], optional): all candidates, i | j << 8
 *     in DFS positions, bond after bond; *n_cand_out is their count.
 * INVALID on bad arguments or cand_cap below the count (query the count
 * with cand_out NULL); the ligand's own errors as ligate_batch_create. */
ligate_status ligate_inspect_ligand(const ligate_ligands *L, int li, int *n_atoms_out,
                                    int32_t *order_out, int *n_rot_out, int32_t *bonds_out,
                                    uint16_t *cand_out, int cand_cap, int *n_cand_out);
/* Realised rotatable-bond count per ligand (host int32[n_ligands]). */
ligate_status ligate_batch_rot_counts(const ligate_batch *batch, int32_t *out);

/* ------------------------------------------------------------------------
 * Search parameters.  orientations: host FP64 [n_orient][4] quaternions
 * (w, x, y, z), normalised and re-orthonormalised in FP32 on the device.
 * The first n_anchor pocket anchors are used.  clash_weight w, clash
 * distance d_c (Angstrom), penalty = score of an out-of-grid atom.
 * rescore_fp32: re-score the top_k poses from the FP32 maps and re-sort
 * (the precision pattern for BF16/FP16 maps). */
typedef struct {
  int n_orient;
  int n_anchor;
  int torsion_steps;      /* S, 1..LIGATE_MAX_STEPS */
  int top_k;              /* K, 1..LIGATE_MAX_TOPK */
  const double *orientations;
  float clash_weight;
  float clash_cutoff;
  float penalty;
  ligate_precision precision;
  ligate_layout layout;   /* CORNER is required for BF16/FP16 */
  int rescore_fp32;
} ligate_sampling;

/* One result slot: score, start id (o * n_anchor + a, or -1 for an unused
 * slot when K exceeds the start count) and the chosen step of each
 * rotatable bond in sweep order (entries beyond the ligand's count are 0). */
typedef struct {
  float score;
  int32_t start_id;
  uint8_t tors[LIGATE_MAX_ROT];
} ligate_pose;

/* Launch shape of the persistent docking kernel (paper Sec. 3.3: batch
 * shapes tuned per ligand size).  Size bucket b of a ligand is
 * min(n_rot / 4, 3) + 4 * (n_atoms > 64); starts_per_item[b] is how many
 * starts one warp takes from the work queue at a time (a multiple of the
 * warp's start group, 32 / pow2ceil(S)).  A zeroed field means "default":
 * 4 warps, the mode's register cap, all SMs, chunks from the work model
 * (see ligate_model_tile). */
#define LIGATE_N_BUCKETS 8
typedef struct {
  int warps_per_cta;   /* 1..4 */
  int ctas_per_sm;
  int starts_per_item[LIGATE_N_BUCKETS];
  int reg_cap;         /* registers per thread: 1: at most 85 (6 CTAs of 128 threads per SM), 2: at most
                          102 (5 CTAs), 3: at most 128 (4 CTAs), 0: default (128 for the plain FP32
                          layout, 102 for the corner layouts) */
} ligate_tile;

/* ------------------------------------------------------------------------
 * Docking plan: packs the work queue (ligand x start-chunk items, largest
 * first), uploads the start frames, allocates the scratch and output
 * buffers and captures the whole docking run (queue reset, persistent
 * kernel, per-ligand merge and optional FP32 rescoring) into one CUDA graph
 * on first run.  tile == NULL picks the autotuner's cached shape for this
 * device (LIGATE_TUNE_CACHE file, see ligate_autotune) or the default.
 * The plan borrows pocket and batch: keep both alive until it is
 * destroyed.  Errors: INVALID, UNSUPPORTED (S, K or layout outside the
 * limits, BF16/FP16 without the matching pocket copy), OOM, CUDA. */
typedef struct ligate_plan ligate_plan;
ligate_status ligate_plan_create(const ligate_pocket *pocket, const ligate_batch *batch,
                                 const ligate_sampling *sampling, const ligate_tile *tile,
                                 ligate_plan **out);
/* Plan over a subset of the batch (paper Sec. 3.5: dock only the ligands a
 * cheaper predictor ranks best): ligands[0..n_ligands) are HOST indices into
 * the batch; output row r holds the poses of ligand ligands[r].  Errors as
 * ligate_plan_create, plus INVALID for an index outside the batch. */
ligate_status ligate_plan_create_subset(const ligate_pocket *pocket, const ligate_batch *batch,
                                        const ligate_sampling *sampling, const ligate_tile *tile,
                                        const int32_t *ligands, int n_ligands, ligate_plan **out);
/* Enqueue one docking run on `stream` (graph replay).  The result,
 * ligate_pose[n_ligands][top_k] in ligand order, stays in the plan's device
 * buffer (ligate_plan_output); if `out` is not NULL it is also copied there
 * (host or device pointer) and, for host memory, the stream is
 * synchronised.  The result is each ligand's top_k over all its starts;
 * a start's greedy sweep stops early once a lower bound of its final
 * energy (the grid energy of the atoms no later bond moves plus each
 * movable atom's map minimum) exceeds the top_k-th best energy already
 * found, which cannot change the result (ligate_work counts such starts). */
ligate_status ligate_plan_run(ligate_plan *plan, ligate_pose *out, void *stream);
/* Enqueue one docking run of a SELECTION of the plan's ligands (paper
 * Sec. 3.5: only the ligands a cheaper predictor ranks best are docked),
 * chosen on the device: ligands is a DEVICE int32 array of n_sel batch
 * indices (0 <= n_sel <= the plan's ligand count), e.g. the index output of
 * ligate_surrogate_rank; output row r holds the poses of ligands[r], the
 * same poses a full run gives that ligand.  The selected ligands' work
 * items are taken, in the plan's largest-first order, from the plan's own
 * item list on the device, so nothing waits for the host and no memory is
 * allocated after the first call.  A repeated or out-of-range index gives an
 * empty row (start ids -1).  The plan must have been created over the whole
 * batch (ligate_plan_create); `out` as for ligate_plan_run, n_sel rows.
 * After a subset run the post-docking stages below (refine, rescore,
 * features, best scores, best passing) act on its n_sel rows. */
ligate_status ligate_plan_run_subset(ligate_plan *plan, const int32_t *ligands, int n_sel, ligate_pose *out,
                                     void *stream);
ligate_status ligate_plan_output(const ligate_plan *plan, const ligate_pose **device_ptr);
/* Best score (the first pose) of every output row r of the plan's last run
 * into DEVICE out[r * stride + column] (FP32; +inf for a row without a
 * pose): e.g. a coarse docking run's scores into a free column of the
 * ligand descriptors, so the triage network sees them (enqueues). */
ligate_status ligate_plan_best_scores(const ligate_plan *plan, float *out, int stride, int column,
                                      void *stream);
/* Screening for a library's best ligands (paper Sec. 2: the campaign keeps
 * the ligands with the best scores; Sec. 3.5: cheaper passes first).
 *
 * ligate_plan_best_quantile: the k-th smallest of the last run's best
 * scores, k = ceil(frac * rows) (1 <= k <= rows), into DEVICE out[0]
 * (enqueues; the first call for a plan of a new size allocates scratch).
 * Run on a plan whose starts are a subset of another plan's (the same
 * pocket, precision, torsion steps and ligands; the first orientations and
 * anchors of the same lists), it gives a value at or above the k-th best
 * score that the full plan will find: each ligand's best over fewer starts
 * is at least its best over all of them.  The quantile is taken over the
 * scores the run reports, so for a cutoff in the search energies of the
 * plan it is attached to, take it from a plan that does not rescore.
 *
 * ligate_plan_set_cutoff: attach DEVICE cutoff[0] (NULL detaches it; the
 * value is read at each run, so it may be written on the device between
 * runs).  With a cutoff, a start also stops once the lower bound of its
 * final energy exceeds *cutoff (ligate_plan_run).  Every ligand whose best
 * energy in the run's map precision is at or below *cutoff gets its exact
 * best pose and all its top_k poses at or below *cutoff; other ligands may
 * report fewer poses or none (start_id -1, score +inf).  So the ligands with
 * the smallest scores up to the cutoff are found exactly.  Changing the
 * cutoff pointer synchronises the device and re-captures the plan's run.
 * Errors: INVALID, CUDA. */
ligate_status ligate_plan_best_quantile(ligate_plan *plan, double frac, float *out, void *stream);
ligate_status ligate_plan_set_cutoff(ligate_plan *plan, const float *cutoff);
/* Kernel launches one run enqueues, and the shape in use. */
ligate_status ligate_plan_get_tile(const ligate_plan *plan, ligate_tile *tile_out,
                                   int *kernel_launches);
/* Work done by one run, counted from the packed batch: unique poses
 * (n_starts * (1 + R (S - 1)) per ligand), atom interpolations and
 * clash-pair evaluations executed by the sweep. */
typedef struct {
  double poses;
  double atom_evals;   /* atom interpolations of the sweep (moved atoms x S per bond + N per start) */
  double pair_evals;   /* candidate clash pairs x S, before pruning */
  double starts;
  /* Counted on the device during the last run: atom interpolations, clash
   * candidate pairs tested against the circle bound (once per bond), and
   * surviving pairs (each evaluated at all S steps). 0 before a run. */
  double done_atom_evals;
  double done_pair_tests;
  double done_pair_survivors;
  /* Candidate clash pairs x S of the bond sweeps the run evaluated (the
   * counterpart of pair_evals after the bound), and the starts whose sweep
   * stopped because a lower bound of their final energy exceeded the K-th
   * best energy already found (they cannot enter the top-K). */
  double done_pair_evals;
  double done_pruned_starts;
  /* Bond sweeps the run evaluated (S trial poses each, one of them the pose
   * already held): the evaluated unique poses are starts + done_bond_sweeps
   * x (S - 1), against `poses` for the whole search space. */
  double done_bond_sweeps;
} ligate_work;
ligate_status ligate_plan_work(const ligate_plan *plan, ligate_work *out);
void ligate_plan_destroy(ligate_plan *plan);

/* One-call docking from HOST arrays to HOST results: packs the batch,
 * uploads it, runs a plan and copies ligate_pose[n_ligands][top_k] back. */
ligate_status ligate_dock_batch(const ligate_pocket *pocket, const ligate_ligands *ligands,
                                const ligate_sampling *sampling, ligate_pose *out, void *stream);

/* Allocation-free docking run.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc, such as a serving
 * process that reserves all device memory for its own pool at start-up, or
 * a latency-bound loop where cudaMalloc's implicit device synchronisation
 * is not acceptable.  It runs the same docking kernel as ligate_plan_run
 * (same results) but keeps all of its scratch (start frames, work items,
 * counters, partial top-K lists) in one fixed device array of
 * LIGATE_NOALLOC_SCRATCH_BYTES inside the library, so the call allocates
 * nothing on the device or the host heap.  pocket and batch are inputs the
 * caller created earlier; out is DEVICE ligate_pose[n_ligands][top_k].
 * The call only enqueues work on `stream`; the orientations travel inside
 * the kernel launches' parameters, so no host buffer must outlive it.
 *  - The array is reserved on a device when the library's device code for
 *    this entry point is loaded there.  With CUDA's default lazy module
 *    loading that happens during the first call on the device (which looks
 *    up the array's address, once per device, with that device current):
 *    make that first call before reserving the rest of the device for a
 *    pool, and before any stream capture, or run with
 *    CUDA_MODULE_LOADING=EAGER.  Later calls allocate nothing; the array
 *    stays until the process exits.
 *  - All calls share the array, which keeps the previous call's contents;
 *    each call clears the counters that must start at zero.  Calls whose
 *    GPU work overlaps (other streams, other host threads) race on it.
 *  - Limits: n_orient <= 1024, n_anchor <= 1024, and the run's scratch must
 *    fit the array: 49,152 B of start frames plus, per ligand,
 *    12 + ceil(n_orient * n_anchor / C) * (32 + 24 * top_k) B, where C is
 *    1024 starts rounded down to a multiple of the start group
 *    (32 / pow2ceil(torsion_steps)), plus up to 1,536 B of alignment.
 *    Larger requests return LIGATE_ERR_UNSUPPORTED with the sizes in
 *    ligate_last_error(). */
#define LIGATE_NOALLOC_SCRATCH_BYTES ((size_t)8 << 20)
ligate_status ligate_dock_noalloc(const ligate_pocket *pocket, const ligate_batch *batch,
                                  const ligate_sampling *sampling, ligate_pose *out, void *stream);

/* Scores of explicit poses (parity checks and rescoring): pose p is ligand
 * lig_idx[p] of the batch at start start_id[p] with torsion steps
 * tors[p][LIGATE_MAX_ROT] (sweep order).  All four arrays are DEVICE
 * memory; out is FP32 [n_poses].  `precision`/`layout` select the maps. */
ligate_status ligate_score_poses(const ligate_pocket *pocket, const ligate_batch *batch,
                                 const ligate_sampling *sampling, int n_poses,
                                 const int32_t *lig_idx, const int32_t *start_id,
                                 const uint8_t *tors, float *out, void *stream);

/* Coordinates of explicit poses, built exactly as the docking, rescoring and
 * feature kernels build them (paper Sec. 2: a docked pose is the ligand
 * placed by its rigid start and turned by its torsion steps; this is the
 * geometry a user writes out for the next stage).  Pose p is ligand
 * lig_idx[p] at start start_id[p] with steps tors[p][LIGATE_MAX_ROT]; all
 * four arrays are DEVICE memory.  out: DEVICE FP32
 * [n_poses][LIGATE_MAX_ATOMS][3] in grid units u = (x - origin) / spacing
 * (the frame the kernels score in; x = origin + spacing * u in Angstrom),
 * atoms in the ligand's INPUT order; rows past the ligand's atom count are
 * not written.  A pose whose ligand or start index is out of range gets NaN
 * in every row.  Synchronises stream.  Errors as ligate_score_poses. */
ligate_status ligate_pose_coords(const ligate_pocket *pocket, const ligate_batch *batch,
                                 const ligate_sampling *sampling, int n_poses, const int32_t *lig_idx,
                                 const int32_t *start_id, const uint8_t *tors, float *out, void *stream);

/* ------------------------------------------------------------------------
 * Pose refinement by gradient descent (paper Sec. 2: the docking search is a
 * gradient descent from multiple restarts; here the best poses of the
 * greedy sweep are the restarts and a local descent refines each one).
 *
 * A pose state is (R, t, phi): atom i sits at x_i = R (y_i - c) + t, with y
 * the input conformation after torsion angle phi_b (radians) is applied to
 * each rotatable bond b in sweep order about its current axis u -> v, c the
 * input centroid, R a rotation matrix (row-major) and t in Angstrom.  The
 * docked pose (start s, steps k) is R = R_o, t = anchor a, phi_b =
 * 2 pi k_b / S.  The energy is the docking score on the FP32 maps.  The
 * generalised gradient is (F, tau, psi): F = sum_i g_i, tau = sum_i
 * (x_i - t) x g_i and psi_b = n_b . sum_{i moved by b} (x_i - x_v) x g_i
 * with g_i = dE/dx_i and n_b the unit axis of bond b (the derivatives of E
 * along a translation, a rotation about t and a turn of bond b; the
 * trilinear derivative is the one of the atom's cell, zero for atoms
 * outside the maps).  Each descent iteration forms the trial
 * t - eta F / N, GS(exp([-eta tau / I_R]x) R), phi - eta psi / I_b with
 * I_R = 1 + sum_i |x_i - t|^2 and I_b = 1 + sum_{moved} |r_perp|^2 (A^2;
 * GS = Gram-Schmidt on the rows) and accepts it when it lowers E (eta
 * grows by 1.25) or rejects it (eta halves). */
typedef struct {
  float rot[9];                /* R, row-major */
  float trans[3];              /* t (Angstrom) */
  float tors[LIGATE_MAX_ROT];  /* phi_b (radians), bonds in sweep order; unused entries 0 */
} ligate_pose_state;
typedef struct {
  ligate_pose_state state;     /* refined state */
  float score_in;              /* energy at the starting state */
  float score;                 /* energy at the refined state (<= score_in) */
  uint32_t accepted;           /* bit i: the trial of iteration i was accepted */
  int32_t ligand;              /* batch index of the ligand */
} ligate_refined;
#define LIGATE_REFINE_MAX_ITERS 32
#define LIGATE_GRAD_DIM (6 + LIGATE_MAX_ROT) /* F (3), tau (3), psi (LIGATE_MAX_ROT) */

/* Energy and generalised gradient of n explicit states: pose p is ligand
 * lig_idx[p] of the batch in state states[p].  All arrays DEVICE memory;
 * energy [n], grad [n][LIGATE_GRAD_DIM] (entries of missing bonds 0).  A
 * ligand index outside the batch gives a NaN energy.  Synchronises stream. */
ligate_status ligate_pose_gradient(const ligate_pocket *pocket, const ligate_batch *batch,
                                   const ligate_sampling *sampling, int n, const int32_t *lig_idx,
                                   const ligate_pose_state *states, float *energy, float *grad,
                                   void *stream);
/* Coordinates of n continuous states as the refinement and the exact
 * rescoring build them (the geometry of a refined pose; paper Sec. 2: the
 * refined pose is the ligand's output).  DEVICE lig_idx [n] and states [n];
 * out DEVICE FP32 [n][LIGATE_MAX_ATOMS][3] in Angstrom, atoms in the
 * ligand's INPUT order; rows past the atom count are not written; an
 * out-of-range ligand index gives NaN rows.  Synchronises stream. */
ligate_status ligate_state_coords(const ligate_pocket *pocket, const ligate_batch *batch,
                                  const ligate_sampling *sampling, int n, const int32_t *lig_idx,
                                  const ligate_pose_state *states, float *out, void *stream);
/* Refine n explicit states (DEVICE arrays; out DEVICE [n]) for
 * `iterations` (0..LIGATE_REFINE_MAX_ITERS) descent iterations with
 * initial step eta0 > 0 (A^2 per score unit).  Synchronises stream. */
ligate_status ligate_refine_states(const ligate_pocket *pocket, const ligate_batch *batch,
                                   const ligate_sampling *sampling, int n, const int32_t *lig_idx,
                                   const ligate_pose_state *init, int iterations, float eta0,
                                   ligate_refined *out, void *stream);
/* Refine every pose of the plan's last run (its ligate_pose[n_ligands]
 * [top_k] device output) into DEVICE out[n_ligands][top_k], same order;
 * empty slots are copied with accepted = 0.  Enqueues on stream. */
ligate_status ligate_plan_refine(const ligate_plan *plan, int iterations, float eta0,
                                 ligate_refined *out, void *stream);

/* ------------------------------------------------------------------------
 * Exact rescoring and pose filter (paper Sec. 2: a more accurate scoring
 * of the generated poses, then a filter keeps the plausible ones).
 *
 * The receptor term of a pose is sum_i min(cap, sum_j eps_ij ((r0/r)^12 -
 * 2 (r0/r)^6)) over the receptor atoms j within `cutoff` of ligand atom i,
 * r floored at rmin, r0 = radius[t_i] + radius[t_j], eps_ij =
 * sqrt(eps[t_i] eps[t_j]): the pair potential the grid maps tabulate,
 * evaluated at the atom instead of interpolated, everywhere (no box
 * penalty).  The clash term is the docking score's.  A pose passes the
 * filter when no atom lies outside the map box and no atom's receptor sum
 * reaches the cap.
 *
 * Attach the receptor to a pocket (HOST arrays, copied): xyz [n][3] A,
 * type [n] in [0, n_types), radius/eps [n_types] (A, well depth); cutoff,
 * cap, rmin > 0.  Replaces a previous receptor.  n_types must cover every
 * ligand atom type of the batches rescored. */
ligate_status ligate_pocket_set_receptor(ligate_pocket *pocket, const float *xyz, const int32_t *type,
                                         int n_atoms, const float *radius, const float *eps,
                                         int n_types, float cutoff, float cap, float rmin);
typedef struct {
  float energy;       /* e_inter + e_clash; +inf for an empty slot */
  float e_inter;      /* exact receptor term */
  float e_clash;      /* clash term (weight included) */
  int32_t n_outside;  /* ligand atoms outside the map box (-1: empty slot) */
  int32_t n_capped;   /* ligand atoms whose receptor sum reached the cap */
  int32_t pass;       /* 1: n_outside == 0 and n_capped == 0 */
} ligate_rescored;
/* Explicit poses (DEVICE lig_idx, start_id, tors[n][LIGATE_MAX_ROT]; out
 * DEVICE [n]).  Errors: INVALID without a receptor or with ligand types
 * beyond it; UNSUPPORTED when the receptor (16 B per atom) does not fit in
 * shared memory (about 12,000 atoms).  Synchronises stream. */
ligate_status ligate_rescore_poses(const ligate_pocket *pocket, const ligate_batch *batch,
                                   const ligate_sampling *sampling, int n, const int32_t *lig_idx,
                                   const int32_t *start_id, const uint8_t *tors, ligate_rescored *out,
                                   void *stream);
/* Every pose of the plan's last run into DEVICE out[n_ligands][top_k]
 * (same order).  Enqueues on stream. */
ligate_status ligate_plan_rescore(const ligate_plan *plan, ligate_rescored *out, void *stream);
/* Poses given as continuous states (see ligate_pose_state): explicit DEVICE
 * lig_idx[n] and states[n] (synchronises), or the DEVICE records of a
 * ligate_plan_refine run of the same plan (refined[n_ligands][top_k], their
 * refined states; enqueues; empty slots, score_in not finite, give the
 * empty-slot record). */
ligate_status ligate_rescore_states(const ligate_pocket *pocket, const ligate_batch *batch,
                                    const ligate_sampling *sampling, int n, const int32_t *lig_idx,
                                    const ligate_pose_state *states, ligate_rescored *out, void *stream);
ligate_status ligate_plan_rescore_refined(const ligate_plan *plan, const ligate_refined *refined,
                                          ligate_rescored *out, void *stream);

/* A ligand's result after the filter (paper Sec. 2: the generated poses are
 * rescored and filtered; a ligand scores as its best pose): for every row r
 * of the plan's output, the slot k of the lowest energy among the rescored
 * poses of row r that pass the filter (ties: the smaller k), or -1 when none
 * passes.  rescored: DEVICE [n_ligands][top_k] as written by
 * ligate_plan_rescore or ligate_plan_rescore_refined for this plan; idx_out
 * DEVICE int32 [n_ligands]; energy_out (DEVICE FP32 [n_ligands], optional)
 * receives that energy (+inf when none passes).  Enqueues on stream. */
ligate_status ligate_plan_best_passing(const ligate_plan *plan, const ligate_rescored *rescored,
                                       int32_t *idx_out, float *energy_out, void *stream);

/* ------------------------------------------------------------------------
 * Per-pose selector features (paper Sec. 3.5: a high-throughput pose
 * selector trading a little accuracy for throughput; a learned model on
 * these features -- e.g. the triage surrogate network trained on exact
 * rescoring results -- picks the pose to keep without rescoring them all).
 * Per pose 256 FP32: [0, 64) log1p of the counts of atoms whose FP32 grid
 * value v (FP32 maps; the penalty outside) falls in bin min(63, max(0,
 * floor((v + 4) * 4))); [64, 72) mean v of the atoms of each type 0..7 (0
 * if none); [72] docking score / atom count; [73] clash term; [74]
 * log1p(atom count); [75] rotatable-bond count; [76] log1p of the count of
 * atoms with v >= 9; [77, 256) zero.  Explicit poses as in
 * ligate_rescore_poses (DEVICE arrays, out DEVICE [n][256], synchronises)
 * or every pose of a plan's last run (out DEVICE [n_ligands][top_k][256];
 * empty slots all zero; enqueues). */
ligate_status ligate_pose_features(const ligate_pocket *pocket, const ligate_batch *batch,
                                   const ligate_sampling *sampling, int n, const int32_t *lig_idx,
                                   const int32_t *start_id, const uint8_t *tors, float *out, void *stream);
ligate_status ligate_plan_pose_features(const ligate_plan *plan, float *out, void *stream);
/* The selector's decision rule (paper Sec. 3.5: keep one pose per ligand
 * from a learned prediction instead of rescoring every pose).  Per row r of
 * n rows of k poses in docking order (poses: DEVICE ligate_pose[n][k], a
 * slot with start_id < 0 is empty; pred: DEVICE FP32 [n][k], the network's
 * predicted label of each pose): the first non-empty slot whose prediction
 * is below pass_below (predicted to pass the filter); else the non-empty
 * slot with the lowest prediction (ties: the smaller slot); -1 for a row
 * without a pose.  idx_out: DEVICE int32 [n].  Enqueues on stream. */
ligate_status ligate_select_poses(const float *pred, const ligate_pose *poses, int n, int k,
                                  float pass_below, int32_t *idx_out, void *stream);
/* Training label of each rescored pose for the selector network: the exact
 * energy of a pose that passes the filter, clipped to fail_label, and
 * fail_label for a pose that fails or an empty slot.  rescored DEVICE [n],
 * out DEVICE FP32 [n].  Enqueues on stream. */
ligate_status ligate_selector_labels(const ligate_rescored *rescored, int64_t n, float fail_label,
                                     float *out, void *stream);

/* ------------------------------------------------------------------------
 * Autotuner (paper Sec. 3.3: per-size batch tuning).  Times the six CTA
 * shapes (2 or 4 warps x register caps 85 / 102 / 128) on up to 2048
 * ligands spread over the batch and writes the fastest to *best with zero
 * chunk fields (and to the cache file named by LIGATE_TUNE_CACHE, when set):
 * a plan fills zero chunk fields from the work model below for its own
 * batch, so a tuned shape carries over to batches of any size.  budget_ms
 * bounds the total measuring time. */
ligate_status ligate_autotune(const ligate_pocket *pocket, const ligate_batch *batch,
                              const ligate_sampling *sampling, double budget_ms,
                              ligate_tile *best);

/* Analytic launch model (paper Sec. 3.3: a batch shape per ligand size),
 * chosen without timing anything.  Shape: the CTA size and register cap
 * that keep the most warps resident on one SM under the register file and
 * shared-memory limits, among the kernel instances that do not spill
 * registers to local memory (for the plain FP32 layout only the
 * 128-register instances: its eight scalar gathers per interpolation need
 * registers for loads in flight).  Chunk of size bucket b (the work model, also used by
 * every plan for zero chunk fields): starts_per_item[b] = W / (8 P c_b)
 * clamped to [128, 2048] and rounded down to the start group, with W the
 * run's total work (sum over ligands of starts x per-start cost atoms +
 * 0.35 clash pairs + 40), P the resident warps of the whole GPU and c_b the
 * bucket's mean per-start cost: the largest item stays under an eighth of a
 * warp's share, small enough to balance the tail, large enough to amortise
 * loading a ligand.  Writes *out; needs the current device. */
ligate_status ligate_model_tile(const ligate_pocket *pocket, const ligate_batch *batch,
                                const ligate_sampling *sampling, ligate_tile *out);

/* ------------------------------------------------------------------------
 * Ligand descriptors for the triage surrogate (paper Sec. 3.5: ligand
 * features as input of an affinity predictor).  Per ligand 256 FP32:
 * [0,8) log1p of the count of each atom type, [8,232) log1p of 8-bin
 * histograms (edges 1.5, 3, ..., 10.5 A; last bin open) of intramolecular
 * distances for the 28 unordered pairs of distinct types in lexicographic
 * order, [232] log1p of the rotatable-bond count, [233,256) zero.  Needs
 * exactly 8 atom types.  out: DEVICE FP32 [n_ligands][256]. */
ligate_status ligate_descriptors(const ligate_batch *batch, float *out, void *stream);

/* ------------------------------------------------------------------------
 * Triage surrogate: MLP 256 -> 512 -> 512 -> 512 -> 1, ReLU hidden layers,
 * BF16 weights and activations on the tensor cores with FP32 accumulation,
 * FP32 master weights, Adam; inputs standardised with the training set's
 * per-feature mean/std, labels with the training labels' mean/std.
 * init_weights: host FP32, all layers concatenated as W1[256][512], b1,
 * W2[512][512], b2, W3[512][512], b3, W4[512][1], b4 (row-major, y = x W
 * + b), or NULL for He-normal weights drawn from `seed`. */
typedef struct ligate_surrogate ligate_surrogate;
#define LIGATE_SURROGATE_PARAMS (256 * 512 + 512 + 512 * 512 + 512 + 512 * 512 + 512 + 512 + 1)
ligate_status ligate_surrogate_create(const float *init_weights, uint64_t seed,
                                      ligate_surrogate **out);
void ligate_surrogate_destroy(ligate_surrogate *s);

/* Train on DEVICE desc[n][256] and labels[n] for `epochs` passes in
 * mini-batches of `batch` (the last partial batch is dropped), learning
 * rate lr; the epoch order is a permutation drawn from `seed`.  Sets the
 * standardisation statistics from these data on the first call.
 * loss_out (optional, host) receives the mean loss of the last epoch. */
ligate_status ligate_surrogate_train(ligate_surrogate *s, const float *desc, const float *labels,
                                     int n, int epochs, int batch, float lr, uint64_t seed,
                                     float *loss_out, void *stream);
/* Predicted scores (label units) of DEVICE desc[n][256] into DEVICE
 * pred[n]. */
ligate_status ligate_surrogate_predict(const ligate_surrogate *s, const float *desc, int n,
                                       float *pred, void *stream);
/* Indices of the ceil(n * keep_frac) ligands with the lowest predicted
 * score, best first (ties: smaller index), into DEVICE idx_out; pred_out
 * (DEVICE, optional) receives every prediction. */
ligate_status ligate_surrogate_rank(const ligate_surrogate *s, const float *desc, int n,
                                    double keep_frac, int32_t *idx_out, float *pred_out,
                                    void *stream);
/* The same ranking by the mean prediction of n_nets networks (host array
 * nets[n_nets], n_nets >= 1), e.g. the networks of a cross-fitted keep
 * fraction, each trained without one fold of the training library (paper
 * Sec. 3.5 keeps a predicted top fraction; the ensemble is what that
 * fraction was calibrated on, out of fold).  pred_out (DEVICE, optional)
 * receives the mean predictions.  INVALID on a NULL network or n_nets < 1. */
ligate_status ligate_surrogate_rank_ensemble(const ligate_surrogate *const *nets, int n_nets,
                                             const float *desc, int n, double keep_frac,
                                             int32_t *idx_out, float *pred_out, void *stream);

/* Low-level pieces of one training step, exposed for gradient checks:
 * forward + MSE + backward of one mini-batch on standardised DEVICE inputs
 * x[b][256] and targets t[b]; gradients (FP32, same layout as the weights)
 * into DEVICE grad[LIGATE_SURROGATE_PARAMS]; *loss_out (host) = MSE. */
ligate_status ligate_surrogate_grad(const ligate_surrogate *s, const float *x, const float *t,
                                    int b, float *grad, float *loss_out, void *stream);
/* Checkpoint of the whole training state (weights, Adam moments and step,
 * input and label standardisation) to a binary file and back; training
 * resumed from a loaded checkpoint continues exactly as it would have
 * without the save.  Errors: INVALID for an unreadable or foreign file. */
ligate_status ligate_surrogate_save(const ligate_surrogate *s, const char *path);
ligate_status ligate_surrogate_load(const char *path, ligate_surrogate **out);
/* Copy the FP32 master weights (host [LIGATE_SURROGATE_PARAMS]). */
ligate_status ligate_surrogate_get_weights(const ligate_surrogate *s, float *out);
/* Contraction engine chosen at creation: 1 when the forward layers and the
 * data gradients run on tcgen05 (TMA-fed, TMEM accumulators), 0 when they
 * run on the mma.sync kernels (environment LIGATE_MLP_GEMM=mma at creation
 * selects these; both use the same operands and rounding points), -1 for
 * a NULL handle.  Weight gradients always use mma.sync.  A tcgen05 wait
 * that runs out makes train/grad/predict/rank return LIGATE_ERR_TIMEOUT;
 * predict then returns only after its kernels have finished. */
int ligate_surrogate_engine(const ligate_surrogate *s);

/* Test hook for the failure path, not for normal use.  kind 1: the next CTA
 * of a tcgen05 contraction on the current device issues none of its tensor
 * loads, so its bounded wait on the first stage runs out (after 2 s); the
 * kernel records the timeout, releases its tensor memory and returns, and
 * the surrogate call that launched it returns LIGATE_ERR_TIMEOUT.  Nothing
 * hangs and the context stays usable.  Other kinds: INVALID. */
ligate_status ligate_debug_inject_fault(int kind);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif
#ifdef __cplusplus
}
#endif
#endif /* LIGATE_H */
