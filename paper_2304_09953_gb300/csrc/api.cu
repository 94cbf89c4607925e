// Host runtime behind the C ABI of include/ligate.h: error reporting, the
// pocket object, packing of ligand batches (DFS renumbering, bond table,
// clash-pair masks), docking plans (work queue, scratch, CUDA graph) and the
// autotuner.  Paper Sec. 2 (docking of every library ligand into a prepared
// pocket) and Sec. 3.3 (batches of ligand-pocket pairs, ligands grouped by
// atom and rotatable-bond count, batch shape tuned per size).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <fstream>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "ligate_internal.h"
#include "mlp.h"

namespace ligate {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

ligate_status cuda_fail(cudaError_t e, const char *what) {
  set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  return e == cudaErrorMemoryAllocation ? LIGATE_ERR_OOM : LIGATE_ERR_CUDA;
}

#define CK(call, what)                              \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

template <class T>
static cudaError_t dmalloc(T **p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  return cudaMalloc((void **)p, n * sizeof(T));
}

static int pow2ceil(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Host worker threads for the per-ligand packing loops, started on first use
// and kept for the life of the process (never destroyed: no join at exit).
// Starting and joining 15 threads costs about half a millisecond, and a
// batch runs two such loops.  One caller uses the pool at a time; a
// concurrent caller, or a forked child (which inherits no workers), runs
// its loop on threads of its own.
struct HostPool {
  std::mutex busy;  // held by the caller whose loop the workers run
  std::mutex m;     // guards the fields below
  std::condition_variable cv_work, cv_done;
  std::vector<std::thread> workers;
  pid_t pid = getpid();
  uint64_t gen = 0;  // loops handed out so far
  int pending = 0;   // workers not yet done with the current loop
  const std::function<void()> *job = nullptr;

  void work() {
    uint64_t seen = 0;
    for (;;) {
      const std::function<void()> *j;
      {
        std::unique_lock<std::mutex> g(m);
        cv_work.wait(g, [&] { return gen != seen; });
        seen = gen;
        j = job;
      }
      (*j)();
      std::lock_guard<std::mutex> g(m);
      if (--pending == 0) cv_done.notify_one();
    }
  }
};

static HostPool &host_pool() {
  static HostPool *pool = new HostPool();
  return *pool;
}

// fn(i) for every i in [0, n), handed out in blocks of 64 to `threads`
// threads (the caller's included).
static void parallel_for(int n, int threads, const std::function<void(int)> &fn) {
  std::atomic<int> next(0);
  const std::function<void()> body = [&]() {
    for (;;) {
      const int i0 = next.fetch_add(64);
      if (i0 >= n) break;
      for (int i = i0; i < std::min(n, i0 + 64); ++i) fn(i);
    }
  };
  if (threads <= 1) { body(); return; }
  HostPool &P = host_pool();
  std::unique_lock<std::mutex> busy(P.busy, std::try_to_lock);
  if (!busy.owns_lock() || P.pid != getpid()) {
    std::vector<std::thread> th;
    for (int t = 1; t < threads; ++t) th.emplace_back(body);
    body();
    for (auto &t : th) t.join();
    return;
  }
  {
    std::lock_guard<std::mutex> g(P.m);
    while ((int)P.workers.size() < threads - 1) P.workers.emplace_back([&P] { P.work(); });
    P.job = &body;
    P.pending = (int)P.workers.size();
    ++P.gen;
  }
  P.cv_work.notify_all();
  body();
  std::unique_lock<std::mutex> g(P.m);
  P.cv_done.wait(g, [&] { return P.pending == 0; });
  P.job = nullptr;
}

}  // namespace ligate

using namespace ligate;

// Least value an atom of each type can score in a sweep over the map of
// layout `mode`: the least FP32 map value rounded as the packed map stores
// it (round to nearest is monotonic, so this is the least stored value; a
// trilinear interpolation of stored values lies above it up to FP32
// rounding), or the out-of-box penalty if that is lower.
std::vector<uint16_t> ligate::anchor_visit_order(const float *xyz, int n) {
  std::vector<uint16_t> order;
  order.reserve(n);
  std::vector<char> used(n, 0);
  for (int a = 0; a < n; ++a) {
    if (used[a]) continue;
    used[a] = 1;
    order.push_back((uint16_t)a);
    int best = -1;
    double bd = 0;
    for (int c = 0; c < n; ++c) {
      if (used[c]) continue;
      const double dx = xyz[3 * a] - xyz[3 * c], dy = xyz[3 * a + 1] - xyz[3 * c + 1],
                   dz = xyz[3 * a + 2] - xyz[3 * c + 2];
      const double d2 = dx * dx + dy * dy + dz * dz;
      if (best < 0 || d2 < bd) { best = c; bd = d2; }
    }
    if (best >= 0) {
      used[best] = 1;
      order.push_back((uint16_t)best);
    }
  }
  return order;
}

void ligate::set_map_minima(DockParams &p, const PocketDev &d, int mode) {
  for (int t = 0; t < LIGATE_MAX_TYPES; ++t) {
    float v = t < d.n_types ? d.h_min[t] : 0.f;
    if (mode == MODE_BF16_CORNER) v = __bfloat162float(__float2bfloat16_rn(v));
    else if (mode == MODE_F16_CORNER) v = __half2float(__float2half_rn(v));
    p.gmin[t] = std::min(v, p.g.penalty);
  }
}


// ===========================================================================

extern "C" const char *ligate_last_error(void) { return g_err; }
extern "C" const char *ligate_version(void) { return "ligate-gb300 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
extern "C" ligate_status ligate_pocket_create(const float *maps, int n_types, int nx, int ny,
                                              int nz, const double origin[3], double spacing,
                                              const float *anchors, int n_anchors,
                                              unsigned precision_mask, ligate_pocket **out) {
  if (!out) { set_error("pocket_create: out is NULL"); return LIGATE_ERR_INVALID; }
  *out = nullptr;
  if (!maps || !origin || (!anchors && n_anchors > 0)) {
    set_error("pocket_create: NULL array");
    return LIGATE_ERR_INVALID;
  }
  if (n_types < 1 || n_types > LIGATE_MAX_TYPES || nx < 2 || ny < 2 || nz < 2 || n_anchors < 0 ||
      !(spacing > 0) || !isfinite(origin[0]) || !isfinite(origin[1]) || !isfinite(origin[2])) {
    set_error("pocket_create: invalid dimensions (types %d, grid %dx%dx%d, spacing %g)", n_types,
              nx, ny, nz, spacing);
    return LIGATE_ERR_INVALID;
  }
  if ((double)n_types * nx * ny * nz * 8.0 > 2147483647.0) {
    set_error("pocket_create: grid too large for 32-bit corner offsets");
    return LIGATE_ERR_UNSUPPORTED;
  }
  const size_t nodes = (size_t)nx * ny * nz;
  for (size_t i = 0; i < nodes * n_types; ++i)
    if (!isfinite(maps[i])) {
      set_error("pocket_create: non-finite map value at %zu", i);
      return LIGATE_ERR_INVALID;
    }
  for (int i = 0; i < 3 * n_anchors; ++i)
    if (!isfinite(anchors[i])) {
      set_error("pocket_create: non-finite anchor");
      return LIGATE_ERR_INVALID;
    }
  ligate_pocket *p = new ligate_pocket();
  PocketDev &d = p->d;
  d.n_types = n_types; d.nx = nx; d.ny = ny; d.nz = nz;
  for (int a = 0; a < 3; ++a) d.origin[a] = origin[a];
  d.spacing = spacing;
  d.n_anchors = n_anchors;
  d.h_anchors.assign(anchors, anchors + 3 * n_anchors);
  for (int t = 0; t < n_types; ++t) {  // each map's least value: the sweep's lower bounds
    const float *m = maps + (size_t)t * nodes;
    float lo = m[0];
    for (size_t i = 1; i < nodes; ++i) lo = std::min(lo, m[i]);
    d.h_min[t] = lo;
  }
  auto fail = [&](cudaError_t e, const char *w) {
    ligate_status st = cuda_fail(e, w);
    ligate_pocket_destroy(p);
    return st;
  };
  cudaError_t e;
  if ((e = dmalloc(&d.map_f32, nodes * n_types)) != cudaSuccess) return fail(e, "pocket maps");
  if ((e = cudaMemcpy(d.map_f32, maps, nodes * n_types * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail(e, "pocket upload");
  if ((e = dmalloc(&d.anchors, (size_t)3 * n_anchors)) != cudaSuccess) return fail(e, "anchors");
  if (n_anchors &&
      (e = cudaMemcpy(d.anchors, anchors, 12 * (size_t)n_anchors, cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail(e, "anchor upload");
  const size_t cells = d.n_cells() * n_types;
  if (precision_mask & LIGATE_POCKET_FP32_CORNER) {
    if ((e = dmalloc(&d.map_f32c, cells * 8)) != cudaSuccess) return fail(e, "corner maps");
    if ((e = launch_corner_pack(d.map_f32, n_types, nx, ny, nz, 0, d.map_f32c, 0)) != cudaSuccess)
      return fail(e, "corner pack");
  }
  if (precision_mask & LIGATE_POCKET_BF16_CORNER) {
    if ((e = dmalloc(&d.map_bf16c, cells * 8)) != cudaSuccess) return fail(e, "bf16 maps");
    if ((e = launch_corner_pack(d.map_f32, n_types, nx, ny, nz, 1, d.map_bf16c, 0)) != cudaSuccess)
      return fail(e, "bf16 pack");
  }
  if (precision_mask & LIGATE_POCKET_FP16_CORNER) {
    if ((e = dmalloc(&d.map_f16c, cells * 8)) != cudaSuccess) return fail(e, "fp16 maps");
    if ((e = launch_corner_pack(d.map_f32, n_types, nx, ny, nz, 2, d.map_f16c, 0)) != cudaSuccess)
      return fail(e, "fp16 pack");
  }
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e, "pocket prepare");
  *out = p;
  return LIGATE_OK;
}

extern "C" ligate_status ligate_probe_gather(const ligate_pocket *P, ligate_precision precision,
                                             double *gbs_out) {
  if (!P || !gbs_out) { set_error("probe_gather: NULL argument"); return LIGATE_ERR_INVALID; }
  const PocketDev &d = P->d;
  const void *cells = precision == LIGATE_FP32 ? (const void *)d.map_f32c
                    : precision == LIGATE_BF16 ? (const void *)d.map_bf16c : (const void *)d.map_f16c;
  if (!cells) {
    set_error("probe_gather: the pocket has no corner-packed map of this precision");
    return LIGATE_ERR_UNSUPPORTED;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "probe_gather");
  double ms = 0, bytes = 0;
  e = probe_gather(cells, d.n_cells() * (size_t)d.n_types, precision == LIGATE_FP32 ? 2 : 1, sms, &ms, &bytes);
  if (e != cudaSuccess) return cuda_fail(e, "probe_gather");
  *gbs_out = bytes / (ms * 1e-3) / 1e9;
  return LIGATE_OK;
}

extern "C" void ligate_pocket_destroy(ligate_pocket *p) {
  if (!p) return;
  cudaFree(p->d.map_f32);
  cudaFree(p->d.map_f32c);
  cudaFree(p->d.map_bf16c);
  cudaFree(p->d.map_f16c);
  cudaFree(p->d.anchors);
  cudaFree(p->d.rec);
  cudaFree(p->d.rec_pair);
  cudaFree(p->d.rec_cell);
  delete p;
}

extern "C" ligate_status ligate_pocket_set_receptor(ligate_pocket *P, const float *xyz, const int32_t *type,
                                                    int n, const float *radius, const float *eps,
                                                    int n_types, float cutoff, float cap, float rmin) {
  if (!P || n < 0 || (n > 0 && (!xyz || !type)) || n_types < 1 || n_types > 64 || !radius || !eps) {
    set_error("pocket_set_receptor: bad arguments");
    return LIGATE_ERR_INVALID;
  }
  if (!(cutoff > 0.f) || !std::isfinite(cutoff) || !std::isfinite(cap) || !(rmin > 0.f) || !std::isfinite(rmin)) {
    set_error("pocket_set_receptor: cutoff and rmin must be finite and > 0, cap finite");
    return LIGATE_ERR_INVALID;
  }
  for (int t = 0; t < n_types; ++t)
    if (!(radius[t] > 0.f) || !std::isfinite(radius[t]) || !(eps[t] >= 0.f) || !std::isfinite(eps[t])) {
      set_error("pocket_set_receptor: bad radius or eps of type %d", t);
      return LIGATE_ERR_INVALID;
    }
  const double h = P->d.spacing;
  std::vector<float4> rec((size_t)n);
  for (int j = 0; j < n; ++j) {
    if (type[j] < 0 || type[j] >= n_types || !std::isfinite(xyz[3 * j]) || !std::isfinite(xyz[3 * j + 1]) ||
        !std::isfinite(xyz[3 * j + 2])) {
      set_error("pocket_set_receptor: bad atom %d", j);
      return LIGATE_ERR_INVALID;
    }
    float tb;
    memcpy(&tb, &type[j], 4);  // type index as the int bits of .w
    rec[j] = make_float4((float)(((double)xyz[3 * j] - P->d.origin[0]) / h),
                         (float)(((double)xyz[3 * j + 1] - P->d.origin[1]) / h),
                         (float)(((double)xyz[3 * j + 2] - P->d.origin[2]) / h), tb);
  }
  // cell grid over the receptor: per axis n_c = floor(extent / (1.001
  // cutoff)) cells (1 to 16), each at least the cutoff wide with a margin
  // for FP32 rounding of the cell index on the device; the extent is padded
  // so no atom sits on the far face
  const double cut_g = (double)cutoff / h;
  int nc[3] = {1, 1, 1};
  double lo[3] = {0, 0, 0}, wd[3] = {1, 1, 1};
  for (int a = 0; a < 3 && n > 0; ++a) {
    double mn = 1e300, mx = -1e300;
    for (int j = 0; j < n; ++j) {
      const double x = a == 0 ? rec[j].x : a == 1 ? rec[j].y : rec[j].z;
      mn = std::min(mn, x);
      mx = std::max(mx, x);
    }
    const double ext = (mx - mn) * (1.0 + 1e-6) + 1e-3;
    nc[a] = (int)std::max(1.0, std::min(16.0, std::floor(ext / (1.001 * cut_g))));
    lo[a] = mn;
    wd[a] = ext / nc[a];
  }
  const int ncells = nc[0] * nc[1] * nc[2];
  std::vector<int> cell_of((size_t)n), start((size_t)ncells + 1, 0);
  for (int j = 0; j < n; ++j) {
    int c[3];
    for (int a = 0; a < 3; ++a) {
      const double x = a == 0 ? rec[j].x : a == 1 ? rec[j].y : rec[j].z;
      c[a] = std::min(nc[a] - 1, std::max(0, (int)std::floor((x - lo[a]) / wd[a])));
    }
    cell_of[j] = (c[2] * nc[1] + c[1]) * nc[0] + c[0];
    ++start[cell_of[j] + 1];
  }
  for (int c = 0; c < ncells; ++c) start[c + 1] += start[c];
  {
    std::vector<int> fill(start.begin(), start.end() - 1);
    std::vector<float4> sorted((size_t)n);
    for (int j = 0; j < n; ++j) sorted[fill[cell_of[j]]++] = rec[j];  // stable: input order within a cell
    rec.swap(sorted);
  }
  std::vector<float2> pair((size_t)n_types * n_types);
  for (int t = 0; t < n_types; ++t)
    for (int u = 0; u < n_types; ++u) {
      const double r0 = ((double)radius[t] + (double)radius[u]) / h;
      pair[(size_t)t * n_types + u] = make_float2((float)(r0 * r0), (float)std::sqrt((double)eps[t] * eps[u]));
    }
  cudaFree(P->d.rec);
  cudaFree(P->d.rec_pair);
  cudaFree(P->d.rec_cell);
  P->d.rec = nullptr;
  P->d.rec_pair = nullptr;
  P->d.rec_cell = nullptr;
  P->d.n_rec = 0;
  cudaError_t e;
  if ((n && ((e = dmalloc(&P->d.rec, (size_t)n)) != cudaSuccess ||
             (e = cudaMemcpy(P->d.rec, rec.data(), 16 * (size_t)n, cudaMemcpyHostToDevice)) != cudaSuccess)) ||
      (e = dmalloc(&P->d.rec_pair, pair.size())) != cudaSuccess ||
      (e = cudaMemcpy(P->d.rec_pair, pair.data(), 8 * pair.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = dmalloc(&P->d.rec_cell, start.size())) != cudaSuccess ||
      (e = cudaMemcpy(P->d.rec_cell, start.data(), 4 * start.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
    cudaFree(P->d.rec); cudaFree(P->d.rec_pair); cudaFree(P->d.rec_cell);
    P->d.rec = nullptr; P->d.rec_pair = nullptr; P->d.rec_cell = nullptr;
    return cuda_fail(e, "pocket_set_receptor");
  }
  for (int a = 0; a < 3; ++a) {
    P->d.rec_nc[a] = nc[a];
    P->d.rec_lo[a] = (float)lo[a];
    P->d.rec_inv[a] = (float)(1.0 / wd[a]);
  }
  P->d.n_rec = n;
  P->d.rec_types = n_types;
  P->d.rec_cut2 = (float)((double)cutoff * cutoff / (h * h));
  P->d.rec_cap = cap;
  P->d.rec_rmin2 = (float)((double)rmin * rmin / (h * h));
  return LIGATE_OK;
}

// ---------------------------------------------------------------------------
// Batch packing.
namespace {

struct LigPack {
  int n = 0, n_rot = 0, words = 0;
  int max_type = 0;
  std::vector<int> order;  // input index of the atom at each DFS position
  std::vector<float4> atoms;
  std::vector<BondRec> bonds;
  std::vector<uint32_t> elig;
  std::vector<uint8_t> types;
  std::vector<uint16_t> cand;
};

// Renumber one ligand in DFS pre-order, build its sweep-ordered bond table
// and the clash-pair bit matrix (pairs >= 4 bonds apart).
ligate_status pack_one(const ligate_ligands *L, int li, LigPack &P, char *err, size_t errlen) {
  const int a0 = L->atom_offset[li], a1 = L->atom_offset[li + 1];
  const int b0 = L->bond_offset[li], b1 = L->bond_offset[li + 1];
  const int n = a1 - a0, nb = b1 - b0;
  if (n < 1) { snprintf(err, errlen, "ligand %d has no atoms", li); return LIGATE_ERR_INVALID; }
  if (n > LIGATE_MAX_ATOMS) {
    snprintf(err, errlen, "ligand %d has %d atoms (limit %d)", li, n, LIGATE_MAX_ATOMS);
    return LIGATE_ERR_UNSUPPORTED;
  }
  if (nb != n - 1) {
    snprintf(err, errlen, "ligand %d: %d bonds for %d atoms (a tree needs n-1)", li, nb, n);
    return LIGATE_ERR_INVALID;
  }
  // adjacency as CSR (atom a's neighbours at nbr[off[a] .. off[a + 1]), ascending)
  // per-thread scratch, reused from ligand to ligand (packing runs on many
  // threads; the allocator would otherwise dominate)
  thread_local std::vector<int> off, nbr, fill, pos, parent, size, stack;
  thread_local std::vector<char> seen;
  off.assign(n + 1, 0);
  nbr.resize(2 * (size_t)nb);
  for (int b = b0; b < b1; ++b) {
    const int x = L->bonds[2 * b], y = L->bonds[2 * b + 1];
    if (x < 0 || y < 0 || x >= n || y >= n || x == y) {
      snprintf(err, errlen, "ligand %d: bond %d has bad atom index", li, b - b0);
      return LIGATE_ERR_INVALID;
    }
    ++off[x + 1];
    ++off[y + 1];
  }
  for (int a = 0; a < n; ++a) off[a + 1] += off[a];
  fill.assign(off.begin(), off.end() - 1);
  for (int b = b0; b < b1; ++b) {
    const int x = L->bonds[2 * b], y = L->bonds[2 * b + 1];
    nbr[fill[x]++] = y;
    nbr[fill[y]++] = x;
  }
  for (int a = 0; a < n; ++a) std::sort(nbr.begin() + off[a], nbr.begin() + off[a + 1]);
  pos.assign(n, -1);
  parent.assign(n, -1);
  size.assign(n, 1);
  stack.clear();
  std::vector<int> &order = P.order;
  order.clear();
  order.reserve(n);
  stack.push_back(0);
  parent[0] = -1;
  seen.assign(n, 0);
  seen[0] = 1;
  while (!stack.empty()) {
    const int a = stack.back();
    stack.pop_back();
    pos[a] = (int)order.size();
    order.push_back(a);
    for (int q = off[a + 1] - 1; q >= off[a]; --q) {  // push descending: pop ascending
      const int c = nbr[q];
      if (c == parent[a]) continue;
      if (seen[c]) { snprintf(err, errlen, "ligand %d: bonds contain a cycle", li); return LIGATE_ERR_INVALID; }
      seen[c] = 1;
      parent[c] = a;
      stack.push_back(c);
    }
  }
  if ((int)order.size() != n) {
    snprintf(err, errlen, "ligand %d: bonds do not connect all atoms", li);
    return LIGATE_ERR_INVALID;
  }
  for (int p = n - 1; p > 0; --p) size[parent[order[p]]] += size[order[p]];
  P.n = n;
  P.words = (n + 31) / 32;
  P.atoms.resize(n);
  P.types.resize(n);
  P.max_type = 0;
  for (int p = 0; p < n; ++p) {
    const int a = order[p];
    const float *x = L->xyz + 3 * (size_t)(a0 + a);
    if (!isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2])) {
      snprintf(err, errlen, "ligand %d: non-finite coordinate", li);
      return LIGATE_ERR_INVALID;
    }
    const int t = L->type[a0 + a];
    P.max_type = std::max(P.max_type, t);
    P.types[p] = (uint8_t)t;
    float4 v;
    v.x = x[0]; v.y = x[1]; v.z = x[2];
    int ti = t;
    memcpy(&v.w, &ti, 4);
    P.atoms[p] = v;
  }
  // rotatable bonds in sweep order (ascending DFS position of the child)
  std::vector<BondRec> br;
  for (int b = b0; b < b1; ++b) {
    if (!L->rotatable[b]) continue;
    const int x = L->bonds[2 * b], y = L->bonds[2 * b + 1];
    const int child = parent[y] == x ? y : x;
    const int par = child == y ? x : y;
    BondRec r;
    memset(&r, 0, sizeof(r));
    r.u = pos[par];
    r.v = pos[child];
    r.end = r.v + size[child];
    br.push_back(r);
  }
  if ((int)br.size() > LIGATE_MAX_ROT) {
    snprintf(err, errlen, "ligand %d has %zu rotatable bonds (limit %d)", li, br.size(), LIGATE_MAX_ROT);
    return LIGATE_ERR_UNSUPPORTED;
  }
  std::sort(br.begin(), br.end(), [](const BondRec &a, const BondRec &b) { return a.v < b.v; });
  P.n_rot = (int)br.size();
  // clash-eligible pairs in DFS numbering: topological distance >= 4, i.e.
  // every atom but those within 3 bonds.  Atoms within d bonds of atom a
  // (input numbering) as bit sets over DFS positions: within 0 = a itself,
  // within d = within d - 1 of a or of a neighbour of a
  const int W = P.words;
  thread_local std::vector<uint32_t> near0, near1;
  near0.assign((size_t)n * W, 0u);
  for (int a = 0; a < n; ++a) near0[(size_t)a * W + (pos[a] >> 5)] |= 1u << (pos[a] & 31);
  for (int d = 0; d < 3; ++d) {
    near1 = near0;
    for (int a = 0; a < n; ++a)
      for (int q = off[a]; q < off[a + 1]; ++q)
        for (int wd = 0; wd < W; ++wd) near1[(size_t)a * W + wd] |= near0[(size_t)nbr[q] * W + wd];
    near0.swap(near1);
  }
  P.elig.assign((size_t)n * W, 0u);
  for (int a = 0; a < n; ++a) {
    uint32_t *row = P.elig.data() + (size_t)pos[a] * W;
    for (int wd = 0; wd < W; ++wd) row[wd] = ~near0[(size_t)a * W + wd];
    if (n & 31) row[W - 1] &= (1u << (n & 31)) - 1u;
  }
  // clash candidates of each bond: moved atom i (v < i < end) x fixed atom j
  // (outside [v, end), j != u), at least 4 bonds apart; ordered by the
  // earlier bonds that separate j from the moved subtree (an earlier bond e
  // separates j when exactly one of j and v lies in e's subtree [v_e, end_e)):
  // none, then the most frequent single bond e1, then the rest
  // this ligand's candidates, written through a cursor into per-thread
  // scratch sized for every moved x other-atom pair, copied out at the end
  thread_local std::vector<uint16_t> cand;
  {
    size_t bound = 0;
    for (const BondRec &b : br) bound += (size_t)(b.end - b.v) * n;
    if (cand.size() < bound) cand.resize(bound);
  }
  uint16_t *const cw = cand.data();
  int nc = 0;
  // bitsets over DFS positions (at most LIGATE_MAX_ATOMS bits): for bond bi,
  // the atoms no earlier bond separates from the moved subtree, those exactly
  // one separates (and which one), and the rest; a candidate's group is its
  // fixed atom's
  constexpr int MW = LIGATE_MAX_ATOMS / 32;
  auto range_bits = [&](int lo, int hi, uint32_t *bits) {  // bits of [lo, hi)
    for (int wd = 0; wd < P.words; ++wd) {
      const int a = std::max(lo, 32 * wd) - 32 * wd, z = std::min(hi, 32 * wd + 32) - 32 * wd;
      bits[wd] = a >= z ? 0u : ((z - a == 32 ? ~0u : (1u << (z - a)) - 1u) << a);
    }
  };
  thread_local std::vector<uint32_t> sep;  // [bond e][MW]: atoms e separates from the current bond's subtree
  sep.assign(br.size() * MW, 0u);
  for (size_t bi = 0; bi < br.size(); ++bi) {
    BondRec &r = br[bi];
    r.cand_off = nc;
    uint32_t once[MW] = {0}, twice[MW] = {0};
    for (size_t e = 0; e < bi; ++e) {
      uint32_t *se = &sep[e * MW];
      range_bits(br[e].v, br[e].end, se);
      if (r.v >= br[e].v && r.v < br[e].end)
        for (int wd = 0; wd < P.words; ++wd) se[wd] = ~se[wd];
      if (n & 31) se[P.words - 1] &= (1u << (n & 31)) - 1u;
      for (int wd = 0; wd < P.words; ++wd) {
        twice[wd] |= once[wd] & se[wd];
        once[wd] |= se[wd];
      }
    }
    // eligible partners of moved atom i: clash-eligible, outside the moved
    // range [v, end) and not u
    uint32_t keep[MW];
    range_bits(r.v, r.end, keep);
    for (int wd = 0; wd < P.words; ++wd) keep[wd] = ~keep[wd];
    keep[r.u >> 5] &= ~(1u << (r.u & 31));
    auto partners = [&](int i, int wd) { return P.elig[(size_t)i * P.words + wd] & keep[wd]; };
    auto emit = [&](const uint32_t *group) {  // i ascending, then j ascending
      for (int i = r.v + 1; i < r.end; ++i)
        for (int wd = 0; wd < P.words; ++wd)
          for (uint32_t m = partners(i, wd) & group[wd]; m; m &= m - 1)
            cw[nc++] = (uint16_t)(i | ((32 * wd + __builtin_ctz(m)) << 8));
    };
    uint32_t none[MW];
    for (int wd = 0; wd < P.words; ++wd) none[wd] = ~once[wd];
    emit(none);
    r.n_cand0 = nc - r.cand_off;
    // e1: the earlier bond that alone separates the most candidates (ties:
    // the earlier bond)
    r.e1 = -1;
    int best = 0;
    for (size_t e = 0; e < bi; ++e) {
      int cnt = 0;
      for (int i = r.v + 1; i < r.end; ++i)
        for (int wd = 0; wd < P.words; ++wd)
          cnt += __builtin_popcount(partners(i, wd) & sep[e * MW + wd] & ~twice[wd]);
      if (cnt > best) { best = cnt; r.e1 = (int)e; }
    }
    uint32_t g1[MW] = {0}, rest_bits[MW];
    if (r.e1 >= 0)
      for (int wd = 0; wd < P.words; ++wd) g1[wd] = sep[r.e1 * MW + wd] & ~twice[wd];
    for (int wd = 0; wd < P.words; ++wd) rest_bits[wd] = once[wd] & ~g1[wd];
    emit(g1);
    r.n_cand1 = nc - r.cand_off - r.n_cand0;
    emit(rest_bits);
    r.n_cand = nc - r.cand_off;
  }
  for (size_t bi = 2, slot = 0; bi < br.size(); ++bi)  // table slots of bonds 2, 3, ...
    if (br[bi].n_cand1 > 0) br[bi].e1 |= (int)(slot++) << 16;
  P.bonds = br;
  P.cand.assign(cand.begin(), cand.begin() + nc);
  return LIGATE_OK;
}

}  // namespace

extern "C" ligate_status ligate_inspect_ligand(const ligate_ligands *L, int li, int *n_atoms_out,
                                              int32_t *order_out, int *n_rot_out, int32_t *bonds_out,
                                              uint16_t *cand_out, int cand_cap, int *n_cand_out) {
  if (!L || li < 0 || li >= L->n_ligands || !L->atom_offset || !L->xyz || !L->type || !L->bond_offset ||
      !L->bonds || !L->rotatable || !n_atoms_out || !n_rot_out || !n_cand_out || cand_cap < 0) {
    set_error("inspect_ligand: bad argument");
    return LIGATE_ERR_INVALID;
  }
  if (L->atom_offset[li + 1] < L->atom_offset[li] || L->bond_offset[li + 1] < L->bond_offset[li]) {
    set_error("inspect_ligand: offsets not ascending at ligand %d", li);
    return LIGATE_ERR_INVALID;
  }
  LigPack P;
  char buf[256];
  buf[0] = 0;
  const ligate_status st = pack_one(L, li, P, buf, sizeof(buf));
  if (st != LIGATE_OK) { set_error("inspect_ligand: %s", buf); return st; }
  *n_atoms_out = P.n;
  *n_rot_out = P.n_rot;
  *n_cand_out = (int)P.cand.size();
  if (order_out) std::copy(P.order.begin(), P.order.end(), order_out);
  if (bonds_out)
    for (int b = 0; b < P.n_rot; ++b) {
      const BondRec &r = P.bonds[b];
      const int32_t row[8] = {r.u, r.v, r.end, r.n_cand, r.cand_off, r.n_cand0, r.n_cand1, r.e1};
      std::copy(row, row + 8, bonds_out + 8 * (size_t)b);
    }
  if (cand_out) {
    if (cand_cap < (int)P.cand.size()) {
      set_error("inspect_ligand: %zu candidates, cand_cap %d", P.cand.size(), cand_cap);
      return LIGATE_ERR_INVALID;
    }
    std::copy(P.cand.begin(), P.cand.end(), cand_out);
  }
  return LIGATE_OK;
}

extern "C" ligate_status ligate_batch_create(const ligate_ligands *L, ligate_batch **out) {
  NvtxRange nvtx_("ligate:batch_create");
  if (!out || !L) { set_error("batch_create: NULL argument"); return LIGATE_ERR_INVALID; }
  *out = nullptr;
  const int n = L->n_ligands;
  if (n < 0) { set_error("batch_create: negative ligand count"); return LIGATE_ERR_INVALID; }
  if (n > 0 && (!L->atom_offset || !L->xyz || !L->type || !L->bond_offset || !L->bonds ||
                !L->rotatable)) {
    set_error("batch_create: NULL array");
    return LIGATE_ERR_INVALID;
  }
  if (n > 0 && (L->atom_offset[0] != 0 || L->bond_offset[0] != 0)) {
    set_error("batch_create: offsets must start at 0");
    return LIGATE_ERR_INVALID;
  }
  for (int i = 0; i < n; ++i)
    if (L->atom_offset[i + 1] < L->atom_offset[i] || L->bond_offset[i + 1] < L->bond_offset[i]) {
      set_error("batch_create: offsets not ascending at ligand %d", i);
      return LIGATE_ERR_INVALID;
    }
  std::vector<LigPack> packs(n);
  std::vector<ligate_status> st(n, LIGATE_OK);
  std::vector<std::string> errs(n);
  const unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  const int nthreads = n < 256 ? 1 : (int)nt;
  parallel_for(n, nthreads, [&](int i) {
    char buf[256];
    buf[0] = 0;
    st[i] = pack_one(L, i, packs[i], buf, sizeof(buf));
    if (st[i] != LIGATE_OK) errs[i] = buf;
  });
  for (int i = 0; i < n; ++i)
    if (st[i] != LIGATE_OK) {
      set_error("batch_create: %s", errs[i].c_str());
      return st[i];
    }
  ligate_batch *B = new ligate_batch();
  BatchDev &d = B->d;
  d.n_ligands = n;
  d.h_lig.resize(n);
  d.h_rot.resize(n);
  int64_t na = 0, nb = 0, ne = 0, nc = 0;
  for (int i = 0; i < n; ++i) {
    LigDesc &ld = d.h_lig[i];
    memset(&ld, 0, sizeof(ld));
    ld.atom_base = (int)na;
    ld.n_atoms = packs[i].n;
    ld.n_rot = packs[i].n_rot;
    ld.bond_base = (int)nb;
    ld.elig_base = (int)ne;
    ld.n_words = packs[i].words;
    ld.cand_base = nc;
    na += packs[i].n;
    nb += packs[i].n_rot;
    ne += (int64_t)packs[i].n * packs[i].words;
    nc += (int64_t)packs[i].cand.size();
    d.max_atoms = std::max(d.max_atoms, packs[i].n);
    d.max_rot = std::max(d.max_rot, packs[i].n_rot);
    B->max_type = std::max(B->max_type, packs[i].max_type);
    d.h_rot[i] = packs[i].n_rot;
  }
  if (na > 2147483647LL || ne > 2147483647LL) {
    delete B;
    set_error("batch_create: batch too large for 32-bit offsets");
    return LIGATE_ERR_UNSUPPORTED;
  }
  d.total_atoms = na;
  std::vector<float4> atoms(na);
  d.h_bonds.resize(nb);
  d.h_elig.resize(ne);
  d.h_types.resize(na);
  d.h_cand.resize(nc);
  d.h_order.resize(na);
  parallel_for(n, nthreads, [&](int i) {  // each ligand into its place, then release its pieces
    const LigDesc &ld = d.h_lig[i];
    LigPack &pk = packs[i];
    for (int q = 0; q < ld.n_atoms; ++q) d.h_order[ld.atom_base + q] = (uint8_t)pk.order[q];
    std::copy(pk.atoms.begin(), pk.atoms.end(), atoms.begin() + ld.atom_base);
    std::copy(pk.types.begin(), pk.types.end(), d.h_types.begin() + ld.atom_base);
    std::copy(pk.bonds.begin(), pk.bonds.end(), d.h_bonds.begin() + ld.bond_base);
    std::copy(pk.elig.begin(), pk.elig.end(), d.h_elig.begin() + ld.elig_base);
    std::copy(pk.cand.begin(), pk.cand.end(), d.h_cand.begin() + ld.cand_base);
    pk = LigPack();
  });
  cudaError_t e;
  if ((e = dmalloc(&d.lig, n)) != cudaSuccess || (e = dmalloc(&d.atoms, na)) != cudaSuccess ||
      (e = dmalloc(&d.bonds, nb)) != cudaSuccess || (e = dmalloc(&d.elig, ne)) != cudaSuccess ||
      (e = dmalloc(&d.cand, nc)) != cudaSuccess || (e = dmalloc(&d.order, na)) != cudaSuccess) {
    ligate_batch_destroy(B);
    return cuda_fail(e, "batch allocation");
  }
  if ((n && (e = cudaMemcpy(d.lig, d.h_lig.data(), sizeof(LigDesc) * n, cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (na && (e = cudaMemcpy(d.atoms, atoms.data(), sizeof(float4) * na, cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (nb && (e = cudaMemcpy(d.bonds, d.h_bonds.data(), sizeof(BondRec) * nb, cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (ne && (e = cudaMemcpy(d.elig, d.h_elig.data(), 4 * ne, cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (nc && (e = cudaMemcpy(d.cand, d.h_cand.data(), 2 * nc, cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (na && (e = cudaMemcpy(d.order, d.h_order.data(), na, cudaMemcpyHostToDevice)) != cudaSuccess)) {
    ligate_batch_destroy(B);
    return cuda_fail(e, "batch upload");
  }
  *out = B;
  return LIGATE_OK;
}

extern "C" void ligate_batch_destroy(ligate_batch *b) {
  if (!b) return;
  cudaFree(b->d.lig);
  cudaFree(b->d.atoms);
  cudaFree(b->d.bonds);
  cudaFree(b->d.elig);
  cudaFree(b->d.cand);
  cudaFree(b->d.order);
  delete b;
}

extern "C" ligate_status ligate_batch_get_info(const ligate_batch *b, ligate_batch_info *out) {
  if (!b || !out) { set_error("batch_get_info: NULL argument"); return LIGATE_ERR_INVALID; }
  out->n_ligands = b->d.n_ligands;
  out->max_atoms = b->d.max_atoms;
  out->max_rot = b->d.max_rot;
  out->total_atoms = b->d.total_atoms;
  return LIGATE_OK;
}

extern "C" ligate_status ligate_batch_rot_counts(const ligate_batch *b, int32_t *out) {
  if (!b || (!out && b->d.n_ligands)) { set_error("batch_rot_counts: NULL argument"); return LIGATE_ERR_INVALID; }
  std::copy(b->d.h_rot.begin(), b->d.h_rot.end(), out);
  return LIGATE_OK;
}

// ===========================================================================
// Plans.
namespace {

int bucket_of(const LigDesc &d) { return std::min(d.n_rot / 4, 3) + 4 * (d.n_atoms > 64); }

// Work of one start of ligand i (atom interpolations, clash pairs).
void start_work(const BatchDev &B, int i, int S, double &atoms, double &pairs) {
  const LigDesc &d = B.h_lig[i];
  atoms = d.n_atoms;
  pairs = 0;
  for (int b = 0; b < d.n_rot; ++b) {
    const BondRec &r = B.h_bonds[d.bond_base + b];
    atoms += (double)S * (r.end - r.v - 1);
    pairs += (double)S * r.n_cand;
  }
}

ligate_status check_sampling(const ligate_pocket *P, const ligate_batch *B, const ligate_sampling *s,
                             int *mode) {
  if (!P || !B || !s) { set_error("NULL pocket, batch or sampling"); return LIGATE_ERR_INVALID; }
  if (s->n_orient < 1 || s->n_anchor < 1 || !s->orientations) {
    set_error("sampling: need n_orient >= 1, n_anchor >= 1 and orientations");
    return LIGATE_ERR_INVALID;
  }
  if (s->n_anchor > P->d.n_anchors) {
    set_error("sampling: n_anchor %d exceeds the pocket's %d anchors", s->n_anchor, P->d.n_anchors);
    return LIGATE_ERR_INVALID;
  }
  if ((double)s->n_orient * s->n_anchor > 2147483647.0) {
    set_error("sampling: too many starts");
    return LIGATE_ERR_UNSUPPORTED;
  }
  if (s->torsion_steps < 1 || s->torsion_steps > LIGATE_MAX_STEPS) {
    set_error("sampling: torsion_steps %d outside 1..%d", s->torsion_steps, LIGATE_MAX_STEPS);
    return LIGATE_ERR_UNSUPPORTED;
  }
  if (s->top_k < 1 || s->top_k > LIGATE_MAX_TOPK) {
    set_error("sampling: top_k %d outside 1..%d", s->top_k, LIGATE_MAX_TOPK);
    return LIGATE_ERR_UNSUPPORTED;
  }
  if (!(s->clash_cutoff > 0) || !isfinite(s->clash_weight) || !isfinite(s->penalty)) {
    set_error("sampling: clash_cutoff must be > 0, weight and penalty finite");
    return LIGATE_ERR_INVALID;
  }
  for (int i = 0; i < 4 * s->n_orient; ++i)
    if (!isfinite(s->orientations[i])) { set_error("sampling: non-finite quaternion"); return LIGATE_ERR_INVALID; }
  for (int i = 0; i < s->n_orient; ++i) {
    const double *q = s->orientations + 4 * i;
    if (q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3] < 1e-12) {
      set_error("sampling: zero quaternion %d", i);
      return LIGATE_ERR_INVALID;
    }
  }
  if (B->d.n_ligands > 0 && B->max_type >= P->d.n_types) {
    set_error("batch uses atom type %d but the pocket has %d maps", B->max_type, P->d.n_types);
    return LIGATE_ERR_INVALID;
  }
  const PocketDev &d = P->d;
  if (s->precision == LIGATE_FP32 && s->layout == LIGATE_LAYOUT_PLAIN) *mode = MODE_F32_PLAIN;
  else if (s->precision == LIGATE_FP32 && s->layout == LIGATE_LAYOUT_CORNER) *mode = MODE_F32_CORNER;
  else if (s->precision == LIGATE_BF16 && s->layout == LIGATE_LAYOUT_CORNER) *mode = MODE_BF16_CORNER;
  else if (s->precision == LIGATE_FP16 && s->layout == LIGATE_LAYOUT_CORNER) *mode = MODE_F16_CORNER;
  else { set_error("sampling: unsupported precision/layout pair"); return LIGATE_ERR_UNSUPPORTED; }
  const void *m = *mode == MODE_F32_PLAIN ? (const void *)d.map_f32
                : *mode == MODE_F32_CORNER ? (const void *)d.map_f32c
                : *mode == MODE_BF16_CORNER ? (const void *)d.map_bf16c : (const void *)d.map_f16c;
  if (!m) {
    set_error("sampling: the pocket was created without this map precision/layout");
    return LIGATE_ERR_UNSUPPORTED;
  }
  return LIGATE_OK;
}

const void *mode_maps(const PocketDev &d, int mode) {
  return mode == MODE_F32_PLAIN ? (const void *)d.map_f32
       : mode == MODE_F32_CORNER ? (const void *)d.map_f32c
       : mode == MODE_BF16_CORNER ? (const void *)d.map_bf16c : (const void *)d.map_f16c;
}

// Start frames + everything of DockParams that does not depend on items.
ligate_status base_params(const ligate_pocket *P, const ligate_batch *B, const ligate_sampling *s,
                          int mode, DockParams &p, float **rot, float **anc, float **quat,
                          const float *rot_in = nullptr, const float *anc_in = nullptr) {
  const PocketDev &d = P->d;
  memset(&p, 0, sizeof(p));
  p.lig = B->d.lig; p.atoms = B->d.atoms; p.bonds = B->d.bonds; p.elig = B->d.elig;
  p.cand = B->d.cand;
  p.n_ligands = B->d.n_ligands;
  p.maps = mode_maps(d, mode);
  p.maps_f32 = d.map_f32;
  p.g.nx = d.nx; p.g.ny = d.ny; p.g.nz = d.nz;
  p.g.fx1 = (float)(d.nx - 1); p.g.fy1 = (float)(d.ny - 1); p.g.fz1 = (float)(d.nz - 1);
  p.g.penalty = s->penalty;
  p.g.cx = 8388608.f + (float)(d.nx - 2); p.g.cy = 8388608.f + (float)(d.ny - 2); p.g.cz = 8388608.f + (float)(d.nz - 2);
  set_map_minima(p, d, mode);
  p.n_anchor = s->n_anchor;
  p.n_starts = s->n_orient * s->n_anchor;
  p.S = s->torsion_steps;
  fill_step_table(p.S, p.cs_tab);
  p.L = pow2ceil(s->torsion_steps);
  p.G = 32 / p.L;
  p.K = s->top_k;
  p.clash_w = s->clash_weight;
  p.inv_dc2_ang = (float)(1.0 / ((double)s->clash_cutoff * s->clash_cutoff));
  p.inv_dc2_grid = (float)(d.spacing * d.spacing / ((double)s->clash_cutoff * s->clash_cutoff));
  p.dc2_grid_margin = (float)((double)s->clash_cutoff * s->clash_cutoff / (d.spacing * d.spacing) * (1.0 + 1e-4));
  p.rescore = s->rescore_fp32 ? 1 : 0;
  p.nmax = std::max(32, (B->d.max_atoms + 31) / 32 * 32);
  p.wmax = p.nmax / 32;
  p.rmax = B->d.max_rot;
  if (rot_in && anc_in) {  // frames of the same sampling and pocket, owned by another plan
    *rot = *anc = *quat = nullptr;
    p.rot = rot_in;
    p.anc = anc_in;
    return LIGATE_OK;
  }
  std::vector<float> qf(4 * (size_t)s->n_orient);
  for (size_t i = 0; i < qf.size(); ++i) qf[i] = (float)s->orientations[i];
  CK(dmalloc(quat, qf.size()), "quaternions");
  CK(cudaMemcpy(*quat, qf.data(), 4 * qf.size(), cudaMemcpyHostToDevice), "quaternion upload");
  CK(dmalloc(rot, 9 * (size_t)s->n_orient), "start frames");
  CK(dmalloc(anc, 3 * (size_t)s->n_anchor), "start frames");
  CK(launch_start_frames(nullptr, *quat, s->n_orient, d.anchors, s->n_anchor, d.origin, d.spacing,
                         *rot, *anc, 0), "start frames");
  // the frames are read by kernels on the caller's stream, which need not
  // be ordered after the legacy default stream
  CK(cudaStreamSynchronize(0), "start frames");
  p.rot = *rot;
  p.anc = *anc;
  return LIGATE_OK;
}

int device_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

struct ligate_plan {
  DockParams p;
  int mode = 0;
  ligate_tile tile;
  int grid = 0, block = 0;
  size_t smem = 0;
  int n_ligands = 0;
  float *rot = nullptr, *anc = nullptr, *quat = nullptr;
  uint16_t *visit = nullptr;  // anchor visiting order (DockParams::visit)
  // scratch of ligate_plan_best_quantile (grown on demand): best scores,
  // sort keys and sorted indices, q_cap entries each
  float *q_scores = nullptr;
  unsigned long long *q_keys = nullptr;
  int32_t *q_idx = nullptr;
  int q_cap = 0;
  Item *items = nullptr;
  int *lig_items = nullptr, *lig_slot0 = nullptr, *counters = nullptr;
  PoseOut *partial = nullptr, *out = nullptr;
  int32_t *row_lig = nullptr;  // [n_ligands] batch index of each output row
  const ligate_pocket *pocket = nullptr;
  const ligate_batch *batch = nullptr;
  double origin[3] = {0, 0, 0}, h = 1.0;
  size_t counter_bytes = 0;
  unsigned long long *stats = nullptr;  // [N_STATS] executed-work counters of the last run
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ligate_work work;
  bool is_subset = false;          // created over a subset (ligate_plan_create_subset)
  // rows of the last run and their batch indices (the whole plan, or a
  // ligate_plan_run_subset selection): what the post-docking stages read
  int rows = 0;
  const int32_t *cur_row_lig = nullptr;
  // subset runs (ligate_plan_run_subset): the work model's inputs for the
  // whole batch, the ligands in descending per-start cost and their size
  // buckets (device, built on the first subset run), and the run's buffers
  double model_W = 0.0, model_cb[LIGATE_N_BUCKETS] = {0};
  int32_t *lig_by_cost = nullptr;
  uint8_t *lig_bucket = nullptr;
  size_t sub_cap = 0;              // capacity of sub_items (items) and sub_partial (items x K poses)
  Item *sub_items = nullptr;
  PoseOut *sub_partial = nullptr;
  int *sub_count = nullptr, *sub_lig_items = nullptr, *sub_slot0 = nullptr;
  int32_t *rowmap = nullptr, *sub_row_lig = nullptr;
};

static void free_plan(ligate_plan *pl) {
  if (!pl) return;
  cudaFree(pl->sub_items); cudaFree(pl->sub_partial); cudaFree(pl->sub_count); cudaFree(pl->sub_lig_items);
  cudaFree(pl->sub_slot0); cudaFree(pl->rowmap); cudaFree(pl->sub_row_lig); cudaFree(pl->lig_by_cost);
  cudaFree(pl->lig_bucket);
  cudaFree(pl->p.memo1);
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
  cudaFree(pl->rot); cudaFree(pl->anc); cudaFree(pl->quat); cudaFree(pl->visit);
  cudaFree(pl->q_scores); cudaFree(pl->q_keys); cudaFree(pl->q_idx);
  cudaFree(pl->items); cudaFree(pl->lig_items); cudaFree(pl->lig_slot0);
  cudaFree(pl->counters); cudaFree(pl->partial); cudaFree(pl->out); cudaFree(pl->stats);
  cudaFree(pl->row_lig);
  delete pl;
}

// Tile shape: explicit, from the autotuner cache file, or the default.
static bool read_tune_cache(int S, int mode, ligate_tile *t);

static void default_tile(ligate_tile *t) {
  if (t->warps_per_cta <= 0) t->warps_per_cta = 4;
}

// Work model of the launch (paper Sec. 3.3: a batch shape per ligand size):
// chunk of size bucket b = W / (8 P c_b) starts, clamped to [128, 2048] and
// rounded down to the start group, with W the run's total work (starts x
// per-start cost atoms + 0.35 clash pairs + 40, the queue's own estimate),
// P the warps resident on the whole GPU and c_b the bucket's mean per-start
// cost: the largest item stays under an eighth of a warp's share (tail
// balance) while still amortising the load of a ligand and its clash memo.
// Buckets without ligands get 512.  Ligands: sel[0..n) or all of B.
static void model_chunks(const BatchDev &B, const int32_t *sel, int n, int S, int n_starts, double P_warps,
                         int G, int *chunks) {
  double W = 0.0, cb[LIGATE_N_BUCKETS] = {0}, nb[LIGATE_N_BUCKETS] = {0};
  for (int r = 0; r < n; ++r) {
    const int i = sel ? sel[r] : r;
    double a, q;
    start_work(B, i, S, a, q);
    const double c = a + 0.35 * q + 40.0;
    W += c * n_starts;
    const int b = bucket_of(B.h_lig[i]);
    cb[b] += c;
    nb[b] += 1.0;
  }
  for (int b = 0; b < LIGATE_N_BUCKETS; ++b) {
    double chunk = 512.0;
    if (nb[b] > 0) chunk = W / (8.0 * std::max(P_warps, 1.0) * (cb[b] / nb[b]));
    chunk = std::min(2048.0, std::max(128.0, chunk));
    chunks[b] = std::max(G, (int)chunk / G * G);
  }
}

// Plan over all ligands of B (sel == NULL) or over the ligands sel[0..n_sel),
// whose results fill output rows 0..n_sel-1 in that order.
// Options of plans made inside the library: start frames borrowed from a
// plan of the same pocket and sampling, and no device-wide synchronisation
// at the end (the caller orders the set-up copies before its launch).
struct PlanOpts {
  const float *rot = nullptr, *anc = nullptr;
  bool no_device_sync = false;
};

static ligate_status plan_create_impl(const ligate_pocket *P, const ligate_batch *B,
                                      const ligate_sampling *s, const ligate_tile *tile,
                                      const int32_t *sel, int n_sel, ligate_plan **out,
                                      const PlanOpts *opt = nullptr) {
  NvtxRange nvtx_("ligate:plan_create");
  if (!out) { set_error("plan_create: out is NULL"); return LIGATE_ERR_INVALID; }
  *out = nullptr;
  int mode = 0;
  ligate_status st = check_sampling(P, B, s, &mode);
  if (st != LIGATE_OK) return st;
  if (sel) {
    if (n_sel < 0) { set_error("plan_create_subset: negative count"); return LIGATE_ERR_INVALID; }
    for (int r = 0; r < n_sel; ++r)
      if (sel[r] < 0 || sel[r] >= B->d.n_ligands) {
        set_error("plan_create_subset: index %d at position %d outside the batch", sel[r], r);
        return LIGATE_ERR_INVALID;
      }
  }
  ligate_plan *pl = new ligate_plan();
  pl->mode = mode;
  pl->n_ligands = sel ? n_sel : B->d.n_ligands;
  pl->is_subset = sel != nullptr;
  for (int d = 0; d < 3; ++d) pl->origin[d] = P->d.origin[d];
  pl->h = P->d.spacing;
  pl->pocket = P;
  pl->batch = B;
  {
    std::vector<int32_t> rl(pl->n_ligands);
    for (int r = 0; r < pl->n_ligands; ++r) rl[r] = sel ? sel[r] : r;
    cudaError_t e0;
    if (!rl.empty() && ((e0 = dmalloc(&pl->row_lig, rl.size())) != cudaSuccess ||
                        (e0 = cudaMemcpy(pl->row_lig, rl.data(), 4 * rl.size(), cudaMemcpyHostToDevice)) != cudaSuccess)) {
      free_plan(pl);
      return cuda_fail(e0, "plan allocation");
    }
  }
  st = base_params(P, B, s, mode, pl->p, &pl->rot, &pl->anc, &pl->quat, opt ? opt->rot : nullptr,
                   opt ? opt->anc : nullptr);
  if (st != LIGATE_OK) { free_plan(pl); return st; }
  DockParams &p = pl->p;
  if (s->n_anchor <= 1024) {  // consecutive starts of a work item at nearby anchors (O(n^2) pairing)
    const std::vector<uint16_t> order = anchor_visit_order(P->d.h_anchors.data(), s->n_anchor);
    cudaError_t e = dmalloc(&pl->visit, order.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(pl->visit, order.data(), sizeof(uint16_t) * order.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { free_plan(pl); return cuda_fail(e, "plan allocation"); }
    p.visit = pl->visit;
  }
  const int sms = device_sms();
  memset(&pl->tile, 0, sizeof(pl->tile));
  if (tile) pl->tile = *tile;
  else read_tune_cache(p.S, mode, &pl->tile);
  default_tile(&pl->tile);
  ligate_tile &t = pl->tile;
  t.warps_per_cta = std::max(1, std::min(4, t.warps_per_cta));
  if (t.reg_cap < 0 || t.reg_cap > 3) t.reg_cap = 0;
  {  // fewer warps per CTA when large ligands or many start groups need more shared memory
    const size_t per_warp = dock_smem_per_warp(p.nmax, p.S, p.G, p.rmax);
    const int fit = (int)std::max<size_t>(1, (size_t)(227 * 1024) / per_warp);
    t.warps_per_cta = std::min(t.warps_per_cta, fit);
  }
  pl->block = 32 * t.warps_per_cta;
  pl->smem = dock_smem_per_warp(p.nmax, p.S, p.G, p.rmax) * t.warps_per_cta;
  if (pl->smem > 227 * 1024) {
    free_plan(pl);
    set_error("plan_create: %zu B shared memory per CTA exceeds 227 KB; use fewer warps", pl->smem);
    return LIGATE_ERR_UNSUPPORTED;
  }
  const int occ = dock_kernel_max_ctas_per_sm(mode, t.reg_cap, pl->block, pl->smem);
  if (occ < 1) {
    free_plan(pl);
    set_error("plan_create: kernel cannot be resident with %d threads, %zu B shared memory",
              pl->block, pl->smem);
    return LIGATE_ERR_UNSUPPORTED;
  }
  t.ctas_per_sm = t.ctas_per_sm > 0 ? std::min(t.ctas_per_sm, occ) : occ;
  pl->grid = sms * t.ctas_per_sm;
  {  // chunks not given: the work model for this batch and these resident warps
    int mc[LIGATE_N_BUCKETS];
    model_chunks(B->d, sel, pl->n_ligands, p.S, p.n_starts, (double)pl->grid * t.warps_per_cta, p.G, mc);
    for (int b = 0; b < LIGATE_N_BUCKETS; ++b)
      if (t.starts_per_item[b] <= 0) t.starts_per_item[b] = mc[b];
  }
  for (int b = 0; b < LIGATE_N_BUCKETS; ++b)
    t.starts_per_item[b] = std::max(p.G, t.starts_per_item[b] / p.G * p.G);
  {  // keep the partial top-K lists (items x K poses) within 1 GiB: larger chunks for large batches
    const double budget = 1024.0 * 1024.0 * 1024.0;
    const int smallest = *std::min_element(t.starts_per_item, t.starts_per_item + LIGATE_N_BUCKETS);
    const double bytes = (double)pl->n_ligands * std::ceil((double)p.n_starts / smallest) * p.K *
                         sizeof(PoseOut);
    if (bytes > budget) {
      const double f = bytes / budget;
      for (int b = 0; b < LIGATE_N_BUCKETS; ++b) {
        const double c = std::ceil(t.starts_per_item[b] * f / p.G) * p.G;
        t.starts_per_item[b] = (int)std::min<double>(c, std::max(p.n_starts, p.G));
      }
    }
  }

  // work queue: (ligand, start chunk) items, most expensive first
  const int n = pl->n_ligands;
  std::vector<Item> items;
  std::vector<int> lig_items(n), lig_slot0(n);
  std::vector<double> cost;
  double poses = 0, aev = 0, pev = 0;
  for (int r = 0; r < n; ++r) {
    const int i = sel ? sel[r] : r;
    double a, q;
    start_work(B->d, i, p.S, a, q);
    aev += a * p.n_starts;
    pev += q * p.n_starts;
    poses += (double)p.n_starts * (1.0 + (double)B->d.h_lig[i].n_rot * (p.S - 1));
    const int chunk = t.starts_per_item[bucket_of(B->d.h_lig[i])];
    lig_slot0[r] = (int)items.size();
    int c = 0;
    for (int s0 = 0; s0 < p.n_starts; s0 += chunk, ++c) {
      Item it;
      memset(&it, 0, sizeof(it));
      it.ligand = i;
      it.row = r;
      it.s0 = s0;
      it.s1 = std::min(p.n_starts, s0 + chunk);
      it.slot = (int)items.size();
      items.push_back(it);
      cost.push_back((a + 0.35 * q + 40.0) * (it.s1 - it.s0));
    }
    lig_items[r] = c;
  }
  pl->work.poses = poses;
  pl->work.atom_evals = aev;
  pl->work.pair_evals = pev;
  pl->work.starts = (double)n * p.n_starts;
  // descending cost (in single precision), ties in list order: an LSD radix
  // sort of the complemented bit patterns (non-negative floats order like
  // their bit patterns), 8 bits per pass, passes whose byte is the same for
  // every item skipped
  std::vector<uint32_t> key(items.size()), key2(items.size());
  std::vector<uint32_t> order(items.size()), order2(items.size());
  for (size_t i = 0; i < items.size(); ++i) {
    const float c = (float)cost[i];
    uint32_t bits;
    memcpy(&bits, &c, 4);
    key[i] = ~bits;
    order[i] = (uint32_t)i;
  }
  for (int sh = 0; sh < 32; sh += 8) {
    size_t cnt[257] = {0};
    for (size_t i = 0; i < key.size(); ++i) ++cnt[((key[i] >> sh) & 255u) + 1];
    if (std::any_of(cnt + 1, cnt + 257, [&](size_t c) { return c == key.size(); })) continue;
    for (int dg = 0; dg < 256; ++dg) cnt[dg + 1] += cnt[dg];
    for (size_t i = 0; i < key.size(); ++i) {
      const size_t q = cnt[(key[i] >> sh) & 255u]++;
      key2[q] = key[i];
      order2[q] = order[i];
    }
    key.swap(key2);
    order.swap(order2);
  }
  std::vector<Item> sorted(items.size());
  for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
  const size_t ni = items.size();
  cudaError_t e;
  pl->counter_bytes = sizeof(int) * (2 * (size_t)n + 1);  // queue, done[n], lig_thr[n]
  if ((e = dmalloc(&pl->stats, N_STATS)) != cudaSuccess) {
    free_plan(pl);
    return cuda_fail(e, "plan allocation");
  }
  if ((e = dmalloc(&pl->items, ni)) != cudaSuccess || (e = dmalloc(&pl->lig_items, n)) != cudaSuccess ||
      (e = dmalloc(&pl->lig_slot0, n)) != cudaSuccess ||
      (e = dmalloc(&pl->counters, 2 * (size_t)n + 1)) != cudaSuccess ||
      (e = dmalloc(&pl->partial, ni * p.K)) != cudaSuccess ||
      (e = dmalloc(&pl->out, (size_t)n * p.K)) != cudaSuccess) {
    free_plan(pl);
    return cuda_fail(e, "plan allocation");
  }
  if ((ni && (e = cudaMemcpy(pl->items, sorted.data(), sizeof(Item) * ni, cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (n && (e = cudaMemcpy(pl->lig_items, lig_items.data(), 4 * (size_t)n, cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (n && (e = cudaMemcpy(pl->lig_slot0, lig_slot0.data(), 4 * (size_t)n, cudaMemcpyHostToDevice)) != cudaSuccess)) {
    free_plan(pl);
    return cuda_fail(e, "plan upload");
  }
  {  // per resident warp: the clash tables of the pairs a single earlier bond separates
    int m1 = 0;
    for (int r = 0; r < n; ++r) {
      const LigDesc &ld = B->d.h_lig[sel ? sel[r] : r];
      m1 = std::max(m1, dock_memo1_tables(ld, B->d.h_bonds.data() + ld.bond_base, p.S));
    }
    if (m1 > 0) {
      const size_t floats = (size_t)pl->grid * t.warps_per_cta * m1 * p.S * p.S;
      if ((e = dmalloc(&p.memo1, floats)) != cudaSuccess) { free_plan(pl); return cuda_fail(e, "plan allocation"); }
      p.m1max = m1;
    }
  }
  p.items = pl->items;
  p.n_items = (int)ni;
  p.lig_items = pl->lig_items;
  p.lig_slot0 = pl->lig_slot0;
  p.queue = pl->counters;
  p.done = pl->counters + 1;
  p.lig_thr = reinterpret_cast<unsigned *>(pl->counters + 1 + n);
  p.stats = pl->stats;
  p.partial = pl->partial;
  p.out = pl->out;
  p.n_items_dev = nullptr;
  pl->rows = n;
  pl->cur_row_lig = pl->row_lig;
  if (!(opt && opt->no_device_sync) && (e = cudaDeviceSynchronize()) != cudaSuccess) {
    free_plan(pl);
    return cuda_fail(e, "plan setup");
  }
  *out = pl;
  return LIGATE_OK;
}

extern "C" ligate_status ligate_plan_create(const ligate_pocket *P, const ligate_batch *B,
                                            const ligate_sampling *s, const ligate_tile *tile,
                                            ligate_plan **out) {
  return plan_create_impl(P, B, s, tile, nullptr, 0, out);
}

extern "C" ligate_status ligate_plan_create_subset(const ligate_pocket *P, const ligate_batch *B,
                                                   const ligate_sampling *s, const ligate_tile *tile,
                                                   const int32_t *ligands, int n_ligands,
                                                   ligate_plan **out) {
  if (!ligands && n_ligands > 0) { set_error("plan_create_subset: ligands is NULL"); return LIGATE_ERR_INVALID; }
  static const int32_t none = 0;
  return plan_create_impl(P, B, s, tile, ligands ? ligands : &none, n_ligands, out);
}

// Capture reset + docking kernel into a graph (once per plan).
static ligate_status plan_capture(ligate_plan *pl) {
  if (pl->exec) return LIGATE_OK;
  CK(cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking), "capture stream");
  CK(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t e = cudaMemsetAsync(pl->counters, 0, pl->counter_bytes, pl->cap_stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->stats, 0, N_STATS * sizeof(unsigned long long), pl->cap_stream);
  if (e == cudaSuccess && pl->p.n_items > 0)
    e = launch_dock(pl->mode, pl->tile.reg_cap, pl->p, pl->grid, pl->block, pl->smem, pl->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(pl->cap_stream, &g);
  if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(e, "capture docking run"); }
  if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
  pl->graph = g;
  CK(cudaGraphInstantiate(&pl->exec, g, 0), "graph instantiate");
  return LIGATE_OK;
}

static bool is_host_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return true; }
  return a.type == cudaMemoryTypeUnregistered || a.type == cudaMemoryTypeHost;
}

extern "C" ligate_status ligate_plan_run(ligate_plan *pl, ligate_pose *out, void *stream) {
  NvtxRange nvtx_("ligate:plan_run");
  if (!pl) { set_error("plan_run: NULL plan"); return LIGATE_ERR_INVALID; }
  ligate_status st = plan_capture(pl);
  if (st != LIGATE_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaGraphLaunch(pl->exec, s), "graph launch");
  pl->rows = pl->n_ligands;
  pl->cur_row_lig = pl->row_lig;
  if (out) {
    const size_t bytes = sizeof(PoseOut) * (size_t)pl->n_ligands * pl->p.K;
    if (bytes) CK(cudaMemcpyAsync(out, pl->out, bytes, cudaMemcpyDefault, s), "result copy");
    if (is_host_ptr(out)) CK(cudaStreamSynchronize(s), "stream synchronize");
  }
  return LIGATE_OK;
}

// ---------------------------------------------------------------------------
// Subset runs on the device: the selected ligands' work items are built on
// the GPU, in the plan's descending per-start cost order and with chunk
// sizes from the work model for the selection's size, so a selection
// produced on the GPU (a triage ranking) is docked without a round trip to
// the host.
__global__ void subset_rows_kernel(const int32_t *__restrict__ ligands, int n_sel, int n_batch,
                                   int32_t *__restrict__ rowmap) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_sel) return;
  const int l = ligands[r];
  if (l >= 0 && l < n_batch) rowmap[l] = r;  // a repeated ligand keeps one of its rows
}

// Rows whose index is out of range or repeated (rowmap holds another row
// for it) get no items: their output is written empty here.  sub_row_lig is
// the batch index of each row for the post-docking stages.
__global__ void subset_meta_kernel(const int32_t *__restrict__ ligands, int n_sel, int n_batch,
                                   const int32_t *__restrict__ rowmap, int32_t *__restrict__ sub_row_lig,
                                   PoseOut *__restrict__ out, int K) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_sel) return;
  const int l = ligands[r];
  const bool ok = l >= 0 && l < n_batch && rowmap[l] == r;
  sub_row_lig[r] = ok ? l : 0;
  if (!ok)
    for (int k = 0; k < K; ++k) {
      PoseOut o;
      o.score = __int_as_float(0x7f800000);
      o.start_id = -1;
      o.tors[0] = o.tors[1] = o.tors[2] = o.tors[3] = 0;
      out[(size_t)r * K + k] = o;
    }
}

struct SubsetChunks {
  int c[LIGATE_N_BUCKETS];  // starts per work item of each size bucket
};

// Work items of the selected ligands (rowmap[l] >= 0), built by one CTA in
// the plan's descending per-start cost order: a ligand's items are its
// starts in chunks of its bucket's size, consecutive, with slots equal to
// their positions; the block scan gives each selected ligand its first slot.
__global__ void __launch_bounds__(1024) subset_build_kernel(const int32_t *__restrict__ lig_by_cost, int n,
                                                            const int32_t *__restrict__ rowmap,
                                                            const uint8_t *__restrict__ lig_bucket,
                                                            const SubsetChunks ch, int n_starts,
                                                            Item *__restrict__ items, int *__restrict__ lig_items,
                                                            int *__restrict__ lig_slot0, int *__restrict__ count) {
  __shared__ int wsum[32];
  __shared__ int base, chunk_total;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += blockDim.x) {
    const int i = c0 + threadIdx.x;
    const int l = i < n ? lig_by_cost[i] : -1;
    const int row = l >= 0 ? rowmap[l] : -1;
    int chunk = 1, c = 0;
    if (row >= 0) {
      chunk = ch.c[lig_bucket[l]];
      c = (n_starts + chunk - 1) / chunk;
    }
    int incl = c;  // inclusive scan of the item counts within the warp
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {  // exclusive prefix of the warp totals, and the chunk's total
      const int v = lane < nw ? wsum[lane] : 0;
      int w_incl = v;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, w_incl, o);
        if (lane >= o) w_incl += t;
      }
      if (lane < nw) wsum[lane] = w_incl - v;
      if (lane == 31) chunk_total = w_incl;
    }
    __syncthreads();
    if (row >= 0) {
      const int off = base + wsum[wid] + incl - c;
      lig_items[row] = c;
      lig_slot0[row] = off;
      for (int q = 0; q < c; ++q) {
        Item it;
        it.ligand = l;
        it.row = row;
        it.s0 = q * chunk;
        it.s1 = min(n_starts, (q + 1) * chunk);
        it.slot = off + q;
        it.pad[0] = it.pad[1] = it.pad[2] = 0;
        items[off + q] = it;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) base += chunk_total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base;
}

extern "C" ligate_status ligate_plan_run_subset(ligate_plan *pl, const int32_t *ligands, int n_sel,
                                                ligate_pose *out, void *stream) {
  NvtxRange nvtx_("ligate:plan_run_subset");
  if (!pl) { set_error("plan_run_subset: NULL plan"); return LIGATE_ERR_INVALID; }
  if (pl->is_subset) {
    set_error("plan_run_subset: the plan was created over a subset; create it over the whole batch");
    return LIGATE_ERR_INVALID;
  }
  if (n_sel < 0 || n_sel > pl->n_ligands || (n_sel > 0 && !ligands)) {
    set_error("plan_run_subset: need 0 <= n_sel <= %d ligands and a device index array", pl->n_ligands);
    return LIGATE_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int n = pl->n_ligands;
  const DockParams &p = pl->p;
  const BatchDev &B = pl->batch->d;
  cudaError_t e;
  if (!pl->lig_by_cost) {  // once: cost order, buckets and the work model of the whole batch
    std::vector<double> cost(n);
    std::vector<int32_t> order(n);
    std::vector<uint8_t> bucket(n);
    double nb[LIGATE_N_BUCKETS] = {0};
    for (int i = 0; i < n; ++i) {
      double a, q;
      start_work(B, i, p.S, a, q);
      cost[i] = a + 0.35 * q + 40.0;
      bucket[i] = (uint8_t)bucket_of(B.h_lig[i]);
      pl->model_W += cost[i] * p.n_starts;
      pl->model_cb[bucket[i]] += cost[i];
      nb[bucket[i]] += 1.0;
      order[i] = i;
    }
    for (int b = 0; b < LIGATE_N_BUCKETS; ++b) pl->model_cb[b] = nb[b] > 0 ? pl->model_cb[b] / nb[b] : 0.0;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    if ((e = dmalloc(&pl->lig_by_cost, n)) != cudaSuccess || (e = dmalloc(&pl->lig_bucket, n)) != cudaSuccess ||
        (e = dmalloc(&pl->sub_count, 1)) != cudaSuccess || (e = dmalloc(&pl->sub_lig_items, n)) != cudaSuccess ||
        (e = dmalloc(&pl->sub_slot0, n)) != cudaSuccess || (e = dmalloc(&pl->rowmap, n)) != cudaSuccess ||
        (e = dmalloc(&pl->sub_row_lig, n)) != cudaSuccess ||
        (n && (e = cudaMemcpy(pl->lig_by_cost, order.data(), 4 * (size_t)n, cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (n && (e = cudaMemcpy(pl->lig_bucket, bucket.data(), (size_t)n, cudaMemcpyHostToDevice)) != cudaSuccess))
      return cuda_fail(e, "plan_run_subset: set-up");
  }
  // chunks from the work model for a selection of n_sel average ligands
  SubsetChunks ch;
  int cmin = 2048;
  const double P_warps = std::max(1.0, (double)pl->grid * pl->tile.warps_per_cta);
  for (int b = 0; b < LIGATE_N_BUCKETS; ++b) {
    double chunk = 512.0;
    if (pl->model_cb[b] > 0) chunk = pl->model_W * ((double)n_sel / std::max(n, 1)) / (8.0 * P_warps * pl->model_cb[b]);
    chunk = std::min(2048.0, std::max(128.0, chunk));
    ch.c[b] = std::max(p.G, (int)chunk / p.G * p.G);
    cmin = std::min(cmin, ch.c[b]);
  }
  const size_t need = (size_t)n_sel * (size_t)((p.n_starts + cmin - 1) / cmin);
  if (need > pl->sub_cap) {  // grows only
    cudaFree(pl->sub_items);
    cudaFree(pl->sub_partial);
    pl->sub_items = nullptr;
    pl->sub_partial = nullptr;
    pl->sub_cap = 0;
    if ((e = dmalloc(&pl->sub_items, need)) != cudaSuccess || (e = dmalloc(&pl->sub_partial, need * p.K)) != cudaSuccess)
      return cuda_fail(e, "plan_run_subset: allocation");
    pl->sub_cap = need;
  }
  pl->rows = n_sel;
  pl->cur_row_lig = pl->sub_row_lig;
  if (n_sel > 0) {
    if ((e = cudaMemsetAsync(pl->rowmap, 0xff, sizeof(int32_t) * (size_t)n, s)) != cudaSuccess)
      return cuda_fail(e, "plan_run_subset");
    const int blocks = (n_sel + 255) / 256;
    subset_rows_kernel<<<blocks, 256, 0, s>>>(ligands, n_sel, B.n_ligands, pl->rowmap);
    subset_build_kernel<<<1, 1024, 0, s>>>(pl->lig_by_cost, n, pl->rowmap, pl->lig_bucket, ch, p.n_starts,
                                           pl->sub_items, pl->sub_lig_items, pl->sub_slot0, pl->sub_count);
    subset_meta_kernel<<<blocks, 256, 0, s>>>(ligands, n_sel, B.n_ligands, pl->rowmap, pl->sub_row_lig, pl->out,
                                              p.K);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "plan_run_subset: selection");
    if ((e = cudaMemsetAsync(pl->counters, 0, sizeof(int) * ((size_t)n_sel + 1), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(pl->counters + 1 + n, 0, sizeof(int) * (size_t)n_sel, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(pl->stats, 0, N_STATS * sizeof(unsigned long long), s)) != cudaSuccess)
      return cuda_fail(e, "plan_run_subset");
    DockParams q = p;
    q.items = pl->sub_items;
    q.n_items = 0;
    q.n_items_dev = pl->sub_count;
    q.lig_items = pl->sub_lig_items;
    q.lig_slot0 = pl->sub_slot0;
    q.partial = pl->sub_partial;
    if ((e = launch_dock(pl->mode, pl->tile.reg_cap, q, pl->grid, pl->block, pl->smem, s)) != cudaSuccess)
      return cuda_fail(e, "plan_run_subset: docking kernel");
  }
  if (out && n_sel > 0) {
    const size_t bytes = sizeof(PoseOut) * (size_t)n_sel * p.K;
    CK(cudaMemcpyAsync(out, pl->out, bytes, cudaMemcpyDefault, s), "result copy");
    if (is_host_ptr(out)) CK(cudaStreamSynchronize(s), "stream synchronize");
  }
  return LIGATE_OK;
}

extern "C" ligate_status ligate_plan_output(const ligate_plan *pl, const ligate_pose **ptr) {
  if (!pl || !ptr) { set_error("plan_output: NULL argument"); return LIGATE_ERR_INVALID; }
  *ptr = reinterpret_cast<const ligate_pose *>(pl->out);
  return LIGATE_OK;
}

extern "C" ligate_status ligate_plan_get_tile(const ligate_plan *pl, ligate_tile *t, int *launches) {
  if (!pl) { set_error("plan_get_tile: NULL plan"); return LIGATE_ERR_INVALID; }
  if (t) *t = pl->tile;
  if (launches) *launches = pl->p.n_items > 0 ? 1 : 0;
  return LIGATE_OK;
}

extern "C" ligate_status ligate_plan_work(const ligate_plan *pl, ligate_work *w) {
  if (!pl || !w) { set_error("plan_work: NULL argument"); return LIGATE_ERR_INVALID; }
  *w = pl->work;
  unsigned long long c[N_STATS] = {};
  if (pl->exec) {
    cudaError_t e = cudaMemcpy(c, pl->stats, sizeof(c), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "plan_work");
  }
  w->done_atom_evals = (double)c[0];
  w->done_pair_tests = (double)c[1];
  w->done_pair_survivors = (double)c[2];
  w->done_pair_evals = (double)c[3] * pl->p.S;
  w->done_pruned_starts = (double)c[4];
  w->done_bond_sweeps = (double)c[5];
  return LIGATE_OK;
}

extern "C" void ligate_plan_destroy(ligate_plan *pl) { free_plan(pl); }

// One docking run of a plan, launched directly on `st` (no graph).
static cudaError_t plan_launch(ligate_plan *pl, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(pl->counters, 0, pl->counter_bytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->stats, 0, N_STATS * sizeof(unsigned long long), st);
  if (e == cudaSuccess && pl->p.n_items > 0)
    e = launch_dock(pl->mode, pl->tile.reg_cap, pl->p, pl->grid, pl->block, pl->smem, st);
  pl->rows = pl->n_ligands;
  pl->cur_row_lig = pl->row_lig;
  return e;
}

extern "C" ligate_status ligate_dock_batch(const ligate_pocket *P, const ligate_ligands *L,
                                           const ligate_sampling *s, ligate_pose *out,
                                           void *stream) {
  NvtxRange nvtx_("ligate:dock_batch");
  if (!L) { set_error("dock_batch: ligands is NULL"); return LIGATE_ERR_INVALID; }
  if (!out && L->n_ligands > 0) { set_error("dock_batch: out is NULL"); return LIGATE_ERR_INVALID; }
  const int n = L->n_ligands;
  if (n < 2048 || !L->atom_offset || !L->bond_offset) {  // one batch, one plan
    ligate_batch *B = nullptr;
    ligate_status st = ligate_batch_create(L, &B);
    if (st != LIGATE_OK) return st;
    ligate_plan *pl = nullptr;
    st = ligate_plan_create(P, B, s, nullptr, &pl);
    if (st == LIGATE_OK) {
      st = ligate_plan_run(pl, out, stream);
      if (st == LIGATE_OK) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) st = cuda_fail(e, "dock_batch");
      }
    }
    ligate_plan_destroy(pl);
    ligate_batch_destroy(B);
    return st;
  }
  // Two parts: the first 1/32 of the ligands is packed, planned and
  // launched, then the rest is packed, uploaded and planned on the host
  // while the first part docks (its kernel time about matches the rest's
  // host time; a larger first part only lengthens the exposed start), and
  // the second kernel fills the SMs as the first one's CTAs finish (two
  // library streams).  The same poses as one plan over all ligands.
  const int first = n / 32;
  const int32_t a0 = L->atom_offset[first], b0 = L->bond_offset[first];
  std::vector<int32_t> aoB(n - first + 1), boB(n - first + 1);
  for (int i = 0; i <= n - first; ++i) {
    aoB[i] = L->atom_offset[first + i] - a0;
    boB[i] = L->bond_offset[first + i] - b0;
  }
  const ligate_ligands part[2] = {
      {first, L->atom_offset, L->xyz, L->type, L->bond_offset, L->bonds, L->rotatable},
      {n - first, aoB.data(), L->xyz ? L->xyz + 3 * (size_t)a0 : nullptr, L->type ? L->type + a0 : nullptr,
       boB.data(), L->bonds ? L->bonds + 2 * (size_t)b0 : nullptr, L->rotatable ? L->rotatable + b0 : nullptr}};
  ligate_batch *B[2] = {nullptr, nullptr};
  ligate_plan *pl[2] = {nullptr, nullptr};
  cudaStream_t st[2] = {nullptr, nullptr};
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  ligate_status res = LIGATE_OK;
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < 2 && e == cudaSuccess; ++q) e = cudaStreamCreateWithFlags(&st[q], cudaStreamNonBlocking);
  for (int q = 0; q < 3 && e == cudaSuccess; ++q) e = cudaEventCreateWithFlags(&ev[q], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev[2], (cudaStream_t)stream);  // after the caller's prior work
  for (int q = 0; q < 2 && e == cudaSuccess; ++q) e = cudaStreamWaitEvent(st[q], ev[2], 0);
  if (e != cudaSuccess) res = cuda_fail(e, "dock_batch: streams");
  for (int q = 0; q < 2 && res == LIGATE_OK; ++q) {
    res = ligate_batch_create(&part[q], &B[q]);
    if (res != LIGATE_OK) {
      if (q == 1) {  // the message counts ligands from the start of the second part
        const std::string m = g_err;
        set_error("%s (ligand numbers counted from ligand %d of the input)", m.c_str(), first);
      }
      break;
    }
    PlanOpts opt;
    opt.no_device_sync = true;
    if (q == 1) {
      opt.rot = pl[0]->p.rot;
      opt.anc = pl[0]->p.anc;
    }
    res = plan_create_impl(P, B[q], s, nullptr, nullptr, 0, &pl[q], &opt);
    if (res != LIGATE_OK) break;
    // the set-up copies ran on the legacy default stream: order them first
    if ((e = cudaEventRecord(ev[q], 0)) != cudaSuccess || (e = cudaStreamWaitEvent(st[q], ev[q], 0)) != cudaSuccess ||
        (e = plan_launch(pl[q], st[q])) != cudaSuccess) {
      res = cuda_fail(e, "dock_batch: launch");
      break;
    }
  }
  for (int q = 0; q < 2 && res == LIGATE_OK; ++q) {
    const size_t bytes = sizeof(PoseOut) * (size_t)pl[q]->n_ligands * pl[q]->p.K;
    if ((e = cudaMemcpyAsync(out + (q ? (size_t)first * s->top_k : 0), pl[q]->out, bytes, cudaMemcpyDefault, st[q])) !=
        cudaSuccess)
      res = cuda_fail(e, "dock_batch: result copy");
  }
  for (int q = 0; q < 2; ++q)
    if (st[q]) {
      e = cudaStreamSynchronize(st[q]);
      if (e != cudaSuccess && res == LIGATE_OK) res = cuda_fail(e, "dock_batch");
    }
  for (int q = 1; q >= 0; --q) {  // plan 1 borrows plan 0's frames
    ligate_plan_destroy(pl[q]);
    ligate_batch_destroy(B[q]);
  }
  for (int q = 0; q < 3; ++q)
    if (ev[q]) cudaEventDestroy(ev[q]);
  for (int q = 0; q < 2; ++q)
    if (st[q]) cudaStreamDestroy(st[q]);
  return res;
}

extern "C" ligate_status ligate_score_poses(const ligate_pocket *P, const ligate_batch *B,
                                            const ligate_sampling *s, int n_poses,
                                            const int32_t *lig_idx, const int32_t *start_id,
                                            const uint8_t *tors, float *out, void *stream) {
  int mode = 0;
  ligate_status st = check_sampling(P, B, s, &mode);
  if (st != LIGATE_OK) return st;
  if (n_poses < 0 || (n_poses > 0 && (!lig_idx || !start_id || !tors || !out))) {
    set_error("score_poses: bad pose arrays");
    return LIGATE_ERR_INVALID;
  }
  if (n_poses == 0) return LIGATE_OK;
  DockParams p;
  float *rot = nullptr, *anc = nullptr, *quat = nullptr;
  st = base_params(P, B, s, mode, p, &rot, &anc, &quat);
  cudaError_t e = cudaSuccess;
  if (st == LIGATE_OK) {
    e = launch_score_poses(mode, p, n_poses, lig_idx, start_id, tors, out, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  }
  cudaFree(rot); cudaFree(anc); cudaFree(quat);
  if (st != LIGATE_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "score_poses");
  return LIGATE_OK;
}

extern "C" ligate_status ligate_pose_coords(const ligate_pocket *P, const ligate_batch *B,
                                            const ligate_sampling *s, int n_poses, const int32_t *lig_idx,
                                            const int32_t *start_id, const uint8_t *tors, float *out,
                                            void *stream) {
  int mode = 0;
  ligate_status st = check_sampling(P, B, s, &mode);
  if (st != LIGATE_OK) return st;
  if (n_poses < 0 || (n_poses > 0 && (!lig_idx || !start_id || !tors || !out))) {
    set_error("pose_coords: bad pose arrays");
    return LIGATE_ERR_INVALID;
  }
  if (n_poses == 0) return LIGATE_OK;
  DockParams p;
  float *rot = nullptr, *anc = nullptr, *quat = nullptr;
  st = base_params(P, B, s, mode, p, &rot, &anc, &quat);
  cudaError_t e = cudaSuccess;
  if (st == LIGATE_OK) {
    e = launch_pose_coords(p, B->d.order, n_poses, lig_idx, start_id, tors, out, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  }
  cudaFree(rot); cudaFree(anc); cudaFree(quat);
  if (st != LIGATE_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "pose_coords");
  return LIGATE_OK;
}

extern "C" ligate_status ligate_state_coords(const ligate_pocket *P, const ligate_batch *B,
                                             const ligate_sampling *s, int n, const int32_t *lig_idx,
                                             const ligate_pose_state *states, float *out, void *stream) {
  int mode = 0;
  ligate_status st = check_sampling(P, B, s, &mode);
  if (st != LIGATE_OK) return st;
  if (n < 0 || (n > 0 && (!lig_idx || !states || !out))) {
    set_error("state_coords: bad state arrays");
    return LIGATE_ERR_INVALID;
  }
  if (n == 0) return LIGATE_OK;
  DockParams p;
  float *rot = nullptr, *anc = nullptr, *quat = nullptr;
  st = base_params(P, B, s, mode, p, &rot, &anc, &quat);
  cudaError_t e = cudaSuccess;
  if (st == LIGATE_OK) {
    e = launch_state_coords(p, B->d.order, n, lig_idx, states, out, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  }
  cudaFree(rot); cudaFree(anc); cudaFree(quat);
  if (st != LIGATE_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "state_coords");
  return LIGATE_OK;
}

__global__ void best_scores_kernel(const PoseOut *__restrict__ poses, int n, int K, float *__restrict__ out,
                                   int stride, int column) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) out[(size_t)r * stride + column] = poses[(size_t)r * K].score;
}

extern "C" ligate_status ligate_plan_best_scores(const ligate_plan *pl, float *out, int stride, int column,
                                                 void *stream) {
  if (!pl || !out || stride < 1 || column < 0 || column >= stride) {
    set_error("plan_best_scores: bad arguments");
    return LIGATE_ERR_INVALID;
  }
  const int n = pl->rows;
  if (n == 0) return LIGATE_OK;
  best_scores_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(pl->out, n, pl->p.K, out, stride, column);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "plan_best_scores");
  return LIGATE_OK;
}

__global__ void pick_value_kernel(const float *__restrict__ v, const int32_t *__restrict__ idx, int k,
                                  float *__restrict__ out) {
  if (threadIdx.x == 0) *out = v[idx[k - 1]];
}

extern "C" ligate_status ligate_plan_best_quantile(ligate_plan *pl, double frac, float *out, void *stream) {
  if (!pl || !out || !(frac > 0.0) || frac > 1.0) {
    set_error("plan_best_quantile: need a plan, an output and 0 < frac <= 1");
    return LIGATE_ERR_INVALID;
  }
  const int n = pl->rows;
  if (n == 0) { set_error("plan_best_quantile: the plan has no rows"); return LIGATE_ERR_INVALID; }
  const int k = std::min(n, std::max(1, (int)std::ceil(frac * n - 1e-9)));
  int n2 = 2048;
  while (n2 < n) n2 <<= 1;
  cudaError_t e = cudaSuccess;
  if (pl->q_cap < n2) {  // grown once per size (allocates: not inside a capture)
    cudaFree(pl->q_scores); cudaFree(pl->q_keys); cudaFree(pl->q_idx);
    pl->q_scores = nullptr; pl->q_keys = nullptr; pl->q_idx = nullptr; pl->q_cap = 0;
    if ((e = dmalloc(&pl->q_scores, n2)) != cudaSuccess || (e = dmalloc(&pl->q_keys, n2)) != cudaSuccess ||
        (e = dmalloc(&pl->q_idx, n2)) != cudaSuccess)
      return cuda_fail(e, "plan_best_quantile");
    pl->q_cap = n2;
  }
  cudaStream_t st = (cudaStream_t)stream;
  best_scores_kernel<<<(n + 255) / 256, 256, 0, st>>>(pl->out, n, pl->p.K, pl->q_scores, 1, 0);
  if ((e = cudaGetLastError()) == cudaSuccess) e = mlp::sort_select(pl->q_scores, n, k, pl->q_keys, n2, pl->q_idx, st);
  if (e == cudaSuccess) {
    pick_value_kernel<<<1, 32, 0, st>>>(pl->q_scores, pl->q_idx, k, out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(e, "plan_best_quantile");
  return LIGATE_OK;
}

extern "C" ligate_status ligate_plan_set_cutoff(ligate_plan *pl, const float *cutoff) {
  if (!pl) { set_error("plan_set_cutoff: NULL plan"); return LIGATE_ERR_INVALID; }
  if (pl->p.cut == cutoff) return LIGATE_OK;
  // the captured run holds the parameters it was captured with: capture it
  // again at the next run, once no launch of it is in flight
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "plan_set_cutoff");
  if (pl->exec) { cudaGraphExecDestroy(pl->exec); pl->exec = nullptr; }
  if (pl->graph) { cudaGraphDestroy(pl->graph); pl->graph = nullptr; }
  if (pl->cap_stream) { cudaStreamDestroy(pl->cap_stream); pl->cap_stream = nullptr; }
  pl->p.cut = cutoff;
  return LIGATE_OK;
}

// ===========================================================================
// Pose refinement (refine.cu).
static ligate_status refine_explicit(int mode, const ligate_pocket *P, const ligate_batch *B,
                                     const ligate_sampling *s, int n, const int32_t *lig_idx,
                                     const ligate_pose_state *states, int iters, float eta0,
                                     ligate_refined *out, float *energy, float *grad, void *stream,
                                     const char *what) {
  int m = 0;
  ligate_status st = check_sampling(P, B, s, &m);
  if (st != LIGATE_OK) return st;
  if (n < 0 || (n > 0 && (!lig_idx || !states || (mode == 0 ? (!energy || !grad) : !out)))) {
    set_error("%s: bad arrays", what);
    return LIGATE_ERR_INVALID;
  }
  if (mode == 1 && (iters < 0 || iters > LIGATE_REFINE_MAX_ITERS || !(eta0 > 0.f) || !std::isfinite(eta0))) {
    set_error("%s: iterations must be 0..%d and eta0 finite and > 0", what, LIGATE_REFINE_MAX_ITERS);
    return LIGATE_ERR_INVALID;
  }
  if (n == 0) return LIGATE_OK;
  DockParams p;
  float *rot = nullptr, *anc = nullptr, *quat = nullptr;
  st = base_params(P, B, s, m, p, &rot, &anc, &quat);
  cudaError_t e = cudaSuccess;
  if (st == LIGATE_OK && refine_smem_bytes(p.nmax) * 4 > 227 * 1024) {
    set_error("%s: ligands too large for the refinement kernel's shared memory", what);
    st = LIGATE_ERR_UNSUPPORTED;
  }
  if (st == LIGATE_OK) {
    e = launch_refine(mode, p, P->d.origin, P->d.spacing, n, lig_idx, states, nullptr, nullptr, iters,
                      eta0, out, energy, grad, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  }
  cudaFree(rot); cudaFree(anc); cudaFree(quat);
  if (st != LIGATE_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, what);
  return LIGATE_OK;
}

extern "C" ligate_status ligate_pose_gradient(const ligate_pocket *P, const ligate_batch *B,
                                              const ligate_sampling *s, int n, const int32_t *lig_idx,
                                              const ligate_pose_state *states, float *energy, float *grad,
                                              void *stream) {
  return refine_explicit(0, P, B, s, n, lig_idx, states, 0, 1.f, nullptr, energy, grad, stream,
                         "pose_gradient");
}

extern "C" ligate_status ligate_refine_states(const ligate_pocket *P, const ligate_batch *B,
                                              const ligate_sampling *s, int n, const int32_t *lig_idx,
                                              const ligate_pose_state *init, int iterations, float eta0,
                                              ligate_refined *out, void *stream) {
  return refine_explicit(1, P, B, s, n, lig_idx, init, iterations, eta0, out, nullptr, nullptr, stream,
                         "refine_states");
}

extern "C" ligate_status ligate_plan_refine(const ligate_plan *pl, int iterations, float eta0,
                                            ligate_refined *out, void *stream) {
  NvtxRange nvtx_("ligate:plan_refine");
  if (!pl || !out) { set_error("plan_refine: NULL argument"); return LIGATE_ERR_INVALID; }
  if (iterations < 0 || iterations > LIGATE_REFINE_MAX_ITERS || !(eta0 > 0.f) || !std::isfinite(eta0)) {
    set_error("plan_refine: iterations must be 0..%d and eta0 finite and > 0", LIGATE_REFINE_MAX_ITERS);
    return LIGATE_ERR_INVALID;
  }
  const int n = pl->rows * pl->p.K;
  if (n == 0) return LIGATE_OK;
  if (refine_smem_bytes(pl->p.nmax) * 4 > 227 * 1024) {
    set_error("plan_refine: ligands too large for the refinement kernel's shared memory");
    return LIGATE_ERR_UNSUPPORTED;
  }
  cudaError_t e = launch_refine(2, pl->p, pl->origin, pl->h, n, nullptr, nullptr,
                                reinterpret_cast<const ligate_pose *>(pl->out), pl->cur_row_lig, iterations,
                                eta0, out, nullptr, nullptr, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "plan_refine");
  return LIGATE_OK;
}

// ===========================================================================
// Exact rescoring (dock.cu).
static ligate_status rec_params(const ligate_pocket *P, const ligate_batch *B, RecParams &r, const char *what) {
  if (!P->d.rec_pair) { set_error("%s: the pocket has no receptor (ligate_pocket_set_receptor)", what); return LIGATE_ERR_INVALID; }
  if (B->max_type >= P->d.rec_types) {
    set_error("%s: ligand atom type %d beyond the receptor's %d types", what, B->max_type, P->d.rec_types);
    return LIGATE_ERR_INVALID;
  }
  r.rec = P->d.rec; r.pair = P->d.rec_pair; r.n_rec = P->d.n_rec; r.n_types = P->d.rec_types;
  r.cell = P->d.rec_cell;
  r.ncx = P->d.rec_nc[0]; r.ncy = P->d.rec_nc[1]; r.ncz = P->d.rec_nc[2];
  r.lox = P->d.rec_lo[0]; r.loy = P->d.rec_lo[1]; r.loz = P->d.rec_lo[2];
  r.icx = P->d.rec_inv[0]; r.icy = P->d.rec_inv[1]; r.icz = P->d.rec_inv[2];
  r.cut2 = P->d.rec_cut2; r.cap = P->d.rec_cap; r.rmin2 = P->d.rec_rmin2;
  r.ox = (float)P->d.origin[0]; r.oy = (float)P->d.origin[1]; r.oz = (float)P->d.origin[2];
  r.inv_h = (float)(1.0 / P->d.spacing);
  return LIGATE_OK;
}

extern "C" ligate_status ligate_rescore_poses(const ligate_pocket *P, const ligate_batch *B,
                                              const ligate_sampling *s, int n, const int32_t *lig_idx,
                                              const int32_t *start_id, const uint8_t *tors,
                                              ligate_rescored *out, void *stream) {
  int mode = 0;
  ligate_status st = check_sampling(P, B, s, &mode);
  if (st != LIGATE_OK) return st;
  if (n < 0 || (n > 0 && (!lig_idx || !start_id || !tors || !out))) {
    set_error("rescore_poses: bad pose arrays");
    return LIGATE_ERR_INVALID;
  }
  RecParams r;
  if ((st = rec_params(P, B, r, "rescore_poses")) != LIGATE_OK) return st;
  if (n == 0) return LIGATE_OK;
  DockParams p;
  float *rot = nullptr, *anc = nullptr, *quat = nullptr;
  st = base_params(P, B, s, mode, p, &rot, &anc, &quat);
  cudaError_t e = cudaSuccess;
  if (st == LIGATE_OK && rescore_smem_bytes(p, r, 1) > 227 * 1024) {
    set_error("rescore_poses: %d receptor atoms do not fit in shared memory", r.n_rec);
    st = LIGATE_ERR_UNSUPPORTED;
  }
  if (st == LIGATE_OK) {
    e = launch_rescore(p, r, n, lig_idx, start_id, tors, nullptr, nullptr, nullptr, out, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  }
  cudaFree(rot); cudaFree(anc); cudaFree(quat);
  if (st != LIGATE_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "rescore_poses");
  return LIGATE_OK;
}

extern "C" ligate_status ligate_plan_rescore(const ligate_plan *pl, ligate_rescored *out, void *stream) {
  NvtxRange nvtx_("ligate:plan_rescore");
  if (!pl || !out) { set_error("plan_rescore: NULL argument"); return LIGATE_ERR_INVALID; }
  RecParams r;
  ligate_status st = rec_params(pl->pocket, pl->batch, r, "plan_rescore");
  if (st != LIGATE_OK) return st;
  const int n = pl->rows * pl->p.K;
  if (n == 0) return LIGATE_OK;
  if (rescore_smem_bytes(pl->p, r, 1) > 227 * 1024) {
    set_error("plan_rescore: %d receptor atoms do not fit in shared memory", r.n_rec);
    return LIGATE_ERR_UNSUPPORTED;
  }
  cudaError_t e = launch_rescore(pl->p, r, n, nullptr, nullptr, nullptr,
                                 reinterpret_cast<const ligate_pose *>(pl->out), pl->cur_row_lig, nullptr, out,
                                 (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "plan_rescore");
  return LIGATE_OK;
}

extern "C" ligate_status ligate_rescore_states(const ligate_pocket *P, const ligate_batch *B,
                                               const ligate_sampling *s, int n, const int32_t *lig_idx,
                                               const ligate_pose_state *states, ligate_rescored *out,
                                               void *stream) {
  int mode = 0;
  ligate_status st = check_sampling(P, B, s, &mode);
  if (st != LIGATE_OK) return st;
  if (n < 0 || (n > 0 && (!lig_idx || !states || !out))) {
    set_error("rescore_states: bad arrays");
    return LIGATE_ERR_INVALID;
  }
  RecParams r;
  if ((st = rec_params(P, B, r, "rescore_states")) != LIGATE_OK) return st;
  if (n == 0) return LIGATE_OK;
  DockParams p;
  float *rot = nullptr, *anc = nullptr, *quat = nullptr;
  st = base_params(P, B, s, mode, p, &rot, &anc, &quat);
  cudaError_t e = cudaSuccess;
  if (st == LIGATE_OK && rescore_smem_bytes(p, r, 1) > 227 * 1024) {
    set_error("rescore_states: %d receptor atoms do not fit in shared memory", r.n_rec);
    st = LIGATE_ERR_UNSUPPORTED;
  }
  if (st == LIGATE_OK) {
    StateSrc ss;
    ss.base = reinterpret_cast<const unsigned char *>(states);
    ss.stride = (int)sizeof(ligate_pose_state);
    ss.lig_offset = 0;
    ss.score_offset = -1;
    ss.lig_idx = lig_idx;
    e = launch_rescore(p, r, n, nullptr, nullptr, nullptr, nullptr, nullptr, &ss, out, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  }
  cudaFree(rot); cudaFree(anc); cudaFree(quat);
  if (st != LIGATE_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "rescore_states");
  return LIGATE_OK;
}

extern "C" ligate_status ligate_plan_rescore_refined(const ligate_plan *pl, const ligate_refined *refined,
                                                     ligate_rescored *out, void *stream) {
  if (!pl || !refined || !out) { set_error("plan_rescore_refined: NULL argument"); return LIGATE_ERR_INVALID; }
  RecParams r;
  ligate_status st = rec_params(pl->pocket, pl->batch, r, "plan_rescore_refined");
  if (st != LIGATE_OK) return st;
  const int n = pl->rows * pl->p.K;
  if (n == 0) return LIGATE_OK;
  if (rescore_smem_bytes(pl->p, r, 1) > 227 * 1024) {
    set_error("plan_rescore_refined: %d receptor atoms do not fit in shared memory", r.n_rec);
    return LIGATE_ERR_UNSUPPORTED;
  }
  StateSrc ss;
  ss.base = reinterpret_cast<const unsigned char *>(refined);
  ss.stride = (int)sizeof(ligate_refined);
  ss.lig_offset = (int)offsetof(ligate_refined, ligand);
  ss.score_offset = (int)offsetof(ligate_refined, score_in);
  ss.lig_idx = nullptr;
  cudaError_t e = launch_rescore(pl->p, r, n, nullptr, nullptr, nullptr, nullptr, nullptr, &ss, out,
                                 (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "plan_rescore_refined");
  return LIGATE_OK;
}

extern "C" ligate_status ligate_pose_features(const ligate_pocket *P, const ligate_batch *B,
                                              const ligate_sampling *s, int n, const int32_t *lig_idx,
                                              const int32_t *start_id, const uint8_t *tors, float *out,
                                              void *stream) {
  int mode = 0;
  ligate_status st = check_sampling(P, B, s, &mode);
  if (st != LIGATE_OK) return st;
  if (n < 0 || (n > 0 && (!lig_idx || !start_id || !tors || !out))) {
    set_error("pose_features: bad pose arrays");
    return LIGATE_ERR_INVALID;
  }
  if (n == 0) return LIGATE_OK;
  DockParams p;
  float *rot = nullptr, *anc = nullptr, *quat = nullptr;
  st = base_params(P, B, s, mode, p, &rot, &anc, &quat);
  cudaError_t e = cudaSuccess;
  if (st == LIGATE_OK) {
    e = launch_pose_features(p, n, lig_idx, start_id, tors, nullptr, nullptr, out, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  }
  cudaFree(rot); cudaFree(anc); cudaFree(quat);
  if (st != LIGATE_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "pose_features");
  return LIGATE_OK;
}

extern "C" ligate_status ligate_plan_pose_features(const ligate_plan *pl, float *out, void *stream) {
  NvtxRange nvtx_("ligate:plan_pose_features");
  if (!pl || !out) { set_error("plan_pose_features: NULL argument"); return LIGATE_ERR_INVALID; }
  const int n = pl->rows * pl->p.K;
  if (n == 0) return LIGATE_OK;
  cudaError_t e = launch_pose_features(pl->p, n, nullptr, nullptr, nullptr,
                                       reinterpret_cast<const ligate_pose *>(pl->out), pl->cur_row_lig, out,
                                       (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "plan_pose_features");
  return LIGATE_OK;
}

extern "C" ligate_status ligate_plan_best_passing(const ligate_plan *pl, const ligate_rescored *rescored,
                                                  int32_t *idx_out, float *energy_out, void *stream) {
  if (!pl || ((!rescored || !idx_out) && pl->rows > 0)) {
    set_error("plan_best_passing: NULL argument");
    return LIGATE_ERR_INVALID;
  }
  cudaError_t e = launch_best_passing(rescored, pl->rows, pl->p.K, idx_out, energy_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "plan_best_passing");
  return LIGATE_OK;
}

extern "C" ligate_status ligate_select_poses(const float *pred, const ligate_pose *poses, int n, int k,
                                             float pass_below, int32_t *idx_out, void *stream) {
  if (n < 0 || k < 1 || (n > 0 && (!pred || !poses || !idx_out)) || !isfinite(pass_below)) {
    set_error("select_poses: bad arguments");
    return LIGATE_ERR_INVALID;
  }
  cudaError_t e = launch_select_poses(pred, poses, n, k, pass_below, idx_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "select_poses");
  return LIGATE_OK;
}

extern "C" ligate_status ligate_selector_labels(const ligate_rescored *rescored, int64_t n, float fail_label,
                                                float *out, void *stream) {
  if (n < 0 || (n > 0 && (!rescored || !out)) || !isfinite(fail_label)) {
    set_error("selector_labels: bad arguments");
    return LIGATE_ERR_INVALID;
  }
  cudaError_t e = launch_selector_labels(rescored, (long long)n, fail_label, out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "selector_labels");
  return LIGATE_OK;
}

// ===========================================================================
// Autotuner: times the CTA shapes and register caps on a sample of the
// batch; chunk sizes per size bucket come from the work model when a plan is
// created.  Results are cached per (device, S, mode) in LIGATE_TUNE_CACHE.
static std::string tune_key(int S, int mode) {
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  std::ostringstream k;
  k << prop.name << "|sm" << prop.major << prop.minor << "|S" << S << "|mode" << mode;
  std::string s = k.str();
  for (auto &c : s) if (c == ' ') c = '_';
  return s;
}

static bool read_tune_cache(int S, int mode, ligate_tile *t) {
  const char *path = getenv("LIGATE_TUNE_CACHE");
  if (!path || !*path) return false;
  std::ifstream f(path);
  if (!f) return false;
  const std::string key = tune_key(S, mode);
  std::string line;
  while (std::getline(f, line)) {
    std::istringstream is(line);
    std::string k;
    is >> k;
    if (k != key) continue;
    ligate_tile r;
    memset(&r, 0, sizeof(r));
    is >> r.warps_per_cta >> r.ctas_per_sm;
    for (int b = 0; b < LIGATE_N_BUCKETS; ++b) is >> r.starts_per_item[b];
    is >> r.reg_cap;
    if (!is) return false;
    *t = r;
    return true;
  }
  return false;
}

static void write_tune_cache(int S, int mode, const ligate_tile &t) {
  const char *path = getenv("LIGATE_TUNE_CACHE");
  if (!path || !*path) return;
  const std::string key = tune_key(S, mode);
  std::vector<std::string> keep;
  {
    std::ifstream f(path);
    std::string line;
    while (f && std::getline(f, line)) {
      std::istringstream is(line);
      std::string k;
      is >> k;
      if (k != key && !line.empty()) keep.push_back(line);
    }
  }
  std::ofstream f(path, std::ios::trunc);
  for (auto &l : keep) f << l << "\n";
  f << key << " " << t.warps_per_cta << " " << t.ctas_per_sm;
  for (int b = 0; b < LIGATE_N_BUCKETS; ++b) f << " " << t.starts_per_item[b];
  f << " " << t.reg_cap << "\n";
}

// Sub-batch of ligands `idx` (host re-packing from the packed batch).
static ligate_status sub_batch(const ligate_batch *B, const std::vector<int> &idx, ligate_batch **out) {
  *out = nullptr;
  ligate_batch *S = new ligate_batch();
  BatchDev &d = S->d;
  const BatchDev &src = B->d;
  d.n_ligands = (int)idx.size();
  std::vector<float4> atoms;
  std::vector<float4> all_atoms(src.total_atoms);
  if (src.total_atoms &&
      cudaMemcpy(all_atoms.data(), src.atoms, sizeof(float4) * src.total_atoms, cudaMemcpyDeviceToHost) != cudaSuccess) {
    delete S;
    return cuda_fail(cudaGetLastError(), "autotune sample");
  }
  for (int i : idx) {
    LigDesc ld = src.h_lig[i];
    const LigDesc o = ld;
    ld.atom_base = (int)atoms.size();
    ld.bond_base = (int)d.h_bonds.size();
    ld.elig_base = (int)d.h_elig.size();
    ld.cand_base = (long long)d.h_cand.size();
    long long nc = 0;
    for (int b = 0; b < o.n_rot; ++b) {
      const BondRec &r = src.h_bonds[o.bond_base + b];
      nc = std::max(nc, (long long)r.cand_off + r.n_cand);
    }
    for (long long c = 0; c < nc; ++c) d.h_cand.push_back(src.h_cand[o.cand_base + c]);
    for (int a = 0; a < o.n_atoms; ++a) {
      atoms.push_back(all_atoms[o.atom_base + a]);
      d.h_types.push_back(src.h_types[o.atom_base + a]);
      d.h_order.push_back(src.h_order[o.atom_base + a]);
    }
    for (int b = 0; b < o.n_rot; ++b) d.h_bonds.push_back(src.h_bonds[o.bond_base + b]);
    for (int w = 0; w < o.n_atoms * o.n_words; ++w) d.h_elig.push_back(src.h_elig[o.elig_base + w]);
    d.h_lig.push_back(ld);
    d.h_rot.push_back(o.n_rot);
    d.max_atoms = std::max(d.max_atoms, o.n_atoms);
    d.max_rot = std::max(d.max_rot, o.n_rot);
  }
  S->max_type = B->max_type;
  d.total_atoms = (int64_t)atoms.size();
  cudaError_t e;
  if ((e = dmalloc(&d.lig, d.h_lig.size())) != cudaSuccess ||
      (e = dmalloc(&d.atoms, atoms.size())) != cudaSuccess ||
      (e = dmalloc(&d.bonds, d.h_bonds.size())) != cudaSuccess ||
      (e = dmalloc(&d.elig, d.h_elig.size())) != cudaSuccess ||
      (e = dmalloc(&d.cand, d.h_cand.size())) != cudaSuccess ||
      (e = dmalloc(&d.order, d.h_order.size())) != cudaSuccess) {
    ligate_batch_destroy(S);
    return cuda_fail(e, "autotune sample");
  }
  if (!d.h_order.empty()) cudaMemcpy(d.order, d.h_order.data(), d.h_order.size(), cudaMemcpyHostToDevice);
  if (!d.h_cand.empty()) cudaMemcpy(d.cand, d.h_cand.data(), 2 * d.h_cand.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(d.lig, d.h_lig.data(), sizeof(LigDesc) * d.h_lig.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(d.atoms, atoms.data(), sizeof(float4) * atoms.size(), cudaMemcpyHostToDevice);
  if (!d.h_bonds.empty()) cudaMemcpy(d.bonds, d.h_bonds.data(), sizeof(BondRec) * d.h_bonds.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(d.elig, d.h_elig.data(), 4 * d.h_elig.size(), cudaMemcpyHostToDevice);
  if ((e = cudaGetLastError()) != cudaSuccess) { ligate_batch_destroy(S); return cuda_fail(e, "autotune sample"); }
  *out = S;
  return LIGATE_OK;
}

// Time one run of `tile` on batch B (ms); negative on failure.
static double time_tile(const ligate_pocket *P, const ligate_batch *B, const ligate_sampling *s,
                        const ligate_tile &tile, int reps) {
  ligate_plan *pl = nullptr;
  if (ligate_plan_create(P, B, s, &tile, &pl) != LIGATE_OK) return -1;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  double best = -1;
  if (ligate_plan_run(pl, nullptr, 0) == LIGATE_OK && cudaDeviceSynchronize() == cudaSuccess) {
    for (int r = 0; r < reps; ++r) {
      cudaEventRecord(a, 0);
      ligate_plan_run(pl, nullptr, 0);
      cudaEventRecord(b, 0);
      cudaEventSynchronize(b);
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      if (best < 0 || ms < best) best = ms;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  ligate_plan_destroy(pl);
  return best;
}

extern "C" ligate_status ligate_model_tile(const ligate_pocket *P, const ligate_batch *B,
                                           const ligate_sampling *s, ligate_tile *out) {
  if (!out) { set_error("model_tile: out is NULL"); return LIGATE_ERR_INVALID; }
  int mode = 0;
  ligate_status st = check_sampling(P, B, s, &mode);
  if (st != LIGATE_OK) return st;
  int dev = 0, sms = 1, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const int S = s->torsion_steps, G = 32 / pow2ceil(S);
  const int nmax = std::max(32, (B->d.max_atoms + 31) / 32 * 32);
  const size_t per_warp = dock_smem_per_warp(nmax, S, G, B->d.max_rot);
  ligate_tile t;
  memset(&t, 0, sizeof(t));
  int best_res = 0;
  for (int cap = 1; cap <= 3; ++cap) {
    if (mode == MODE_F32_PLAIN && cap != 3) continue;
    if (cap < 3 && dock_kernel_local_bytes(mode, cap) > 0) continue;  // spills: registers too tight
    const int minb = cap == 1 ? 6 : cap == 2 ? 5 : 4;  // CTAs of 128 threads the register cap allows
    for (int warps : {2, 4}) {
      const size_t cta_smem = per_warp * warps + 1024;  // + the per-CTA reserve
      if (cta_smem > 227 * 1024) continue;
      const int by_regs = minb * 4 / warps;
      const int by_smem = (int)(smem_sm / cta_smem);
      const int res = std::min(by_regs, by_smem) * warps;  // resident warps per SM
      if (res > best_res) { best_res = res; t.warps_per_cta = warps; t.reg_cap = cap; }
    }
  }
  if (best_res == 0) {
    set_error("model_tile: ligands too large for any CTA shape");
    return LIGATE_ERR_UNSUPPORTED;
  }
  model_chunks(B->d, nullptr, B->d.n_ligands, S, s->n_orient * s->n_anchor, (double)sms * best_res, G,
               t.starts_per_item);
  *out = t;
  return LIGATE_OK;
}

extern "C" ligate_status ligate_autotune(const ligate_pocket *P, const ligate_batch *B,
                                         const ligate_sampling *s, double budget_ms,
                                         ligate_tile *best) {
  NvtxRange nvtx_("ligate:autotune");
  int mode = 0;
  ligate_status st = check_sampling(P, B, s, &mode);
  if (st != LIGATE_OK) return st;
  if (!best) { set_error("autotune: best is NULL"); return LIGATE_ERR_INVALID; }
  const auto t_start = std::chrono::steady_clock::now();
  auto elapsed = [&]() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  };
  ligate_tile cur;
  memset(&cur, 0, sizeof(cur));
  if (B->d.n_ligands == 0) {  // nothing to time: the default shape
    cur.warps_per_cta = 4;
    *best = cur;
    return LIGATE_OK;
  }
  // CTA shape and register cap, timed on up to 2048 ligands spread over the
  // batch (long enough a run for the steady state the full run sees); chunk
  // sizes come from the work model at plan time (zero fields), so the shape
  // carries over to batches of any size
  std::vector<int> shape_sample;
  {
    const int n = B->d.n_ligands, m = std::min(n, 2048);
    for (int j = 0; j < m; ++j) shape_sample.push_back((int)((long long)j * n / m));
  }
  ligate_batch *SB = nullptr;
  if ((st = sub_batch(B, shape_sample, &SB)) != LIGATE_OK) return st;
  double best_ms = -1;
  ligate_tile best_t = cur;
  for (int shape = 0; shape < 6; ++shape) {  // 2 or 4 warps x register caps 85 / 102 / 128
    ligate_tile t;
    memset(&t, 0, sizeof(t));
    t.warps_per_cta = (shape & 1) ? 4 : 2;
    t.reg_cap = 1 + (shape >> 1);
    const double ms = time_tile(P, SB, s, t, 3);
    if (ms > 0 && (best_ms < 0 || ms < best_ms)) { best_ms = ms; best_t = t; }
    if (elapsed() > budget_ms) break;
  }
  ligate_batch_destroy(SB);
  if (best_ms < 0) { set_error("autotune: no candidate shape ran"); return LIGATE_ERR_CUDA; }
  cur = best_t;
  *best = cur;
  write_tune_cache(s->torsion_steps, mode, cur);
  return LIGATE_OK;
}
