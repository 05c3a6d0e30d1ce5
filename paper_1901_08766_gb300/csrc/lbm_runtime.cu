// Host runtime of the TRT-LBM-VP library: domains, batches with tile work lists,
// CUDA-graph replay of step chunks, the tile autotuner, and the C ABI of include/lbm.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <nvtx3/nvToolsExt.h>

#include "lbm_internal.h"

namespace lbm {
namespace {
thread_local std::string g_last_error;
}  // namespace

void set_last_error(const char *msg) { g_last_error = msg; }

namespace {

// A named NVTX range over a scope (seen by profilers that record NVTX; inert otherwise).
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range &) = delete;
  Range &operator=(const Range &) = delete;
};

lbm_status fail(lbm_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define LBM_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(LBM_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                              \
  } while (0)

size_t elem_size(int storage) {
  switch (storage) {
    case LBM_F64: return 8;
    case LBM_F32: return 4;
    case LBM_F16S: return 2;
    case LBM_BF16S: return 2;
    default: return 0;
  }
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int pitch_of(int nx) { return static_cast<int>(align_up(static_cast<size_t>(nx), kPitchAlign)); }

struct Alloc {
  lbm_alloc_fn fn = nullptr;
  lbm_free_fn ffn = nullptr;
  void *ctx = nullptr;
  cudaStream_t st = nullptr;
  void *get(size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (fn) return fn(bytes, ctx);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void *p) {
    if (!p) return;
    if (ffn) ffn(p, ctx);
    else cudaFreeAsync(p, st);
  }
};

// Fixed part of a domain's device footprint (populations x2, mask, bodies, offsets,
// force ring, status word), each piece 256-byte aligned.
struct Layout {
  size_t lat_bytes, mask_off, fvp_off, bodies_off, bodies_f_off, kappa_off, off_off, ring_off, status_off,
      shapes_off, centre0_off, rowsum_off, fsi_off, def_off, total;
};

Layout layout_of(const lbm_params &p, int nbodies) {
  Layout L;
  const size_t pitch = pitch_of(p.nx);
  const size_t es = elem_size(p.storage);
  const int cap = p.force_capacity > 0 ? p.force_capacity : 8192;
  L.lat_bytes = align_up(static_cast<size_t>(kQ) * p.ny * pitch * es, 256);
  size_t o = 2 * L.lat_bytes;
  L.mask_off = o;
  o += align_up(static_cast<size_t>(p.ny) * pitch, 256);
  L.fvp_off = o;  // two F_VP fields (by lattice parity)
  o += 2 * align_up(static_cast<size_t>(p.ny) * pitch * 2 * (p.storage == LBM_F64 ? 8 : 4), 256);
  L.bodies_off = o;
  o += align_up(sizeof(double) * 5 * std::max(1, nbodies), 256);
  L.bodies_f_off = o;
  o += align_up(sizeof(float) * 5 * std::max(1, nbodies), 256);
  // dilation rates of the bodies, FP64 then FP32 (zero unless a body pulsates)
  L.kappa_off = o;
  o += align_up(sizeof(double) * std::max(1, nbodies), 256) + align_up(sizeof(float) * std::max(1, nbodies), 256);
  L.off_off = o;
  o += align_up(sizeof(int32_t) * (nbodies + 1), 256);
  L.ring_off = o;
  o += align_up(p.force_every > 0 ? sizeof(double) * 2 * std::max(1, nbodies) * cap : 16, 256);
  L.status_off = o;
  o += 256;
  // moving domains: reference geometry, reference centres, per-row force sums
  L.shapes_off = L.centre0_off = L.rowsum_off = L.fsi_off = L.def_off = o;
  if (p.moving) {
    // the shapes, their FP32 centre and extent (the move kernel's culling), and the
    // shapes placed at the next step index (written each step by the shape table kernel)
    o += align_up((sizeof(ShapeDev) + sizeof(float4) + sizeof(PlacedShape)) * kMaxMovingShapes, 256);
    L.centre0_off = o;
    o += align_up(sizeof(double) * 2 * std::max(1, nbodies), 256);
    L.rowsum_off = o;  // two tables (by lattice parity)
    o += align_up(2 * sizeof(double) * 3 * std::max(1, nbodies) * static_cast<size_t>(p.ny), 256);
    // coupled bodies: state of two step parities [2][nbodies][6], parameters [nbodies][8]
    L.fsi_off = o;
    o += align_up(sizeof(double) * 20 * std::max(1, nbodies), 256);
    // pulsating bodies: amplitude and rate [nbodies][2]; turning or pulsating bodies: cos,
    // sin and scale of the next step index [2][nbodies][3]
    L.def_off = o;
    o += align_up(sizeof(double) * 8 * std::max(1, nbodies), 256);
  }
  L.total = o;
  return L;
}

lbm_status validate(const lbm_params *p, int nbodies) {
  if (!p) return fail(LBM_EINVAL, "params is NULL");
  if (p->nx < 3 || p->ny < 3) return fail(LBM_EINVAL, "nx, ny must be >= 3 (got %d, %d)", p->nx, p->ny);
  if (static_cast<long long>(pitch_of(p->nx)) * p->ny > (1ll << 31) / 2)
    return fail(LBM_EINVAL, "grid too large for 32-bit node indices");
  if (elem_size(p->storage) == 0) return fail(LBM_EINVAL, "unknown storage %d", p->storage);
  const double tau = p->nu > 0 ? 3.0 * p->nu + 0.5 : p->tau_plus;
  if (!(tau > 0.5)) return fail(LBM_EINVAL, "tau_plus must exceed 1/2 (got %g)", tau);
  if (!(p->magic_lambda > 0)) return fail(LBM_EINVAL, "magic parameter must be > 0");
  if (!(p->eta > 0)) return fail(LBM_EINVAL, "eta must be > 0");
  if (!(p->rho0 > 0)) return fail(LBM_EINVAL, "rho0 must be > 0");
  if (p->west != LBM_PERIODIC && p->west != LBM_INLET_EQ) return fail(LBM_EINVAL, "west edge must be PERIODIC or INLET_EQ");
  if (p->east != LBM_PERIODIC && p->east != LBM_OUTFLOW_ZG) return fail(LBM_EINVAL, "east edge must be PERIODIC or OUTFLOW_ZG");
  if ((p->west == LBM_PERIODIC) != (p->east == LBM_PERIODIC)) return fail(LBM_EINVAL, "x edges: both periodic or neither");
  if (p->south != LBM_PERIODIC && p->south != LBM_FREE_SLIP) return fail(LBM_EINVAL, "south edge must be PERIODIC or FREE_SLIP");
  if (p->north != LBM_PERIODIC && p->north != LBM_FREE_SLIP) return fail(LBM_EINVAL, "north edge must be PERIODIC or FREE_SLIP");
  if ((p->south == LBM_PERIODIC) != (p->north == LBM_PERIODIC)) return fail(LBM_EINVAL, "y edges: both periodic or neither");
  if (nbodies < 0 || nbodies > kMaxBodies) return fail(LBM_EINVAL, "nbodies must be in [0, 255]");
  if (p->force_every < 0 || p->force_capacity < 0) return fail(LBM_EINVAL, "force_every/capacity must be >= 0");
  if (p->moving < 0 || p->moving > 2) return fail(LBM_EINVAL, "moving must be 0, 1 or 2");
  if ((p->storage == LBM_F16S || p->storage == LBM_BF16S) && p->x_origin % 8 != 0)
    return fail(LBM_EINVAL, "16-bit storage needs x_origin divisible by 8 (rounding bits are keyed by 8-column groups)");
  if (p->moving && nbodies > kMaxMovingBodies)
    return fail(LBM_EINVAL, "a moving domain has at most %d bodies", kMaxMovingBodies);
  return LBM_OK;
}

struct Slot {
  bool used = false;
  lbm_params p{};
  int nbodies = 0;
  int pitch = 0;
  long long target = 0;
  long long done = 0;
  int parity = 0;
  long long drained = 0;
  void *block = nullptr;
  void *solid = nullptr;
  size_t bytes = 0;
  std::vector<int32_t> solid_off;  // host copy of the per-body offsets into the solid list
  int link_west = -1, link_east = -1;  // slots linked across the x edges (-1: none, -2: a
                                       // halo edge fed from a caller's buffer)
  void *halo_send[2] = {nullptr, nullptr};  // halo edges: where lbm_batch_pack_halos writes
  bool fsi = false;                    // some body responds to its force
  int group = -1;  // >= 0: block and solid list are carved from the shared allocations of
                   // a batched admission (lbm_batch::groups[group])
  DomDev dev{};
};

// The two allocations a batched admission takes for all of its domains (domain blocks,
// solid lists), returned when the last of those domains leaves the batch; `bytes` is
// what the domains count against the memory budget until then.
struct Group {
  void *block = nullptr, *solid = nullptr;
  int members = 0;
  size_t bytes = 0;
};

}  // namespace

// Collision constants of a domain in FP32 and FP64 (per-class products of the relaxation
// rates with the D2Q9 weights, the penalization factor, the shifts and the inlet ghost).
template <typename T> void fill_const(CellConst<T> &c, const DomDev &d) {
  const double w0 = 4.0 / 9.0, w1 = 1.0 / 9.0, w2 = 1.0 / 36.0;
  const double op = d.omega_p, om = d.omega_m;
  c.omp = T(op);
  c.omm = T(om);
  c.hp = T(0.5 * op);
  c.hm = T(0.5 * om);
  c.one_m_omp = T(1.0 - op);
  c.inv_2eta1 = T(d.inv_2eta1);
  c.rho0 = T(d.rho0);
  c.pw0 = T(op * w0);
  c.pw1 = T(op * w1);
  c.pw2 = T(op * w2);
  c.mw1 = T(3.0 * om * w1);
  c.mw2 = T(3.0 * om * w2);
  c.kw0 = T((1.0 - 0.5 * op) * w0);
  c.kw1 = T((1.0 - 0.5 * op) * w1);
  c.kw2 = T((1.0 - 0.5 * op) * w2);
  c.qw1 = T(3.0 * (1.0 - 0.5 * om) * w1);
  c.qw2 = T(3.0 * (1.0 - 0.5 * om) * w2);
  c.wr0 = T(w0 * d.rho0);
  c.wr1 = T(w1 * d.rho0);
  c.wr2 = T(w2 * d.rho0);
  for (int a = 0; a < kQ; ++a) c.ghost[a] = T(d.ghost[a]);
}

// The inlet ghost enters the update like a stored node: in FP32 compute it is the value
// an FP32/FP16/BF16 lattice would hold for f^eq(rho0, u_in), so that the inflow and the
// free stream leaving through the outflow carry the same rounding (otherwise the
// mismatch adds or removes mass at every step).
void fill_cell_const(DomDev &d, int storage) {
  fill_const(d.cd, d);
  fill_const(d.cf, d);
  if (storage == LBM_F16S) d.cf.rho0 = float(d.rho0 * kF16Scale);  // compute space is scaled
  const double w[kQ] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
  for (int a = 0; a < kQ; ++a) {
    const float shift = float(w[a] * d.rho0);
    if (storage == LBM_F32) {
      d.cf.ghost[a] = float(d.ghost[a]) - shift;  // stored f, minus the shift as after loading
    } else if (storage == LBM_F16S) {
      d.cf.ghost[a] = __half2float(__float2half_rn(float(d.ghost[a] * kF16Scale)));
    } else if (storage == LBM_BF16S) {
      d.cf.ghost[a] = __bfloat162float(__float2bfloat16_rn(float(d.ghost[a])));
    }
  }
}

}  // namespace lbm

using namespace lbm;

struct lbm_batch {
  int max_domains = 0;
  size_t budget = 0;
  int storage = 0;
  int graph_steps = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  Alloc al;
  std::vector<Slot> slots;
  DomDev *d_doms = nullptr;
  DomDyn *d_dyn = nullptr;
  DomDyn *h_dyn = nullptr;  // pinned staging
  cudaEvent_t dyn_ev = nullptr;
  // the force reduction of a fixed-geometry batch runs on a second stream beside the next
  // step's sweep: ev_sweep orders it after its sweep, ev_force[s & 1] the sweep two steps
  // later (which rewrites the F_VP field it reads) after it, ev_join the batch stream
  // after the last of them
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_sweep = nullptr, ev_force[2] = {nullptr, nullptr}, ev_join = nullptr;
  TileDev *d_tiles = nullptr;
  int tiles_cap = 0;
  ForceItem *d_items = nullptr;
  int items_cap = 0;
  MoveRow *d_moves = nullptr;  // rows of moving domains (geometry update after each sweep)
  BusyRow *d_busy = nullptr;   // the move kernels' list of busy rows (as many entries as d_moves)
  int moves_cap = 0;
  int nmove = 0;               // rows in the list; 0: no move kernel in the step
  int nmovedom = 0;            // moving domains, listed after the rows (d_moves + nmove)
  bool has_fsi = false;        // some resident domain has coupled bodies: fsi kernel per step
  bool has_deform = false;     // some resident domain has pulsating bodies: the sweep with
                               // the dilation term of U_O
  Counters *d_ctr = nullptr;
  Counters *h_ctr = nullptr;  // pinned staging for tile/item counts
  int vec = 0, warps = 0, rows = 0, pipe = 0;
  int grid_sweep = 0, grid_force = 0;
  // the move kernels' per-row pass: four of its 256-thread blocks (64 registers, 44 KB
  // of shared memory) fit on an SM; each listed row gets a warp, so more warps leave
  // fewer rows to one warp (a move kernel that walked its rows itself: 400.5 -> 392.3 us
  // per step of the all-moving 64-domain batch at three blocks per SM against two)
  int grid_move = 0;
  int ntiles = 0, nitems = 0;
  bool dirty = true;
  cudaGraphExec_t graph = nullptr;
  long long launches = 0;
  size_t bytes_in_use = 0;
  int sm_count = 0;
  int inject = 0;  // SweepArgs::inject of later sweep launches (host failure injection)
  char *h_poll = nullptr;  // pinned staging of lbm_batch_poll_many (grows as needed)
  size_t h_poll_cap = 0;
  bool h_poll_own = false;  // h_poll is its own allocation (else a part of h_pin)
  char *h_pin = nullptr;    // one pinned block: h_dyn, h_ctr and the first h_poll
  void *d_base = nullptr;   // one device block: d_doms, d_dyn, d_ctr
  char *d_poll = nullptr;  // device staging where lbm_batch_poll_many gathers (grows as needed)
  size_t d_poll_cap = 0;
  std::vector<Group> groups;  // shared allocations of batched admissions (free entries reused)
  bool group_admit = true;    // lbm_batch_admit_many takes shared allocations
  cudaEvent_t adm_ev = nullptr;  // lbm_batch_admit_many: the per-row counts are on the host
  // moving domains: the shape table of a step runs on st2 beside its sweep, after ev_pre
  // (the previous step's move kernel); the move kernel waits for ev_tab
  cudaEvent_t ev_pre = nullptr, ev_tab = nullptr;
};

struct lbm_domain {
  lbm_batch *b = nullptr;
};

namespace lbm {
namespace {

cudaError_t sweep_launch(lbm_batch *b, int grid, int vec, int pipe, int warps, int rows, int s) {
  SweepArgs a{b->d_doms, b->d_dyn, b->d_tiles, b->d_ctr, rows, b->inject};
  const bool def = b->has_deform;  // the direct sweep instantiated with the kappa term
  switch (b->storage) {
    case LBM_F64: return launch_sweep_f64(vec, pipe, grid, warps, b->st, a, s, def);
    case LBM_F32: return launch_sweep_f32(vec, pipe, grid, warps, b->st, a, s, def);
    case LBM_F16S: return launch_sweep_f16s(vec, pipe, grid, warps, b->st, a, s, def);
    case LBM_BF16S: return launch_sweep_bf16s(vec, pipe, grid, warps, b->st, a, s, def);
  }
  return cudaErrorInvalidValue;
}

int sweep_occupancy(int storage, int vec, int pipe, int warps) {
  switch (storage) {
    case LBM_F64: return max_blocks_f64(vec, pipe, warps);
    case LBM_F32: return max_blocks_f32(vec, pipe, warps);
    case LBM_F16S: return max_blocks_f16s(vec, pipe, warps);
    case LBM_BF16S: return max_blocks_bf16s(vec, pipe, warps);
  }
  return 0;
}

bool vec_ok(int storage, int vec) {
  switch (storage) {
    case LBM_F64: return vec == 1 || vec == 2;
    case LBM_F32: return vec == 2 || vec == 4;
    default: return vec == 4 || vec == 8;
  }
}

// The tile a batch starts with: the autotuner's choice on the 64-domain batched workload
// (16-bit storage: 8 cells per thread, 12-warp blocks at 24 resident warps per SM, 376 us;
// FP32: 4 cells per thread, 16-warp blocks, 623 us); FP64 (ALU-bound) 4-warp blocks.
void default_tile(int storage, int &vec, int &warps, int &rows, int &pipe) {
  vec = storage == LBM_F64 ? 2 : (storage == LBM_F32 ? 4 : 8);
  warps = storage == LBM_F64 ? 4 : (storage == LBM_F32 ? 16 : 12);
  rows = 4;
  pipe = (storage == LBM_F16S || storage == LBM_BF16S) ? 4 : 0;
}

void drop_graph(lbm_batch *b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

lbm_status set_config(lbm_batch *b, int vec, int warps, int rows, int pipe) {
  if (!vec_ok(b->storage, vec)) return fail(LBM_EINVAL, "cells per thread %d unsupported for storage %d", vec, b->storage);
  if (warps < 1 || warps > 16 || rows < 1 || rows > 16) return fail(LBM_EINVAL, "warps and rows must be in [1, 16]");
  if (pipe < 0 || pipe > 4)
    return fail(LBM_EINVAL, "pipeline must be 0 (direct), 1 (TMA-staged), 2 (register-prefetched), "
                            "3 or 4 (direct for 20 or 24 resident warps)");
  if (vec == b->vec && warps == b->warps && rows == b->rows && pipe == b->pipe && b->grid_sweep > 0)
    return LBM_OK;  // unchanged: the work lists and the captured graph stay valid
  const int occ = sweep_occupancy(b->storage, vec, pipe, warps);
  if (occ <= 0) return fail(LBM_ECUDA, "sweep kernel cannot run with %d warps per block", warps);
  b->vec = vec;
  b->warps = warps;
  b->rows = rows;
  b->pipe = pipe;
  b->grid_sweep = occ * b->sm_count;
  b->dirty = true;
  drop_graph(b);
  return LBM_OK;
}

// Rebuild the tile and force-item lists of the resident slots and upload them.
lbm_status rebuild_lists(lbm_batch *b) {
  std::vector<TileDev> tiles;
  std::vector<ForceItem> items;
  std::vector<MoveRow> moves;
  const int tw = 32 * b->vec, th = b->warps * b->rows;
  for (int k = 0; k < b->max_domains; ++k) {
    const Slot &s = b->slots[k];
    if (!s.used) continue;
    for (int y0 = 0; y0 < s.p.ny; y0 += th)
      for (int x0 = 0; x0 < s.p.nx; x0 += tw) tiles.push_back(TileDev{k, x0, y0, 0});
    if (s.p.moving)
      for (int j = 0; j < s.p.ny; ++j) moves.push_back(MoveRow{k, j});
    if (s.p.force_every > 0)
      for (int body = 1; body <= s.nbodies; ++body)
        items.push_back(s.p.moving ? ForceItem{k, body, 0, s.p.ny, 1, 0}
                                   : ForceItem{k, body, s.solid_off[body - 1], s.solid_off[body], 0, 0});
  }
  // a captured graph holds the move kernel only if there were moving rows at capture,
  // and the fsi kernel only if some domain had coupled bodies
  bool has_fsi = false, has_deform = false;
  for (const Slot &s : b->slots) {
    has_fsi = has_fsi || (s.used && s.fsi);
    has_deform = has_deform || (s.used && s.dev.deform != 0u);
  }
  if ((b->nmove > 0) != !moves.empty() || has_fsi != b->has_fsi || has_deform != b->has_deform) drop_graph(b);
  // after the rows: one entry per moving domain (the shape table kernel's blocks)
  const int nrows_move = static_cast<int>(moves.size());
  for (int k = 0; k < b->max_domains && nrows_move > 0; ++k)
    if (b->slots[k].used && b->slots[k].p.moving) moves.push_back(MoveRow{k, -1});
  b->has_fsi = has_fsi;
  b->has_deform = has_deform;
  if (static_cast<int>(moves.size()) > b->moves_cap || (!moves.empty() && !b->d_moves)) {
    const int cap = std::max<int>(static_cast<int>(moves.size()) * 2, 1024);
    LBM_CUDA(cudaStreamSynchronize(b->st));
    b->al.put(b->d_moves);
    b->al.put(b->d_busy);
    b->d_moves = static_cast<MoveRow *>(b->al.get(sizeof(MoveRow) * cap));
    b->d_busy = static_cast<BusyRow *>(b->al.get(sizeof(BusyRow) * cap));
    if (!b->d_moves || !b->d_busy) { b->moves_cap = 0; return fail(LBM_ENOMEM, "move list allocation failed"); }
    b->moves_cap = cap;
    drop_graph(b);
  }
  b->nmove = nrows_move;
  b->nmovedom = static_cast<int>(moves.size()) - nrows_move;
  if (!moves.empty())
    LBM_CUDA(cudaMemcpyAsync(b->d_moves, moves.data(), sizeof(MoveRow) * moves.size(),
                             cudaMemcpyHostToDevice, b->st));
  if (static_cast<int>(tiles.size()) > b->tiles_cap || !b->d_tiles) {
    const int cap = std::max<int>(static_cast<int>(tiles.size()) * 2, 1024);
    LBM_CUDA(cudaStreamSynchronize(b->st));
    b->al.put(b->d_tiles);
    b->d_tiles = static_cast<TileDev *>(b->al.get(sizeof(TileDev) * cap));
    if (!b->d_tiles) { b->tiles_cap = 0; return fail(LBM_ENOMEM, "tile list allocation failed"); }
    b->tiles_cap = cap;
    drop_graph(b);
  }
  if (static_cast<int>(items.size()) > b->items_cap || !b->d_items) {
    const int cap = std::max<int>(static_cast<int>(items.size()) * 2, 256);
    LBM_CUDA(cudaStreamSynchronize(b->st));
    b->al.put(b->d_items);
    b->d_items = static_cast<ForceItem *>(b->al.get(sizeof(ForceItem) * cap));
    if (!b->d_items) { b->items_cap = 0; return fail(LBM_ENOMEM, "force item allocation failed"); }
    b->items_cap = cap;
    drop_graph(b);
  }
  b->ntiles = static_cast<int>(tiles.size());
  b->nitems = static_cast<int>(items.size());
  // synchronous uploads from pageable vectors: the copies complete before return
  if (!tiles.empty())
    LBM_CUDA(cudaMemcpyAsync(b->d_tiles, tiles.data(), sizeof(TileDev) * tiles.size(),
                             cudaMemcpyHostToDevice, b->st));
  if (!items.empty())
    LBM_CUDA(cudaMemcpyAsync(b->d_items, items.data(), sizeof(ForceItem) * items.size(),
                             cudaMemcpyHostToDevice, b->st));
  LBM_CUDA(cudaEventSynchronize(b->dyn_ev));
  b->h_ctr->ntiles = b->ntiles;
  b->h_ctr->nforce = b->nitems;
  b->h_ctr->run_base = 0;
  b->h_ctr->nmove = b->nmove;
  b->h_ctr->nmovedom = b->nmovedom;
  b->h_ctr->item_next = 0;
  b->h_ctr->item_done = 0;
  b->h_ctr->nbusy = 0;
  b->h_ctr->busy_done = 0;
  LBM_CUDA(cudaMemcpyAsync(b->d_ctr, b->h_ctr, sizeof(Counters), cudaMemcpyHostToDevice, b->st));
  LBM_CUDA(cudaStreamSynchronize(b->st));
  b->dirty = false;
  return LBM_OK;
}

// Enqueue step s of the current run: the force reduction reads the same lattice as the
// sweep, so the two are ordered only against the next step.
// Step s of the current run: the sweep, then the force reduction over the F_VP field the
// sweep wrote. The force kernel is launched even when no body records forces (it returns
// at once), so that a captured graph stays valid when the batch membership changes.
// Batches without coupled bodies fork the force reduction to the second stream: it reads
// the F_VP field (and, for moving domains, the row sums) of step s's parity while step
// s + 1's sweep and move kernel write the other ones, so it runs beside that sweep (its
// small blocks fit next to the sweep's). Coupled bodies keep one stream: their next state
// and geometry depend on the forces.
bool forks(const lbm_batch *b) { return !b->has_fsi; }

lbm_status enqueue_step(lbm_batch *b, int s) {
  const bool fork = forks(b);
  if (fork && b->nmove > 0) {
    // the moving shapes at the next index and the list of rows they reach, on the second
    // stream beside the sweep (neither reads what the sweep writes)
    LBM_CUDA(cudaEventRecord(b->ev_pre, b->st));
    LBM_CUDA(cudaStreamWaitEvent(b->st2, b->ev_pre, 0));
    LBM_CUDA(launch_shape_table(b->grid_force, b->st2, b->d_doms, b->d_dyn, b->d_moves, b->d_ctr, s));
    LBM_CUDA(launch_move_cull(b->grid_force, b->st2, b->d_doms, b->d_dyn, b->d_moves, b->d_ctr, b->d_busy, s));
    LBM_CUDA(cudaEventRecord(b->ev_tab, b->st2));
    b->launches += 2;
  }
  // the sweep rewrites the F_VP field that step s - 2's force reduction read
  if (fork && s >= 2) LBM_CUDA(cudaStreamWaitEvent(b->st, b->ev_force[s & 1], 0));
  LBM_CUDA(sweep_launch(b, b->grid_sweep, b->vec, b->pipe, b->warps, b->rows, s));
  b->launches++;
  if (fork) {
    if (b->nmove > 0) {  // moving domains: row force sums (by parity), then the next geometry
      LBM_CUDA(cudaStreamWaitEvent(b->st, b->ev_tab, 0));
      LBM_CUDA(launch_move_rows(b->grid_move, b->st, b->d_doms, b->d_dyn, b->d_moves, b->d_ctr, b->d_busy, s, b->storage));
      b->launches++;
    }
    LBM_CUDA(cudaEventRecord(b->ev_sweep, b->st));
    LBM_CUDA(cudaStreamWaitEvent(b->st2, b->ev_sweep, 0));
    LBM_CUDA(launch_forces(b->storage, b->grid_force, b->st2, b->d_doms, b->d_dyn, b->d_items, b->d_ctr, s));
    LBM_CUDA(cudaEventRecord(b->ev_force[s & 1], b->st2));
    b->launches++;
    return LBM_OK;
  }
  if (b->nmove > 0) {  // moving domains: row force sums, then the next step's geometry
    LBM_CUDA(launch_shape_table(b->grid_force, b->st, b->d_doms, b->d_dyn, b->d_moves, b->d_ctr, s));
    LBM_CUDA(launch_move_cull(b->grid_force, b->st, b->d_doms, b->d_dyn, b->d_moves, b->d_ctr, b->d_busy, s));
    LBM_CUDA(launch_move_rows(b->grid_move, b->st, b->d_doms, b->d_dyn, b->d_moves, b->d_ctr, b->d_busy, s, b->storage));
    b->launches += 3;
  }
  LBM_CUDA(launch_forces(b->storage, b->grid_force, b->st, b->d_doms, b->d_dyn, b->d_items,
                         b->d_ctr, s));
  b->launches++;
  if (b->has_fsi) {  // coupled bodies: new state from this step's force, next geometry
    LBM_CUDA(launch_fsi(b->grid_force, b->st, b->d_doms, b->d_dyn, b->d_moves, b->d_ctr, s));
    b->launches++;
  }
  return LBM_OK;
}

// The batch stream waits for the force reductions forked to the second stream.
lbm_status join_side(lbm_batch *b) {
  if (!forks(b)) return LBM_OK;
  LBM_CUDA(cudaEventRecord(b->ev_join, b->st2));
  LBM_CUDA(cudaStreamWaitEvent(b->st, b->ev_join, 0));
  return LBM_OK;
}

lbm_status capture_graph(lbm_batch *b) {
  drop_graph(b);
  cudaGraph_t g = nullptr;
  LBM_CUDA(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
  const long long before = b->launches;
  lbm_status rc = LBM_OK;
  for (int s = 0; s < b->graph_steps && rc == LBM_OK; ++s) rc = enqueue_step(b, s);
  if (rc == LBM_OK) rc = join_side(b);
  cudaError_t e = rc == LBM_OK ? launch_advance(b->st, b->d_ctr, b->graph_steps) : cudaSuccess;
  cudaError_t e2 = cudaStreamEndCapture(b->st, &g);
  b->launches = before;  // capture only records; replays count
  if (rc != LBM_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(LBM_ECUDA, "graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  cudaError_t e3 = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e3 != cudaSuccess) {
    b->graph = nullptr;
    return fail(LBM_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e3));
  }
  return LBM_OK;
}

lbm_status upload_dyn(lbm_batch *b) {
  LBM_CUDA(cudaEventSynchronize(b->dyn_ev));
  for (int k = 0; k < b->max_domains; ++k) {
    const Slot &s = b->slots[k];
    DomDyn &d = b->h_dyn[k];
    d.step0 = s.done;
    d.step_end = s.used ? s.target : s.done;
    d.parity = s.parity;
    d.pad = 0;
  }
  LBM_CUDA(cudaMemcpyAsync(b->d_dyn, b->h_dyn, sizeof(DomDyn) * b->max_domains,
                           cudaMemcpyHostToDevice, b->st));
  LBM_CUDA(cudaMemsetAsync(&b->d_ctr->run_base, 0, sizeof(long long), b->st));
  LBM_CUDA(cudaEventRecord(b->dyn_ev, b->st));
  return LBM_OK;
}

long long entries_at(const Slot &s, long long steps) {
  return s.p.force_every > 0 ? steps / s.p.force_every : 0;
}

struct Profile {
  double sweep_ms = 0.0, force_ms = 0.0;
};

lbm_status run(lbm_batch *b, long long max_steps, long long *steps_run, Profile *prof = nullptr) {
  if (steps_run) *steps_run = 0;
  if (max_steps < 0) return fail(LBM_EINVAL, "max_steps must be >= 0");
  long long steps = 0;
  for (const Slot &s : b->slots)
    if (s.used && s.done < s.target) steps = std::max(steps, std::min(max_steps, s.target - s.done));
  if (steps == 0) return LBM_OK;
  for (const Slot &s : b->slots) {
    if (!s.used || s.p.force_every <= 0) continue;
    const long long end = std::min(s.target, s.done + steps);
    const int cap = s.dev.force_cap;
    if (entries_at(s, end) - s.drained > cap)
      return fail(LBM_EBUSY, "force ring would overflow (%lld undrained + new > %d)",
                  entries_at(s, end) - s.drained, cap);
  }
  if (b->dirty) {
    lbm_status rc = rebuild_lists(b);
    if (rc != LBM_OK) return rc;
  }
  lbm_status rc = upload_dyn(b);
  if (rc != LBM_OK) return rc;
  long long s0 = 0;
  if (prof) {
    // one kernel at a time, each bracketed by events on the batch stream
    std::vector<cudaEvent_t> ev(3 * steps);
    for (auto &e : ev) LBM_CUDA(cudaEventCreate(&e));
    lbm_status prc = LBM_OK;
    for (long long s = 0; s < steps && prc == LBM_OK; ++s) {
      cudaEventRecord(ev[3 * s], b->st);
      if (sweep_launch(b, b->grid_sweep, b->vec, b->pipe, b->warps, b->rows, static_cast<int>(s)) != cudaSuccess)
        prc = fail(LBM_ECUDA, "sweep launch failed");
      cudaEventRecord(ev[3 * s + 1], b->st);
      if (b->nmove > 0) {
        if (launch_shape_table(b->grid_force, b->st, b->d_doms, b->d_dyn, b->d_moves, b->d_ctr,
                               static_cast<int>(s)) != cudaSuccess ||
            launch_move_cull(b->grid_force, b->st, b->d_doms, b->d_dyn, b->d_moves, b->d_ctr, b->d_busy,
                             static_cast<int>(s)) != cudaSuccess ||
            launch_move_rows(b->grid_move, b->st, b->d_doms, b->d_dyn, b->d_moves, b->d_ctr, b->d_busy,
                             static_cast<int>(s), b->storage) != cudaSuccess)
          prc = fail(LBM_ECUDA, "move launch failed");
        b->launches += 3;
      }
      if (launch_forces(b->storage, b->grid_force, b->st, b->d_doms, b->d_dyn, b->d_items, b->d_ctr,
                        static_cast<int>(s)) != cudaSuccess)
        prc = fail(LBM_ECUDA, "force launch failed");
      if (b->has_fsi) {
        if (launch_fsi(b->grid_force, b->st, b->d_doms, b->d_dyn, b->d_moves, b->d_ctr,
                       static_cast<int>(s)) != cudaSuccess)
          prc = fail(LBM_ECUDA, "fsi launch failed");
        b->launches++;
      }
      cudaEventRecord(ev[3 * s + 2], b->st);
      b->launches += 2;
    }
    cudaStreamSynchronize(b->st);
    for (long long s = 0; s < steps && prc == LBM_OK; ++s) {
      float a = 0.f, c = 0.f;
      cudaEventElapsedTime(&a, ev[3 * s], ev[3 * s + 1]);
      cudaEventElapsedTime(&c, ev[3 * s + 1], ev[3 * s + 2]);
      prof->sweep_ms += a;
      prof->force_ms += c;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (prc != LBM_OK) return prc;
    s0 = steps;
  }
  if (!prof && b->graph_steps > 0 && steps >= b->graph_steps) {
    if (!b->graph) {
      rc = capture_graph(b);
      if (rc != LBM_OK) return rc;
    }
    const long long reps = steps / b->graph_steps;
    for (long long r = 0; r < reps; ++r) {
      LBM_CUDA(cudaGraphLaunch(b->graph, b->st));
      // per step: sweep, forces; moving domains: shape table, cull, rows; coupled: fsi
      b->launches += (2 + (b->nmove > 0 ? 3 : 0) + (b->has_fsi ? 1 : 0)) * static_cast<long long>(b->graph_steps) + 1;
    }
    s0 = reps * b->graph_steps;
  }
  // remaining steps as direct launches; the device counter already holds s0
  for (long long s = s0; s < steps; ++s) {
    rc = enqueue_step(b, static_cast<int>(s - s0));
    if (rc != LBM_OK) return rc;
  }
  if (s0 < steps) {
    rc = join_side(b);
    if (rc != LBM_OK) return rc;
  }
  for (Slot &s : b->slots) {
    if (!s.used || s.done >= s.target) continue;
    const long long adv = std::min(steps, s.target - s.done);
    s.done += adv;
    s.parity = static_cast<int>((s.parity + adv) & 1);
  }
  if (steps_run) *steps_run = steps;
  return LBM_OK;
}

lbm_status read_status(lbm_batch *b, const Slot &s, int *st) {
  LBM_CUDA(cudaMemcpyAsync(st, s.dev.status, sizeof(int32_t), cudaMemcpyDeviceToHost, b->st));
  LBM_CUDA(cudaStreamSynchronize(b->st));
  return LBM_OK;
}

// Host-side part of admitting a domain: the slot's parameters, its device block (one
// allocation holding lattices, mask, F_VP field, body tables, force ring, status word;
// or, with `block` given, that part of a batched admission's shared allocation) and its
// device description with the collision constants. No GPU work is issued.
lbm_status prepare_slot(lbm_batch *b, const lbm_params *p, const lbm_geometry *geom, int nbodies,
                        long long nsteps, const Layout &L, Slot &s, void *block = nullptr) {
  s = Slot();
  s.p = *p;
  if (s.p.force_capacity == 0) s.p.force_capacity = 8192;
  s.nbodies = nbodies;
  s.pitch = pitch_of(p->nx);
  s.target = nsteps;
  s.block = block ? block : b->al.get(L.total);
  if (!s.block) return fail(LBM_ENOMEM, "device allocation of %zu bytes failed", L.total);
  s.bytes = L.total;
  char *base = static_cast<char *>(s.block);
  DomDev &D = s.dev;
  D.lat[0] = base;
  D.lat[1] = base + L.lat_bytes;
  uint8_t *mask = reinterpret_cast<uint8_t *>(base + L.mask_off);
  D.mask = mask;
  double *bod = reinterpret_cast<double *>(base + L.bodies_off);
  D.bodies = bod;
  float *bodf = reinterpret_cast<float *>(base + L.bodies_f_off);
  D.bodies_f = bodf;
  int32_t *off = reinterpret_cast<int32_t *>(base + L.off_off);
  D.solid_off = off;
  D.fvp[0] = base + L.fvp_off;
  D.fvp[1] = base + L.fvp_off + (L.bodies_off - L.fvp_off) / 2;
  D.ring = reinterpret_cast<double *>(base + L.ring_off);
  D.status = reinterpret_cast<int32_t *>(base + L.status_off);
  D.moving = p->moving;
  D.x0 = p->x_origin;
  D.nshapes = p->moving ? geom->nshapes : 0;
  D.shapes = p->moving ? reinterpret_cast<const ShapeDev *>(base + L.shapes_off) : nullptr;
  D.shapes_f = p->moving ? reinterpret_cast<const float4 *>(base + L.shapes_off + sizeof(ShapeDev) * kMaxMovingShapes)
                         : nullptr;
  D.placed = p->moving ? reinterpret_cast<PlacedShape *>(base + L.shapes_off + (sizeof(ShapeDev) + sizeof(float4)) *
                                                                                  kMaxMovingShapes)
                       : nullptr;
  D.centre0 = p->moving ? reinterpret_cast<const double *>(base + L.centre0_off) : nullptr;
  D.rowsum[0] = p->moving ? reinterpret_cast<double *>(base + L.rowsum_off) : nullptr;
  D.rowsum[1] = p->moving ? D.rowsum[0] + 3 * static_cast<size_t>(std::max(1, nbodies)) * p->ny : nullptr;
  D.fsi = p->moving ? reinterpret_cast<double *>(base + L.fsi_off) : nullptr;
  D.fsi_par = p->moving ? reinterpret_cast<const double *>(base + L.fsi_off) + 12 * std::max(1, nbodies) : nullptr;
  D.fsi_on = 0;
  D.dpar = p->moving ? reinterpret_cast<const double *>(base + L.def_off) : nullptr;
  D.turn = p->moving ? reinterpret_cast<double *>(base + L.def_off) + 2 * std::max(1, nbodies) : nullptr;
  D.kappa = reinterpret_cast<double *>(base + L.kappa_off);
  D.kappa_f = reinterpret_cast<float *>(base + L.kappa_off + align_up(sizeof(double) * std::max(1, nbodies), 256));
  D.deform = 0u;
  D.nx = p->nx;
  D.ny = p->ny;
  D.pitch = s.pitch;
  D.west = p->west;
  D.east = p->east;
  D.south = p->south;
  D.north = p->north;
  D.nbodies = nbodies;
  D.force_every = p->force_every;
  D.force_cap = s.p.force_capacity;
  const double tau_s = p->nu > 0 ? 3.0 * p->nu + 0.5 : p->tau_plus;  // tau_s = nu/c_s^2 + 1/2
  const double tau_a = 0.5 + p->magic_lambda / (tau_s - 0.5);         // Lambda = (tau_s-1/2)(tau_a-1/2)
  D.omega_p = 1.0 / tau_s;
  D.omega_m = 1.0 / tau_a;
  D.inv_2eta1 = 1.0 / (2.0 * p->eta + 1.0);
  D.rho0 = p->rho0;
  {
    // inlet ghost populations f^eq(rho0, u_in), Eq. (feq), in compute space
    const int ex[kQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, ey[kQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const double w[kQ] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    const double ux = p->u_in_x, uy = p->u_in_y, usq = ux * ux + uy * uy;
    const bool shift = p->storage == LBM_F16S || p->storage == LBM_BF16S;
    for (int a = 0; a < kQ; ++a) {
      const double eu = ex[a] * ux + ey[a] * uy;
      const double dev = p->rho0 * w[a] * (3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
      D.ghost[a] = shift ? dev : p->rho0 * w[a] + dev;
    }
  }
  fill_cell_const(D, p->storage);
  return LBM_OK;
}

lbm_status admit(lbm_batch *b, const lbm_params *p, const uint8_t *mask_host,
                 const lbm_geometry *geom, const lbm_body *bodies, int nbodies, long long nsteps,
                 int *slot_out) {
  lbm_status rc = validate(p, nbodies);
  if (rc != LBM_OK) return rc;
  if (p->storage != b->storage) return fail(LBM_EINVAL, "domain storage %d differs from batch storage %d", p->storage, b->storage);
  if (nbodies > 0 && !bodies) return fail(LBM_EINVAL, "bodies is NULL");
  if (!mask_host && geom && geom->nshapes > 0 && !geom->shapes) return fail(LBM_EINVAL, "geometry shapes NULL");
  if (nsteps < 0) return fail(LBM_EINVAL, "nsteps must be >= 0");
  if (p->moving) {
    if (mask_host) return fail(LBM_EINVAL, "a moving domain is rasterised from its geometry (mask given)");
    if (!geom || geom->nshapes < 1 || geom->nshapes > kMaxMovingShapes)
      return fail(LBM_EINVAL, "a moving domain needs 1..%d shapes", kMaxMovingShapes);
  }
  int k = -1;
  for (int i = 0; i < b->max_domains; ++i)
    if (!b->slots[i].used) { k = i; break; }
  if (k < 0) return fail(LBM_EBUSY, "no free slot");
  const Layout L = layout_of(*p, nbodies);
  if (b->budget > 0 && b->bytes_in_use + L.total > b->budget)
    return fail(LBM_EBUSY, "memory budget exceeded (%zu + %zu > %zu)", b->bytes_in_use, L.total, b->budget);
  if (geom && !mask_host)
    for (int i = 0; i < geom->nshapes; ++i) {
      const lbm_shape &sh = geom->shapes[i];
      if (sh.kind < 0 || sh.kind > LBM_SHAPE_NACA4) return fail(LBM_EINVAL, "shape %d: unknown kind", i);
      if (sh.body < 1 || sh.body > nbodies) return fail(LBM_EINVAL, "shape %d: body id %d not in [1, %d]", i, sh.body, nbodies);
      if (sh.kind == LBM_SHAPE_NACA4 && !(sh.chord > 0)) return fail(LBM_EINVAL, "shape %d: chord must be > 0", i);
    }

  Slot s;
  {
    lbm_status prc = prepare_slot(b, p, geom, nbodies, nsteps, L, s);
    if (prc != LBM_OK) return prc;
  }
  char *base = static_cast<char *>(s.block);
  DomDev &D = s.dev;
  uint8_t *mask = D.mask;
  double *bod = D.bodies;
  float *bodf = D.bodies_f;
  int32_t *off = const_cast<int32_t *>(D.solid_off);
  cudaStream_t st = b->st;
  void *tmp = nullptr;  // admission temporaries (row counts, offsets, shapes)
  auto bail = [&](lbm_status r) {
    cudaStreamSynchronize(st);
    b->al.put(s.block);
    b->al.put(s.solid);
    b->al.put(tmp);
    return r;
  };
#define ADM_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return bail(fail(LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)));      \
  } while (0)

  // mask: uploaded (pitched, zero padding) or rasterised on the device
  ADM_CUDA(cudaMemsetAsync(mask, 0, static_cast<size_t>(p->ny) * s.pitch, st));
  std::vector<ShapeDev> shapes;
  // temporary: per-row counts [nbodies+1][ny], bad-id word, row offsets [nbodies][ny], shapes
  const size_t counts_n = static_cast<size_t>(nbodies + 1) * p->ny;
  const size_t counts_bytes = align_up(sizeof(int32_t) * (counts_n + 1), 256);
  const size_t offs_bytes = align_up(sizeof(int32_t) * std::max<size_t>(1, static_cast<size_t>(nbodies) * p->ny), 256);
  const int ns = (!mask_host && geom) ? geom->nshapes : 0;
  tmp = b->al.get(counts_bytes + offs_bytes + sizeof(ShapeDev) * std::max(1, ns));
  if (!tmp) return bail(fail(LBM_ENOMEM, "temporary allocation failed"));
  int32_t *counts = static_cast<int32_t *>(tmp);
  int32_t *bad = counts + counts_n;
  int32_t *row_off = reinterpret_cast<int32_t *>(static_cast<char *>(tmp) + counts_bytes);
  if (mask_host) {
    ADM_CUDA(cudaMemcpy2DAsync(mask, s.pitch, mask_host, p->nx, p->nx, p->ny, cudaMemcpyHostToDevice, st));
  } else if (ns > 0) {
    for (int i = 0; i < ns; ++i) {
      const lbm_shape &sh = geom->shapes[i];
      ShapeDev d{sh.kind, sh.body, sh.cx, sh.cy, sh.radius, sh.chord, sh.thickness,
                 std::cos(sh.aoa_rad), std::sin(sh.aoa_rad)};
      shapes.push_back(d);
    }
    ShapeDev *dsh = p->moving ? const_cast<ShapeDev *>(D.shapes)
                              : reinterpret_cast<ShapeDev *>(static_cast<char *>(tmp) + counts_bytes + offs_bytes);
    ADM_CUDA(cudaMemcpyAsync(dsh, shapes.data(), sizeof(ShapeDev) * ns, cudaMemcpyHostToDevice, st));
    std::vector<float4> shapes_f;
    if (p->moving) {
      for (const ShapeDev &d : shapes)
        shapes_f.push_back(make_float4(static_cast<float>(d.cx), static_cast<float>(d.cy),
                                       static_cast<float>(shape_extent(d)), 0.f));
      ADM_CUDA(cudaMemcpyAsync(const_cast<float4 *>(D.shapes_f), shapes_f.data(), sizeof(float4) * ns,
                               cudaMemcpyHostToDevice, st));
    }
    // a moving domain is placed at its step index below, once its body table is resident
    if (!p->moving) ADM_CUDA(launch_rasterize(st, mask, p->nx, p->ny, s.pitch, dsh, ns, p->x_origin));
  }
  // body table
  std::vector<double> hb(5 * std::max(1, nbodies), 0.0);
  for (int i = 0; i < nbodies; ++i) {
    hb[5 * i + 0] = bodies[i].cx;
    hb[5 * i + 1] = bodies[i].cy;
    hb[5 * i + 2] = bodies[i].vx;
    hb[5 * i + 3] = bodies[i].vy;
    hb[5 * i + 4] = bodies[i].omega;
  }
  ADM_CUDA(cudaMemcpyAsync(bod, hb.data(), sizeof(double) * hb.size(), cudaMemcpyHostToDevice, st));
  std::vector<float> hbf(hb.begin(), hb.end());
  ADM_CUDA(cudaMemcpyAsync(bodf, hbf.data(), sizeof(float) * hbf.size(), cudaMemcpyHostToDevice, st));
  ADM_CUDA(cudaMemsetAsync(base + L.kappa_off, 0,
                           align_up(sizeof(double) * std::max(1, nbodies), 256) + sizeof(float) * std::max(1, nbodies), st));
  if (p->moving) {
    // reference centres, then the mask and centres of step index 0
    std::vector<double> hc0(2 * std::max(1, nbodies), 0.0);
    for (int i = 0; i < nbodies; ++i) {
      hc0[2 * i] = bodies[i].cx;
      hc0[2 * i + 1] = bodies[i].cy;
    }
    ADM_CUDA(cudaMemcpyAsync(const_cast<double *>(D.centre0), hc0.data(), sizeof(double) * hc0.size(),
                             cudaMemcpyHostToDevice, st));
    // per-row force sums start untagged (all-ones bytes: a NaN tag equals no step)
    ADM_CUDA(cudaMemsetAsync(D.rowsum[0], 0xff, 2 * sizeof(double) * 3 * std::max(1, nbodies) * static_cast<size_t>(p->ny), st));
    ADM_CUDA(cudaMemsetAsync(D.fsi, 0, sizeof(double) * 20 * std::max(1, nbodies), st));
    ADM_CUDA(cudaMemsetAsync(const_cast<double *>(D.dpar), 0, sizeof(double) * 8 * std::max(1, nbodies), st));
    ADM_CUDA(cudaMemcpyAsync(b->d_doms + k, &D, sizeof(DomDev), cudaMemcpyHostToDevice, st));
    ADM_CUDA(launch_place(st, b->d_doms + k, p->nx, p->ny, s.pitch, 0));
  }
  // per-row node counts of every body id, then the row offsets of each body's nodes
  ADM_CUDA(cudaMemsetAsync(bad, 0, sizeof(int32_t), st));
  ADM_CUDA(launch_row_counts(st, mask, p->nx, p->ny, s.pitch, nbodies, counts, bad));
  std::vector<int32_t> hc(counts_n + 1, 0);
  ADM_CUDA(cudaMemcpyAsync(hc.data(), counts, sizeof(int32_t) * (counts_n + 1), cudaMemcpyDeviceToHost, st));
  ADM_CUDA(cudaStreamSynchronize(st));
  if (hc[counts_n] > 0)
    return bail(fail(LBM_EINVAL, "mask holds body id %d but only %d bodies were given", hc[counts_n], nbodies));
  std::vector<int32_t> ho(nbodies + 1, 0), hro(std::max<size_t>(1, static_cast<size_t>(nbodies) * p->ny), 0);
  {
    int32_t acc = 0;
    for (int k = 1; k <= nbodies; ++k) {
      ho[k - 1] = acc;
      for (int j = 0; j < p->ny; ++j) {
        hro[static_cast<size_t>(k - 1) * p->ny + j] = acc;
        acc += hc[static_cast<size_t>(k) * p->ny + j];
      }
    }
    ho[nbodies] = acc;
  }
  const size_t nsolid = static_cast<size_t>(ho[nbodies]);
  s.solid = b->al.get(sizeof(int32_t) * std::max<size_t>(1, nsolid));
  if (!s.solid) return bail(fail(LBM_ENOMEM, "solid list allocation failed"));
  D.solid = static_cast<const int32_t *>(s.solid);
  ADM_CUDA(cudaMemcpyAsync(off, ho.data(), sizeof(int32_t) * ho.size(), cudaMemcpyHostToDevice, st));
  s.solid_off = ho;
  if (nbodies > 0)
    ADM_CUDA(cudaMemcpyAsync(row_off, hro.data(), sizeof(int32_t) * hro.size(), cudaMemcpyHostToDevice, st));
  ADM_CUDA(launch_row_scatter(st, mask, p->nx, p->ny, s.pitch, nbodies, row_off, static_cast<int32_t *>(s.solid)));
  // initial state (step (1)): lattice A = f^eq(rho0, u0), lattice B zero
  ADM_CUDA(launch_init(p->storage, st, D.lat[0], p->nx, p->ny, s.pitch, p->rho0, p->u0_x, p->u0_y));
  ADM_CUDA(cudaMemsetAsync(D.lat[1], 0, L.lat_bytes, st));
  ADM_CUDA(cudaMemsetAsync(D.status, 0, sizeof(int32_t), st));
  ADM_CUDA(cudaMemsetAsync(D.fvp[0], 0, L.bodies_off - L.fvp_off, st));
  if (p->force_every > 0)
    ADM_CUDA(cudaMemsetAsync(D.ring, 0, sizeof(double) * 2 * std::max(1, nbodies) * s.p.force_capacity, st));
  ADM_CUDA(cudaMemcpyAsync(b->d_doms + k, &D, sizeof(DomDev), cudaMemcpyHostToDevice, st));
  ADM_CUDA(cudaStreamSynchronize(st));
  b->al.put(tmp);
  tmp = nullptr;
#undef ADM_CUDA
  s.used = true;
  s.bytes = L.total + sizeof(int32_t) * std::max<size_t>(1, nsolid);
  b->bytes_in_use += s.bytes;
  b->slots[k] = s;
  b->dirty = true;
  *slot_out = k;
  return LBM_OK;
}

// Many fixed-geometry domains at once: the work of admit() for every domain, batched
// into a few launches over the rows of all of them, one upload of host tables, one
// read-back of the per-row counts (the only synchronisation before the solid lists can
// be sized) and a final one. All or none are admitted.
lbm_status admit_many(lbm_batch *b, int n, const lbm_params *ps, const lbm_geometry *geoms,
                      const lbm_body *const *bodies, const int32_t *nbs, const int64_t *nsteps,
                      int32_t *slots_out) {
  if (n < 0) return fail(LBM_EINVAL, "n must be >= 0");
  if (n == 0) return LBM_OK;
  if (!ps || !geoms || !nbs || !nsteps || !slots_out) return fail(LBM_EINVAL, "an argument array is NULL");
  for (int i = 0; i < n; ++i) {
    const lbm_params *p = &ps[i];
    lbm_status rc = validate(p, nbs[i]);
    if (rc != LBM_OK) return fail(rc, "domain %d: %s", i, lbm_last_error());
    if (p->storage != b->storage) return fail(LBM_EINVAL, "domain %d: storage %d differs from batch storage %d", i, p->storage, b->storage);
    if (p->moving) return fail(LBM_EINVAL, "domain %d: moving domains are admitted with lbm_batch_admit", i);
    if (nbs[i] > 0 && (!bodies || !bodies[i])) return fail(LBM_EINVAL, "domain %d: bodies is NULL", i);
    if (nsteps[i] < 0) return fail(LBM_EINVAL, "domain %d: nsteps must be >= 0", i);
    const lbm_geometry &g = geoms[i];
    if (g.nshapes < 0 || (g.nshapes > 0 && !g.shapes)) return fail(LBM_EINVAL, "domain %d: geometry shapes NULL", i);
    for (int q = 0; q < g.nshapes; ++q) {
      const lbm_shape &sh = g.shapes[q];
      if (sh.kind < 0 || sh.kind > LBM_SHAPE_NACA4) return fail(LBM_EINVAL, "domain %d shape %d: unknown kind", i, q);
      if (sh.body < 1 || sh.body > nbs[i]) return fail(LBM_EINVAL, "domain %d shape %d: body id %d not in [1, %d]", i, q, sh.body, nbs[i]);
      if (sh.kind == LBM_SHAPE_NACA4 && !(sh.chord > 0)) return fail(LBM_EINVAL, "domain %d shape %d: chord must be > 0", i, q);
    }
  }
  std::vector<int> ks;
  for (int k = 0; k < b->max_domains && static_cast<int>(ks.size()) < n; ++k)
    if (!b->slots[k].used) ks.push_back(k);
  if (static_cast<int>(ks.size()) < n) return fail(LBM_EBUSY, "%d free slots for %d domains", static_cast<int>(ks.size()), n);
  std::vector<Layout> Ls(n);
  size_t need = 0;
  for (int i = 0; i < n; ++i) {
    Ls[i] = layout_of(ps[i], nbs[i]);
    need += Ls[i].total;
  }
  if (b->budget > 0 && b->bytes_in_use + need > b->budget)
    return fail(LBM_EBUSY, "memory budget exceeded (%zu + %zu > %zu)", b->bytes_in_use, need, b->budget);

  cudaStream_t st = b->st;
  std::vector<Slot> S(n);
  void *tmp = nullptr;
  // Two or more domains share one allocation for their blocks and one for their solid
  // lists (two allocator calls instead of two per domain; the group's memory returns when
  // its last domain leaves).
  const bool grouped = n > 1 && b->group_admit;
  void *gblock = nullptr, *gsolid = nullptr;
  auto release = [&](lbm_status r) {
    cudaStreamSynchronize(st);
    if (grouped) {
      b->al.put(gblock);
      b->al.put(gsolid);
    } else {
      for (Slot &x : S) {
        b->al.put(x.block);
        b->al.put(x.solid);
      }
    }
    b->al.put(tmp);
    return r;
  };
  std::vector<size_t> boff(n, 0);
  if (grouped) {
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
      boff[i] = total;
      total += align_up(Ls[i].total, 256);
    }
    gblock = b->al.get(total);
    if (!gblock) return fail(LBM_ENOMEM, "device allocation of %zu bytes failed", total);
  }
  for (int i = 0; i < n; ++i) {
    lbm_status rc = prepare_slot(b, &ps[i], &geoms[i], nbs[i], nsteps[i], Ls[i], S[i],
                                 grouped ? static_cast<char *>(gblock) + boff[i] : nullptr);
    if (rc != LBM_OK) return release(rc);
  }

  // device temporaries, packed: descriptors, per-row counts, row offsets, shapes, body
  // tables and solid offsets (staged for copying into each domain's block), fill spans
  size_t rows = 0, counts_n = 0, offs_n = 0, nsh = 0, nbt = 0, nso = 0;
  for (int i = 0; i < n; ++i) {
    rows += ps[i].ny;
    counts_n += static_cast<size_t>(nbs[i] + 1) * ps[i].ny;
    offs_n += static_cast<size_t>(nbs[i]) * ps[i].ny;
    nsh += geoms[i].nshapes;
    nbt += 5 * static_cast<size_t>(std::max(1, nbs[i]));
    nso += static_cast<size_t>(nbs[i]) + 1;
  }
  int nrings = 0;
  for (int i = 0; i < n; ++i) nrings += ps[i].force_every > 0 ? 1 : 0;
  const int nseg1 = 4 * n + nrings, nseg2 = 2 * n;  // fills before and after the counts are known
  const size_t o_ad = 0;
  const size_t o_cnt = align_up(o_ad + sizeof(AdmitDev) * n, 256);
  const size_t o_ro = align_up(o_cnt + sizeof(int32_t) * counts_n, 256);
  const size_t o_sh = align_up(o_ro + sizeof(int32_t) * std::max<size_t>(1, offs_n), 256);
  const size_t o_bd = align_up(o_sh + sizeof(ShapeDev) * std::max<size_t>(1, nsh), 256);
  const size_t o_bf = align_up(o_bd + sizeof(double) * nbt, 256);
  const size_t o_so = align_up(o_bf + sizeof(float) * nbt, 256);
  const size_t o_dd = align_up(o_so + sizeof(int32_t) * nso, 256);
  const size_t o_s1 = align_up(o_dd + sizeof(DomDev) * n, 256);
  const size_t o_s2 = align_up(o_s1 + sizeof(FillSeg) * nseg1, 256);
  const size_t tmp_bytes = o_s2 + sizeof(FillSeg) * nseg2;
  tmp = b->al.get(tmp_bytes);
  if (!tmp) return release(fail(LBM_ENOMEM, "temporary allocation of %zu bytes failed", tmp_bytes));
  char *t = static_cast<char *>(tmp);
  std::vector<AdmitDev> ad(n);
  std::vector<ShapeDev> shapes;
  std::vector<double> hb;
  std::vector<float> hbf;
  std::vector<FillSeg> seg1;
  seg1.reserve(nseg1);
  shapes.reserve(nsh);
  hb.reserve(nbt);
  hbf.reserve(nbt);
  size_t r0 = 0, c0 = 0, s0 = 0;
  for (int i = 0; i < n; ++i) {
    const lbm_params &p = ps[i];
    Slot &x = S[i];
    DomDev &D = x.dev;
    AdmitDev &A = ad[i];
    A.mask = D.mask;
    A.lat[0] = D.lat[0];
    A.lat[1] = D.lat[1];
    A.counts = reinterpret_cast<int32_t *>(t + o_cnt) + c0;
    A.row_off = nullptr;
    A.solid = nullptr;
    A.shapes = reinterpret_cast<const ShapeDev *>(t + o_sh) + s0;
    A.nshapes = geoms[i].nshapes;
    A.nx = p.nx;
    A.ny = p.ny;
    A.pitch = x.pitch;
    A.nbodies = nbs[i];
    A.x0 = p.x_origin;
    A.row0 = static_cast<int32_t>(r0);
    A.bad = 0;
    A.rho0 = p.rho0;
    A.u0x = p.u0_x;
    A.u0y = p.u0_y;
    for (int q = 0; q < geoms[i].nshapes; ++q) {
      const lbm_shape &sh = geoms[i].shapes[q];
      shapes.push_back(ShapeDev{sh.kind, sh.body, sh.cx, sh.cy, sh.radius, sh.chord, sh.thickness,
                                std::cos(sh.aoa_rad), std::sin(sh.aoa_rad)});
    }
    const size_t bt0 = hb.size();
    for (int q = 0; q < std::max(1, nbs[i]); ++q) {
      const bool real = q < nbs[i];
      const double v[5] = {real ? bodies[i][q].cx : 0.0, real ? bodies[i][q].cy : 0.0,
                           real ? bodies[i][q].vx : 0.0, real ? bodies[i][q].vy : 0.0,
                           real ? bodies[i][q].omega : 0.0};
      for (double e : v) {
        hb.push_back(e);
        hbf.push_back(static_cast<float>(e));
      }
    }
    const size_t bt = hb.size() - bt0;
    const Layout &L = Ls[i];
    char *base = static_cast<char *>(x.block);
    seg1.push_back(FillSeg{D.bodies, t + o_bd + sizeof(double) * bt0, sizeof(double) * bt});
    seg1.push_back(FillSeg{D.bodies_f, t + o_bf + sizeof(float) * bt0, sizeof(float) * bt});
    // dilation rates (zero: no body pulsates), status word, force ring (the F_VP fields
    // are not cleared: a sweep writes F_VP of every solid node before the force
    // reduction of its step reads it, and nothing reads it elsewhere)
    seg1.push_back(FillSeg{base + L.kappa_off, nullptr,
                           align_up(sizeof(double) * std::max(1, nbs[i]), 256) + sizeof(float) * std::max(1, nbs[i])});
    seg1.push_back(FillSeg{D.status, nullptr, sizeof(int32_t)});
    r0 += p.ny;
    c0 += static_cast<size_t>(nbs[i] + 1) * p.ny;
    s0 += geoms[i].nshapes;
  }
  // force rings (of the domains that record forces)
  for (int i = 0; i < n; ++i)
    if (ps[i].force_every > 0)
      seg1.push_back(FillSeg{S[i].dev.ring, nullptr,
                             sizeof(double) * 2 * std::max(1, nbs[i]) * S[i].p.force_capacity});
  FillSeg *d_fill1 = reinterpret_cast<FillSeg *>(t + o_s1);
#define ADM_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return release(fail(LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)));  \
  } while (0)
  ADM_CUDA(cudaMemcpyAsync(t + o_ad, ad.data(), sizeof(AdmitDev) * n, cudaMemcpyHostToDevice, st));
  if (!shapes.empty())
    ADM_CUDA(cudaMemcpyAsync(t + o_sh, shapes.data(), sizeof(ShapeDev) * shapes.size(), cudaMemcpyHostToDevice, st));
  ADM_CUDA(cudaMemcpyAsync(t + o_bd, hb.data(), sizeof(double) * hb.size(), cudaMemcpyHostToDevice, st));
  ADM_CUDA(cudaMemcpyAsync(t + o_bf, hbf.data(), sizeof(float) * hbf.size(), cudaMemcpyHostToDevice, st));
  ADM_CUDA(cudaMemcpyAsync(d_fill1, seg1.data(), sizeof(FillSeg) * seg1.size(), cudaMemcpyHostToDevice, st));
  AdmitDev *d_ad = reinterpret_cast<AdmitDev *>(t + o_ad);
  ADM_CUDA(launch_fill(st, d_fill1, static_cast<int>(seg1.size())));
  ADM_CUDA(launch_admit_raster_count(st, d_ad, n, static_cast<int>(rows)));
  // per-row counts and unknown body ids back to the host: the one synchronisation needed
  // (on an event before the initial state, which runs while the host sizes the lists)
  std::vector<int32_t> hc(counts_n);
  ADM_CUDA(cudaMemcpyAsync(hc.data(), t + o_cnt, sizeof(int32_t) * counts_n, cudaMemcpyDeviceToHost, st));
  ADM_CUDA(cudaMemcpyAsync(ad.data(), d_ad, sizeof(AdmitDev) * n, cudaMemcpyDeviceToHost, st));
  ADM_CUDA(cudaEventRecord(b->adm_ev, st));
  ADM_CUDA(launch_admit_init(b->storage, st, d_ad, n, static_cast<int>(rows)));
  ADM_CUDA(cudaEventSynchronize(b->adm_ev));
  for (int i = 0; i < n; ++i)
    if (ad[i].bad > 0)
      return release(fail(LBM_EINVAL, "domain %d: mask holds body id %d but only %d bodies were given", i, ad[i].bad, nbs[i]));
  // solid-node offsets per body and per (body, row); the solid lists
  std::vector<int32_t> hro(std::max<size_t>(1, offs_n), 0), hso;
  hso.reserve(nso);
  std::vector<size_t> nsolid(n);
  {
    size_t cc = 0, oo = 0;
    for (int i = 0; i < n; ++i) {
      const int ny = ps[i].ny, nb = nbs[i];
      int32_t acc = 0;
      std::vector<int32_t> ho(nb + 1, 0);
      for (int q = 1; q <= nb; ++q) {
        ho[q - 1] = acc;
        for (int j = 0; j < ny; ++j) {
          hro[oo + static_cast<size_t>(q - 1) * ny + j] = acc;
          acc += hc[cc + static_cast<size_t>(q) * ny + j];
        }
      }
      ho[nb] = acc;
      hso.insert(hso.end(), ho.begin(), ho.end());
      S[i].solid_off = ho;
      nsolid[i] = static_cast<size_t>(acc);
      ad[i].row_off = reinterpret_cast<const int32_t *>(t + o_ro) + oo;
      cc += static_cast<size_t>(nb + 1) * ny;
      oo += static_cast<size_t>(nb) * ny;
    }
  }
  if (grouped) {
    std::vector<size_t> soff(n);
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
      soff[i] = total;
      total += align_up(sizeof(int32_t) * std::max<size_t>(1, nsolid[i]), 256);
    }
    gsolid = b->al.get(total);
    if (!gsolid) return release(fail(LBM_ENOMEM, "solid list allocation failed"));
    for (int i = 0; i < n; ++i) S[i].solid = static_cast<char *>(gsolid) + soff[i];
  } else {
    for (int i = 0; i < n; ++i) {
      S[i].solid = b->al.get(sizeof(int32_t) * std::max<size_t>(1, nsolid[i]));
      if (!S[i].solid) return release(fail(LBM_ENOMEM, "solid list allocation failed"));
    }
  }
  for (int i = 0; i < n; ++i) {
    S[i].dev.solid = static_cast<const int32_t *>(S[i].solid);
    ad[i].solid = static_cast<int32_t *>(S[i].solid);
  }
  // second upload: row offsets, descriptors with the solid lists, per-domain solid
  // offsets and the domains' device descriptions, copied into place by one fill launch
  std::vector<DomDev> dd(n);
  std::vector<FillSeg> seg2;
  {
    size_t so = 0;
    for (int i = 0; i < n; ++i) {
      dd[i] = S[i].dev;
      seg2.push_back(FillSeg{const_cast<int32_t *>(S[i].dev.solid_off), t + o_so + sizeof(int32_t) * so,
                             sizeof(int32_t) * (nbs[i] + 1)});
      seg2.push_back(FillSeg{b->d_doms + ks[i], t + o_dd + sizeof(DomDev) * i, sizeof(DomDev)});
      so += static_cast<size_t>(nbs[i]) + 1;
    }
  }
  if (offs_n > 0)
    ADM_CUDA(cudaMemcpyAsync(t + o_ro, hro.data(), sizeof(int32_t) * offs_n, cudaMemcpyHostToDevice, st));
  ADM_CUDA(cudaMemcpyAsync(d_ad, ad.data(), sizeof(AdmitDev) * n, cudaMemcpyHostToDevice, st));
  ADM_CUDA(cudaMemcpyAsync(t + o_so, hso.data(), sizeof(int32_t) * hso.size(), cudaMemcpyHostToDevice, st));
  ADM_CUDA(cudaMemcpyAsync(t + o_dd, dd.data(), sizeof(DomDev) * n, cudaMemcpyHostToDevice, st));
  ADM_CUDA(cudaMemcpyAsync(t + o_s2, seg2.data(), sizeof(FillSeg) * seg2.size(), cudaMemcpyHostToDevice, st));
  int max_nb = 0;
  for (int i = 0; i < n; ++i) max_nb = std::max(max_nb, nbs[i]);
  ADM_CUDA(launch_admit_scatter(st, d_ad, n, static_cast<int>(rows), max_nb));
  ADM_CUDA(launch_fill(st, reinterpret_cast<const FillSeg *>(t + o_s2), static_cast<int>(seg2.size())));
  ADM_CUDA(cudaStreamSynchronize(st));
#undef ADM_CUDA
  b->al.put(tmp);
  tmp = nullptr;
  int g = -1;
  if (grouped) {
    for (size_t q = 0; q < b->groups.size() && g < 0; ++q)
      if (b->groups[q].members == 0) g = static_cast<int>(q);
    if (g < 0) {
      g = static_cast<int>(b->groups.size());
      b->groups.emplace_back();
    }
    b->groups[g] = Group{gblock, gsolid, n, 0};
  }
  for (int i = 0; i < n; ++i) {
    Slot &x = S[i];
    x.used = true;
    x.group = g;
    x.bytes = Ls[i].total + sizeof(int32_t) * std::max<size_t>(1, nsolid[i]);
    b->bytes_in_use += x.bytes;
    if (g >= 0) b->groups[g].bytes += x.bytes;
    b->slots[ks[i]] = x;
    slots_out[i] = ks[i];
  }
  b->dirty = true;
  return LBM_OK;
}

// Return a slot's device memory: its own two allocations, or its share of a batched
// admission's, which go back (and leave the memory budget) with the group's last domain.
void release_memory(lbm_batch *b, Slot &s) {
  if (s.group >= 0) {
    Group &g = b->groups[s.group];
    if (--g.members == 0) {
      b->al.put(g.block);
      b->al.put(g.solid);
      b->bytes_in_use -= g.bytes;
      g = Group();
    }
  } else {
    b->al.put(s.block);
    b->al.put(s.solid);
    b->bytes_in_use -= s.bytes;
  }
}

lbm_status check_slot(lbm_batch *b, int slot) {
  if (!b) return fail(LBM_EINVAL, "batch is NULL");
  if (slot < 0 || slot >= b->max_domains || !b->slots[slot].used)
    return fail(LBM_ENOTFOUND, "slot %d is not resident", slot);
  return LBM_OK;
}

lbm_status poll(lbm_batch *b, int slot, double *out, long long max_entries, long long *written,
                int *done) {
  if (written) *written = 0;
  if (done) *done = 0;
  lbm_status rc = check_slot(b, slot);
  if (rc != LBM_OK) return rc;
  Slot &s = b->slots[slot];
  int status = 0;
  rc = read_status(b, s, &status);
  if (rc != LBM_OK) return rc;
  const long long produced = entries_at(s, s.done);
  long long n = std::min(produced - s.drained, std::max(0ll, max_entries));
  if (n > 0 && !out) return fail(LBM_EINVAL, "out is NULL");
  const size_t per = 2 * static_cast<size_t>(s.nbodies);
  long long copied = 0;
  while (copied < n && per > 0) {
    const long long e = s.drained + copied;
    const long long pos = e % s.dev.force_cap;
    const long long chunk = std::min(n - copied, static_cast<long long>(s.dev.force_cap) - pos);
    LBM_CUDA(cudaMemcpyAsync(out + copied * per, s.dev.ring + pos * per, sizeof(double) * per * chunk,
                             cudaMemcpyDeviceToHost, b->st));
    copied += chunk;
  }
  LBM_CUDA(cudaStreamSynchronize(b->st));
  s.drained += n;
  if (written) *written = n;
  if (done) *done = (s.done >= s.target && s.drained >= produced) ? 1 : 0;
  if (status & 2) return fail(LBM_ETIMEOUT, "slot %d: a sweep gave up waiting for its row copies", slot);
  if (status & 1) return fail(LBM_EUNSTABLE, "slot %d diverged (rho out of range or not finite)", slot);
  return LBM_OK;
}

// Many slots' new force entries and status words, staged in pinned host memory by
// asynchronous copies and read after one synchronisation.
lbm_status poll_many(lbm_batch *b, int n, const int32_t *slots, double *const *outs,
                     const int64_t *max_entries, int64_t *written, int32_t *done, int32_t *status) {
  if (n < 0) return fail(LBM_EINVAL, "n must be >= 0");
  if (n == 0) return LBM_OK;
  if (!slots || !outs || !max_entries || !written || !done || !status)
    return fail(LBM_EINVAL, "an argument array is NULL");
  std::vector<long long> cnt(n);
  std::vector<size_t> at(n);
  size_t bytes = align_up(sizeof(int32_t) * n, 16), nspan = 0;
  for (int i = 0; i < n; ++i) {
    lbm_status rc = check_slot(b, slots[i]);
    if (rc != LBM_OK) return rc;
    const Slot &s = b->slots[slots[i]];
    cnt[i] = std::min(entries_at(s, s.done) - s.drained, std::max<long long>(0, max_entries[i]));
    if (cnt[i] > 0 && !outs[i]) return fail(LBM_EINVAL, "outs[%d] is NULL", i);
    at[i] = bytes;
    bytes += sizeof(double) * 2 * static_cast<size_t>(s.nbodies) * static_cast<size_t>(std::max(0ll, cnt[i]));
    // copy spans of this slot: its status word and the ring entries up to each wrap
    nspan += 1;
    if (s.nbodies > 0)
      for (long long c = 0; c < cnt[i];) {
        c += std::min(cnt[i] - c, static_cast<long long>(s.dev.force_cap) - (s.drained + c) % s.dev.force_cap);
        nspan += 1;
      }
  }
  // From four slots on, the status words and ring entries are gathered into device
  // staging by one copy launch and read back by one transfer (two copies per slot cost
  // more host time); the copy descriptors follow the results in both staging buffers.
  const bool gather = n >= 4;
  const size_t seg_at = align_up(bytes, 16);
  const size_t need = gather ? seg_at + sizeof(FillSeg) * nspan : bytes;
  if (need > b->h_poll_cap) {
    if (b->h_poll && b->h_poll_own) cudaFreeHost(b->h_poll);
    b->h_poll = nullptr;
    b->h_poll_cap = 0;
    const size_t cap = std::max<size_t>(need * 2, 1 << 16);
    if (cudaMallocHost(&b->h_poll, cap) != cudaSuccess) {
      cudaGetLastError();
      b->h_poll = nullptr;
      return fail(LBM_ENOMEM, "pinned staging of %zu bytes failed", cap);
    }
    b->h_poll_cap = cap;
    b->h_poll_own = true;
  }
  if (gather && need > b->d_poll_cap) {
    b->al.put(b->d_poll);
    b->d_poll_cap = 0;
    const size_t cap = std::max<size_t>(need * 2, 1 << 16);
    b->d_poll = static_cast<char *>(b->al.get(cap));
    if (!b->d_poll) return fail(LBM_ENOMEM, "device staging of %zu bytes failed", cap);
    b->d_poll_cap = cap;
  }
  int32_t *st_words = reinterpret_cast<int32_t *>(b->h_poll);
  FillSeg *segs = reinterpret_cast<FillSeg *>(b->h_poll + seg_at);
  int nseg = 0;
  // one span from the device to the results at offset `off`
  auto take = [&](size_t off, const void *src, size_t len) -> cudaError_t {
    if (gather) {
      segs[nseg++] = FillSeg{b->d_poll + off, src, len};
      return cudaSuccess;
    }
    return cudaMemcpyAsync(b->h_poll + off, src, len, cudaMemcpyDeviceToHost, b->st);
  };
  for (int i = 0; i < n; ++i) {
    const Slot &s = b->slots[slots[i]];
    LBM_CUDA(take(sizeof(int32_t) * i, s.dev.status, sizeof(int32_t)));
    const size_t per = 2 * static_cast<size_t>(s.nbodies);
    long long copied = 0;
    while (copied < cnt[i] && per > 0) {
      const long long e = s.drained + copied;
      const long long pos = e % s.dev.force_cap;
      const long long chunk = std::min(cnt[i] - copied, static_cast<long long>(s.dev.force_cap) - pos);
      LBM_CUDA(take(at[i] + sizeof(double) * copied * per, s.dev.ring + pos * per, sizeof(double) * per * chunk));
      copied += chunk;
    }
  }
  if (gather) {
    FillSeg *d_segs = reinterpret_cast<FillSeg *>(b->d_poll + seg_at);
    LBM_CUDA(cudaMemcpyAsync(d_segs, segs, sizeof(FillSeg) * nseg, cudaMemcpyHostToDevice, b->st));
    LBM_CUDA(launch_fill(b->st, d_segs, nseg));
    b->launches++;
    LBM_CUDA(cudaMemcpyAsync(b->h_poll, b->d_poll, bytes, cudaMemcpyDeviceToHost, b->st));
  }
  LBM_CUDA(cudaStreamSynchronize(b->st));
  for (int i = 0; i < n; ++i) {
    Slot &s = b->slots[slots[i]];
    const size_t per = 2 * static_cast<size_t>(s.nbodies);
    if (cnt[i] > 0 && per > 0) std::memcpy(outs[i], b->h_poll + at[i], sizeof(double) * per * cnt[i]);
    s.drained += std::max(0ll, cnt[i]);
    written[i] = std::max(0ll, cnt[i]);
    done[i] = (s.done >= s.target && s.drained >= entries_at(s, s.done)) ? 1 : 0;
    const int w = st_words[i];
    status[i] = (w & 2) ? LBM_ETIMEOUT : ((w & 1) ? LBM_EUNSTABLE : LBM_OK);
  }
  return LBM_OK;
}

lbm_status moments(lbm_batch *b, int slot, double *rho, double *ux, double *uy) {
  lbm_status rc = check_slot(b, slot);
  if (rc != LBM_OK) return rc;
  Slot &s = b->slots[slot];
  const size_t cells = static_cast<size_t>(s.p.nx) * s.p.ny;
  double *tmp = static_cast<double *>(b->al.get(sizeof(double) * 3 * cells));
  if (!tmp) return fail(LBM_ENOMEM, "moments buffer allocation failed");
  cudaError_t e = launch_moments_sized(b->storage, b->st, b->d_doms + slot, s.p.nx, s.p.ny, s.parity,
                                       tmp, tmp + cells, tmp + 2 * cells);
  double *outs[3] = {rho, ux, uy};
  for (int q = 0; q < 3 && e == cudaSuccess; ++q)
    if (outs[q]) e = cudaMemcpyAsync(outs[q], tmp + q * cells, sizeof(double) * cells, cudaMemcpyDefault, b->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  b->al.put(tmp);
  if (e != cudaSuccess) return fail(LBM_ECUDA, "moments failed: %s", cudaGetErrorString(e));
  int status = 0;
  rc = read_status(b, s, &status);
  if (rc != LBM_OK) return rc;
  if (status & 2) return fail(LBM_ETIMEOUT, "slot %d: a sweep gave up waiting for its row copies", slot);
  if (status & 1) return fail(LBM_EUNSTABLE, "slot %d diverged", slot);
  return LBM_OK;
}

lbm_status populations(lbm_batch *b, int slot, void *out, const void *in, size_t bytes) {
  lbm_status rc = check_slot(b, slot);
  if (rc != LBM_OK) return rc;
  Slot &s = b->slots[slot];
  const size_t es = elem_size(b->storage);
  const size_t want = es * kQ * s.p.nx * s.p.ny;
  if (bytes != want) return fail(LBM_EINVAL, "population buffer must be %zu bytes (got %zu)", want, bytes);
  char *lat = static_cast<char *>(s.dev.lat[s.parity]);
  const size_t rowb = es * s.p.nx, pitchb = es * s.pitch;
  if (out) {
    LBM_CUDA(cudaMemcpy2DAsync(out, rowb, lat, pitchb, rowb, static_cast<size_t>(kQ) * s.p.ny, cudaMemcpyDefault, b->st));
  } else {
    if (!in) return fail(LBM_EINVAL, "input is NULL");
    LBM_CUDA(cudaMemcpy2DAsync(lat, pitchb, in, rowb, rowb, static_cast<size_t>(kQ) * s.p.ny, cudaMemcpyDefault, b->st));
  }
  LBM_CUDA(cudaStreamSynchronize(b->st));
  return LBM_OK;
}

lbm_status get_mask(lbm_batch *b, int slot, uint8_t *out) {
  lbm_status rc = check_slot(b, slot);
  if (rc != LBM_OK) return rc;
  if (!out) return fail(LBM_EINVAL, "out is NULL");
  const Slot &s = b->slots[slot];
  LBM_CUDA(cudaMemcpy2DAsync(out, s.p.nx, s.dev.mask, s.pitch, s.p.nx, s.p.ny, cudaMemcpyDefault, b->st));
  LBM_CUDA(cudaStreamSynchronize(b->st));
  return LBM_OK;
}

void destroy(lbm_batch *b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  drop_graph(b);
  for (Slot &s : b->slots)
    if (s.used) release_memory(b, s);
  b->al.put(b->d_poll);
  b->al.put(b->d_base);
  b->al.put(b->d_tiles);
  b->al.put(b->d_items);
  b->al.put(b->d_moves);
  b->al.put(b->d_busy);
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->h_pin) cudaFreeHost(b->h_pin);
  if (b->h_poll && b->h_poll_own) cudaFreeHost(b->h_poll);
  if (b->dyn_ev) cudaEventDestroy(b->dyn_ev);
  if (b->st2) {
    cudaStreamSynchronize(b->st2);
    cudaStreamDestroy(b->st2);
  }
  for (cudaEvent_t e : {b->ev_sweep, b->ev_force[0], b->ev_force[1], b->ev_join, b->adm_ev, b->ev_pre, b->ev_tab})
    if (e) cudaEventDestroy(e);
  if (b->own_stream && b->st) cudaStreamDestroy(b->st);
  delete b;
}

lbm_status create(int max_domains, size_t budget, int storage, int graph_steps, void *stream,
                  lbm_alloc_fn alloc, lbm_free_fn free_fn, void *ctx, lbm_batch **out) {
  if (!out) return fail(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_domains < 1 || max_domains > 4096) return fail(LBM_EINVAL, "max_domains must be in [1, 4096]");
  if (elem_size(storage) == 0) return fail(LBM_EINVAL, "unknown storage %d", storage);
  if (graph_steps < 0 || graph_steps > 4096) return fail(LBM_EINVAL, "graph_steps must be in [0, 4096]");
  if ((alloc == nullptr) != (free_fn == nullptr)) return fail(LBM_EINVAL, "alloc and free must both be given or both NULL");
  lbm_batch *b = new (std::nothrow) lbm_batch();
  if (!b) return fail(LBM_ENOMEM, "host allocation failed");
  b->max_domains = max_domains;
  b->budget = budget;
  b->storage = storage;
  b->graph_steps = graph_steps;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete b;
    return fail(LBM_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
  }
  if (stream) {
    b->st = static_cast<cudaStream_t>(stream);
  } else {
    e = cudaStreamCreate(&b->st);
    if (e != cudaSuccess) { delete b; return fail(LBM_ECUDA, "stream creation failed: %s", cudaGetErrorString(e)); }
    b->own_stream = true;
  }
  b->al = Alloc{alloc, free_fn, ctx, b->st};
  b->grid_force = 2 * b->sm_count;
  b->grid_move = 4 * b->sm_count;
  b->slots.resize(max_domains);
  // domain descriptions, dynamic state and counters in one device allocation; their
  // pinned staging and the first poll staging in one pinned block
  const size_t doms_b = align_up(sizeof(DomDev) * max_domains, 256);
  const size_t dyn_b = align_up(sizeof(DomDyn) * max_domains, 256);
  b->d_base = b->al.get(doms_b + dyn_b + sizeof(Counters));
  if (!b->d_base) { destroy(b); return fail(LBM_ENOMEM, "device allocation failed"); }
  b->d_doms = static_cast<DomDev *>(b->d_base);
  b->d_dyn = reinterpret_cast<DomDyn *>(static_cast<char *>(b->d_base) + doms_b);
  b->d_ctr = reinterpret_cast<Counters *>(static_cast<char *>(b->d_base) + doms_b + dyn_b);
  const size_t ctr_b = align_up(sizeof(Counters), 256), poll_b = size_t(1) << 16;
  if (cudaMallocHost(&b->h_pin, dyn_b + ctr_b + poll_b) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->dyn_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    destroy(b);
    return fail(LBM_ENOMEM, "pinned host allocation failed");
  }
  b->h_dyn = reinterpret_cast<DomDyn *>(b->h_pin);
  b->h_ctr = reinterpret_cast<Counters *>(b->h_pin + dyn_b);
  b->h_poll = b->h_pin + dyn_b + ctr_b;
  b->h_poll_cap = poll_b;
  if (cudaStreamCreateWithFlags(&b->st2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_sweep, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_force[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_force[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->adm_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_pre, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_tab, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    destroy(b);
    return fail(LBM_ECUDA, "stream or event creation failed");
  }
  cudaEventRecord(b->dyn_ev, b->st);
  cudaMemsetAsync(b->d_ctr, 0, sizeof(Counters), b->st);
  cudaMemsetAsync(b->d_dyn, 0, sizeof(DomDyn) * max_domains, b->st);
  int vec, warps, rows, pipe;
  default_tile(storage, vec, warps, rows, pipe);
  lbm_status rc = set_config(b, vec, warps, rows, pipe);
  if (rc != LBM_OK) { destroy(b); return rc; }
  *out = b;
  return LBM_OK;
}

lbm_status autotune(lbm_batch *b, int reps, double *best_us) {
  if (reps < 1) return fail(LBM_EINVAL, "reps must be >= 1");
  bool any = false;
  for (const Slot &s : b->slots) any |= s.used;
  if (!any) return fail(LBM_EINVAL, "autotune needs resident domains");
  const int vecs[2] = {b->storage == LBM_F64 ? 1 : (b->storage == LBM_F32 ? 2 : 4),
                       b->storage == LBM_F64 ? 2 : (b->storage == LBM_F32 ? 4 : 8)};
  // warps per block that fit each pipeline: the direct sweep at 16, 20 and 24 resident
  // warps per SM (pipelines 0, 3, 4), the TMA-staged and register-prefetched rows
  const std::vector<int> warp_opts[5] = {{4, 8, 16}, {4, 8, 16}, {4, 8}, {5, 10}, {6, 8, 12}};
  const int row_opts[3] = {1, 2, 4};
  // every resident domain active for the timing launches (s = 0 only: the spare
  // lattice is written, the current state is read and left as it is)
  LBM_CUDA(cudaEventSynchronize(b->dyn_ev));
  for (int k = 0; k < b->max_domains; ++k) {
    const Slot &s = b->slots[k];
    b->h_dyn[k] = DomDyn{s.done, s.used ? s.done + 1 : s.done, s.parity, 0};
  }
  LBM_CUDA(cudaMemcpyAsync(b->d_dyn, b->h_dyn, sizeof(DomDyn) * b->max_domains, cudaMemcpyHostToDevice, b->st));
  LBM_CUDA(cudaEventRecord(b->dyn_ev, b->st));
  cudaEvent_t e0, e1;
  LBM_CUDA(cudaEventCreate(&e0));
  LBM_CUDA(cudaEventCreate(&e1));
  double best = 1e300;
  int bv = b->vec, bw = b->warps, br = b->rows, bp = b->pipe;
  lbm_status rc = LBM_OK;
  for (int p = 0; p < 5 && rc == LBM_OK; ++p)
    for (int v : vecs)
      for (int w : warp_opts[p])
        for (int r : row_opts) {
          if (sweep_occupancy(b->storage, v, p, w) <= 0) continue;
          rc = set_config(b, v, w, r, p);
          if (rc == LBM_OK) rc = rebuild_lists(b);
          if (rc != LBM_OK) break;
          for (int q = 0; q < 2 && rc == LBM_OK; ++q)
            if (sweep_launch(b, b->grid_sweep, v, p, w, r, 0) != cudaSuccess) rc = fail(LBM_ECUDA, "autotune launch failed");
          cudaEventRecord(e0, b->st);
          for (int q = 0; q < reps && rc == LBM_OK; ++q)
            if (sweep_launch(b, b->grid_sweep, v, p, w, r, 0) != cudaSuccess) rc = fail(LBM_ECUDA, "autotune launch failed");
          cudaEventRecord(e1, b->st);
          cudaEventSynchronize(e1);
          if (rc != LBM_OK) break;
          b->launches += reps + 2;
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          const double us = 1000.0 * ms / reps;
          if (us < best) { best = us; bv = v; bw = w; br = r; bp = p; }
        }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != LBM_OK) return rc;
  rc = set_config(b, bv, bw, br, bp);
  if (rc == LBM_OK) rc = rebuild_lists(b);
  if (best_us) *best_us = best;
  return rc;
}

}  // namespace
}  // namespace lbm

namespace lbm {
// Device address of lbm_moments_noalloc's fixed staging array on `dev` (defined below).
lbm_status noalloc_scratch_on(int dev, double **out);
}  // namespace lbm

// ======================================================================================
// C ABI

extern "C" {

void lbm_params_default(lbm_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->nx = 64;
  p->ny = 64;
  p->nu = 0.1;
  p->tau_plus = 0.8;
  p->magic_lambda = 3.0 / 16.0;
  p->eta = 1e-4;
  p->rho0 = 1.0;
  p->west = p->east = p->south = p->north = LBM_PERIODIC;
  p->storage = LBM_F32;
  p->force_every = 1;
  p->force_capacity = 8192;
}

const char *lbm_status_string(lbm_status s) {
  switch (s) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of memory";
    case LBM_ECUDA: return "CUDA error";
    case LBM_EUNSTABLE: return "simulation diverged";
    case LBM_ETIMEOUT: return "timed out";
    case LBM_EBUSY: return "busy";
    case LBM_ENOTFOUND: return "not found";
  }
  return "unknown status";
}

const char *lbm_last_error(void) { return g_last_error.c_str(); }

size_t lbm_domain_bytes(const lbm_params *p, int32_t nbodies) {
  if (!p || elem_size(p->storage) == 0 || p->nx < 1 || p->ny < 1) return 0;
  lbm_params q = *p;
  if (q.force_capacity == 0) q.force_capacity = 8192;
  return layout_of(q, std::max(0, nbodies)).total;
}

lbm_status lbm_batch_create(int32_t max_domains, size_t hbm_budget_bytes, int32_t storage,
                            int32_t graph_steps, void *cuda_stream, lbm_alloc_fn alloc,
                            lbm_free_fn free_fn, void *alloc_ctx, lbm_batch **out) {
  return create(max_domains, hbm_budget_bytes, storage, graph_steps, cuda_stream, alloc, free_fn,
                alloc_ctx, out);
}

lbm_status lbm_batch_admit(lbm_batch *b, const lbm_params *p, const uint8_t *mask,
                           const lbm_geometry *geom, const lbm_body *bodies, int32_t nbodies,
                           int64_t nsteps, int32_t *slot) {
  Range range("lbm_batch_admit");
  if (!b || !slot) return fail(LBM_EINVAL, "batch or slot pointer is NULL");
  int k = -1;
  lbm_status rc = admit(b, p, mask, geom, bodies, nbodies, nsteps, &k);
  if (rc == LBM_OK) *slot = k;
  return rc;
}

lbm_status lbm_batch_admit_many(lbm_batch *b, int32_t n, const lbm_params *params,
                                const lbm_geometry *geoms, const lbm_body *const *bodies,
                                const int32_t *nbodies, const int64_t *nsteps, int32_t *slots) {
  Range range("lbm_batch_admit_many");
  if (!b) return fail(LBM_EINVAL, "batch is NULL");
  return admit_many(b, n, params, geoms, bodies, nbodies, nsteps, slots);
}

lbm_status lbm_batch_run(lbm_batch *b, int64_t max_steps, int64_t *steps_run) {
  Range range("lbm_batch_run");
  if (!b) return fail(LBM_EINVAL, "batch is NULL");
  long long n = 0;
  lbm_status rc = run(b, max_steps, &n);
  if (steps_run) *steps_run = n;
  return rc;
}

lbm_status lbm_batch_poll(lbm_batch *b, int32_t slot, double *out, int64_t max_entries,
                          int64_t *written, int32_t *done) {
  Range range("lbm_batch_poll");
  long long w = 0;
  int d = 0;
  lbm_status rc = poll(b, slot, out, max_entries, &w, &d);
  if (written) *written = w;
  if (done) *done = d;
  return rc;
}

lbm_status lbm_batch_poll_many(lbm_batch *b, int32_t n, const int32_t *slots, double *const *outs,
                               const int64_t *max_entries, int64_t *written, int32_t *done,
                               int32_t *status) {
  Range range("lbm_batch_poll_many");
  if (!b) return fail(LBM_EINVAL, "batch is NULL");
  return poll_many(b, n, slots, outs, max_entries, written, done, status);
}

lbm_status lbm_batch_moments(lbm_batch *b, int32_t slot, double *rho, double *ux, double *uy) {
  Range range("lbm_batch_moments");
  return moments(b, slot, rho, ux, uy);
}

lbm_status lbm_batch_get_populations(lbm_batch *b, int32_t slot, void *out, size_t bytes) {
  if (!out) return fail(LBM_EINVAL, "out is NULL");
  return populations(b, slot, out, nullptr, bytes);
}

lbm_status lbm_batch_set_populations(lbm_batch *b, int32_t slot, const void *in, size_t bytes) {
  return populations(b, slot, nullptr, in, bytes);
}

lbm_status lbm_batch_steps_done(lbm_batch *b, int32_t slot, int64_t *steps) {
  lbm_status rc = check_slot(b, slot);
  if (rc != LBM_OK) return rc;
  if (steps) *steps = b->slots[slot].done;
  return LBM_OK;
}

lbm_status lbm_batch_set_steps_done(lbm_batch *b, int32_t slot, int64_t steps) {
  lbm_status rc = check_slot(b, slot);
  if (rc != LBM_OK) return rc;
  Slot &s = b->slots[slot];
  if (steps < 0 || steps > s.target)
    return fail(LBM_EINVAL, "step index %lld outside [0, %lld]", static_cast<long long>(steps), s.target);
  if (s.fsi && steps != s.done)
    return fail(LBM_EINVAL, "a domain with coupled bodies cannot change its step index (its geometry is state)");
  if (s.p.moving)  // the mask and centres of the new step index
    LBM_CUDA(launch_place(b->st, b->d_doms + slot, s.p.nx, s.p.ny, s.pitch, steps));
  LBM_CUDA(cudaStreamSynchronize(b->st));
  s.done = steps;
  s.drained = entries_at(s, steps);  // nothing pending: entries before the index are gone
  return LBM_OK;
}

lbm_status lbm_batch_get_mask(lbm_batch *b, int32_t slot, uint8_t *out) {
  return get_mask(b, slot, out);
}

lbm_status lbm_batch_set_dynamics(lbm_batch *b, int32_t slot, int32_t body, const lbm_body_dynamics *dyn) {
  lbm_status rc = check_slot(b, slot);
  if (rc != LBM_OK) return rc;
  Slot &s = b->slots[slot];
  if (!dyn) return fail(LBM_EINVAL, "dynamics is NULL");
  if (!s.p.moving) return fail(LBM_EINVAL, "coupled bodies need a moving domain");
  if (s.p.moving == 2) return fail(LBM_EINVAL, "coupled bodies do not turn their shapes (moving = 2)");
  if (s.p.force_every != 1) return fail(LBM_EINVAL, "coupled bodies need the force of every step (force_every = 1)");
  if (s.done != 0) return fail(LBM_EINVAL, "dynamics are set before the first step");
  if (s.link_west != -1 || s.link_east != -1) return fail(LBM_EINVAL, "a linked domain cannot have coupled bodies");
  if (s.dev.deform) return fail(LBM_EINVAL, "a domain with pulsating bodies cannot have coupled bodies");
  if (body < 1 || body > s.nbodies) return fail(LBM_EINVAL, "body %d not in [1, %d]", body, s.nbodies);
  if (!(dyn->mass > 0) || !std::isfinite(dyn->mass)) return fail(LBM_EINVAL, "mass must be finite and > 0");
  for (int e = 0; e < 2; ++e) {
    if (!(dyn->stiffness[e] >= 0) || !std::isfinite(dyn->stiffness[e]) || !(dyn->damping[e] >= 0) ||
        !std::isfinite(dyn->damping[e]))
      return fail(LBM_EINVAL, "stiffness and damping must be finite and >= 0");
    if (dyn->free_axis[e] != 0 && dyn->free_axis[e] != 1) return fail(LBM_EINVAL, "free_axis must be 0 or 1");
  }
  DomDev &D = s.dev;
  LBM_CUDA(cudaStreamSynchronize(b->st));
  // the state of step 0 is the body's own centre and velocity, no earlier force
  double bt[5];
  LBM_CUDA(cudaMemcpyAsync(bt, D.bodies + 5 * (body - 1), sizeof(bt), cudaMemcpyDeviceToHost, b->st));
  LBM_CUDA(cudaStreamSynchronize(b->st));
  const double st0[6] = {bt[0], bt[1], bt[2], bt[3], 0.0, 0.0};
  const double par[8] = {dyn->mass, dyn->stiffness[0], dyn->stiffness[1], dyn->damping[0], dyn->damping[1],
                         double(dyn->free_axis[0]), double(dyn->free_axis[1]), 1.0};
  LBM_CUDA(cudaMemcpyAsync(D.fsi + 6 * (body - 1), st0, sizeof(st0), cudaMemcpyHostToDevice, b->st));
  LBM_CUDA(cudaMemcpyAsync(const_cast<double *>(D.fsi_par) + 8 * (body - 1), par, sizeof(par),
                           cudaMemcpyHostToDevice, b->st));
  D.fsi_on = 1;
  LBM_CUDA(cudaMemcpyAsync(b->d_doms + slot, &D, sizeof(DomDev), cudaMemcpyHostToDevice, b->st));
  LBM_CUDA(cudaStreamSynchronize(b->st));
  s.fsi = true;
  b->dirty = true;
  return LBM_OK;
}

lbm_status lbm_batch_set_deformation(lbm_batch *b, int32_t slot, int32_t body, double amplitude, double rate) {
  lbm_status rc = check_slot(b, slot);
  if (rc != LBM_OK) return rc;
  Slot &s = b->slots[slot];
  if (!s.p.moving) return fail(LBM_EINVAL, "pulsating bodies need a moving domain");
  if (s.done != 0) return fail(LBM_EINVAL, "a deformation is set before the first step");
  if (s.fsi) return fail(LBM_EINVAL, "coupled bodies do not deform");
  if (s.link_west != -1 || s.link_east != -1) return fail(LBM_EINVAL, "a linked domain cannot have pulsating bodies");
  if (body < 1 || body > s.nbodies) return fail(LBM_EINVAL, "body %d not in [1, %d]", body, s.nbodies);
  if (!(std::fabs(amplitude) < 1.0) || !std::isfinite(rate))
    return fail(LBM_EINVAL, "the amplitude must satisfy |a| < 1 and the rate be finite");
  DomDev &D = s.dev;
  LBM_CUDA(cudaStreamSynchronize(b->st));
  const double par[2] = {amplitude, rate};
  LBM_CUDA(cudaMemcpyAsync(const_cast<double *>(D.dpar) + 2 * (body - 1), par, sizeof(par), cudaMemcpyHostToDevice,
                           b->st));
  D.deform |= 1u << (body - 1);
  LBM_CUDA(cudaMemcpyAsync(b->d_doms + slot, &D, sizeof(DomDev), cudaMemcpyHostToDevice, b->st));
  // the mask, centres and dilation rates of step index 0 with the pulsating placement
  LBM_CUDA(launch_place(b->st, b->d_doms + slot, s.p.nx, s.p.ny, s.pitch, 0));
  LBM_CUDA(cudaStreamSynchronize(b->st));
  b->dirty = true;
  return LBM_OK;
}

lbm_status lbm_batch_coupled_state(lbm_batch *b, int32_t slot, double *out) {
  lbm_status rc = check_slot(b, slot);
  if (rc != LBM_OK) return rc;
  Slot &s = b->slots[slot];
  if (!out) return fail(LBM_EINVAL, "out is NULL");
  if (!s.fsi) return fail(LBM_EINVAL, "the slot has no coupled body");
  std::vector<double> st(6 * s.nbodies), par(8 * s.nbodies);
  const double *cur = s.dev.fsi + static_cast<size_t>(s.done & 1) * s.nbodies * 6;
  LBM_CUDA(cudaMemcpyAsync(st.data(), cur, sizeof(double) * st.size(), cudaMemcpyDeviceToHost, b->st));
  LBM_CUDA(cudaMemcpyAsync(par.data(), s.dev.fsi_par, sizeof(double) * par.size(), cudaMemcpyDeviceToHost, b->st));
  LBM_CUDA(cudaStreamSynchronize(b->st));
  for (int k = 0; k < s.nbodies; ++k)
    for (int e = 0; e < 6; ++e) out[6 * k + e] = par[8 * k + 7] != 0.0 ? st[6 * k + e] : 0.0;
  return LBM_OK;
}

lbm_status lbm_batch_restore_coupled(lbm_batch *b, int32_t slot, int64_t steps, const double *in) {
  lbm_status rc = check_slot(b, slot);
  if (rc != LBM_OK) return rc;
  Slot &s = b->slots[slot];
  if (!in) return fail(LBM_EINVAL, "in is NULL");
  if (!s.fsi) return fail(LBM_EINVAL, "the slot has no coupled body");
  if (steps < 0 || steps > s.target)
    return fail(LBM_EINVAL, "step index %lld outside [0, %lld]", static_cast<long long>(steps), s.target);
  for (int q = 0; q < 6 * s.nbodies; ++q)
    if (!std::isfinite(in[q])) return fail(LBM_EINVAL, "coupled state holds a non-finite value");
  std::vector<double> par(8 * s.nbodies);
  LBM_CUDA(cudaMemcpyAsync(par.data(), s.dev.fsi_par, sizeof(double) * par.size(), cudaMemcpyDeviceToHost, b->st));
  LBM_CUDA(cudaStreamSynchronize(b->st));
  double *cur = s.dev.fsi + static_cast<size_t>(steps & 1) * s.nbodies * 6;
  for (int k = 0; k < s.nbodies; ++k) {
    if (par[8 * k + 7] == 0.0) continue;  // prescribed bodies follow the step index
    LBM_CUDA(cudaMemcpyAsync(cur + 6 * k, in + 6 * k, sizeof(double) * 6, cudaMemcpyHostToDevice, b->st));
  }
  // body table and mask of that geometry (coupled bodies from the state just written)
  LBM_CUDA(launch_place(b->st, b->d_doms + slot, s.p.nx, s.p.ny, s.pitch, steps));
  LBM_CUDA(cudaStreamSynchronize(b->st));
  s.done = steps;
  s.drained = entries_at(s, steps);
  return LBM_OK;
}

lbm_status lbm_batch_body_state(lbm_batch *b, int32_t slot, double *out) {
  lbm_status rc = check_slot(b, slot);
  if (rc != LBM_OK) return rc;
  Slot &s = b->slots[slot];
  if (!out) return fail(LBM_EINVAL, "out is NULL");
  if (s.nbodies == 0) return LBM_OK;
  LBM_CUDA(cudaMemcpyAsync(out, s.dev.bodies, sizeof(double) * 5 * s.nbodies, cudaMemcpyDeviceToHost, b->st));
  LBM_CUDA(cudaStreamSynchronize(b->st));
  return LBM_OK;
}

lbm_status lbm_batch_profile(lbm_batch *b, int32_t steps, double *sweep_us, double *force_us,
                             int64_t *steps_run) {
  if (!b) return fail(LBM_EINVAL, "batch is NULL");
  if (steps < 1 || steps > 100000) return fail(LBM_EINVAL, "steps must be in [1, 100000]");
  Profile prof;
  long long n = 0;
  lbm_status rc = run(b, steps, &n, &prof);
  if (steps_run) *steps_run = n;
  if (sweep_us) *sweep_us = n > 0 ? 1000.0 * prof.sweep_ms / n : 0.0;
  if (force_us) *force_us = n > 0 ? 1000.0 * prof.force_ms / n : 0.0;
  return rc;
}

lbm_status lbm_batch_link_x(lbm_batch *b, int32_t west_slot, int32_t east_slot) {
  lbm_status rc = check_slot(b, west_slot);
  if (rc == LBM_OK) rc = check_slot(b, east_slot);
  if (rc != LBM_OK) return rc;
  Slot &A = b->slots[west_slot];
  Slot &B = b->slots[east_slot];
  if (A.p.ny != B.p.ny) return fail(LBM_EINVAL, "linked domains need the same ny (%d, %d)", A.p.ny, B.p.ny);
  if (A.p.south != B.p.south || A.p.north != B.p.north)
    return fail(LBM_EINVAL, "linked domains need the same y edges");
  if (A.done != B.done || A.target != B.target || A.parity != B.parity)
    return fail(LBM_EINVAL, "linked domains must step together (same steps done and admitted)");
  if (A.link_east != -1 || B.link_west != -1) return fail(LBM_EINVAL, "an edge is linked already");
  if (A.fsi || B.fsi) return fail(LBM_EINVAL, "domains with coupled bodies cannot be linked");
  if (A.dev.deform || B.dev.deform) return fail(LBM_EINVAL, "domains with pulsating bodies cannot be linked");
  LBM_CUDA(cudaStreamSynchronize(b->st));
  // A's east edge pulls B's first column; B's west edge pulls A's last column
  A.dev.east = LBM_NEIGHBOR;
  A.dev.nb_nx[1] = B.p.nx;
  A.dev.nb_pitch[1] = B.pitch;
  A.dev.nb_lat[1][0] = B.dev.lat[0];
  A.dev.nb_lat[1][1] = B.dev.lat[1];
  B.dev.west = LBM_NEIGHBOR;
  B.dev.nb_nx[0] = A.p.nx;
  B.dev.nb_pitch[0] = A.pitch;
  B.dev.nb_lat[0][0] = A.dev.lat[0];
  B.dev.nb_lat[0][1] = A.dev.lat[1];
  A.link_east = east_slot;
  B.link_west = west_slot;
  LBM_CUDA(cudaMemcpyAsync(b->d_doms + west_slot, &A.dev, sizeof(DomDev), cudaMemcpyHostToDevice, b->st));
  LBM_CUDA(cudaMemcpyAsync(b->d_doms + east_slot, &B.dev, sizeof(DomDev), cudaMemcpyHostToDevice, b->st));
  LBM_CUDA(cudaStreamSynchronize(b->st));
  return LBM_OK;
}

lbm_status lbm_batch_set_halo(lbm_batch *b, int32_t slot, int32_t side, void *recv, void *send) {
  lbm_status rc = check_slot(b, slot);
  if (rc != LBM_OK) return rc;
  if (side != 0 && side != 1) return fail(LBM_EINVAL, "side must be 0 (west) or 1 (east)");
  Slot &s = b->slots[slot];
  int &link = side == 0 ? s.link_west : s.link_east;
  int32_t &edge = side == 0 ? s.dev.west : s.dev.east;
  if (link >= 0) return fail(LBM_EINVAL, "the %s edge is linked to slot %d", side ? "east" : "west", link);
  if ((recv == nullptr) != (send == nullptr)) return fail(LBM_EINVAL, "recv and send must both be given or both NULL");
  if (recv) {
    if (s.fsi) return fail(LBM_EINVAL, "domains with coupled bodies cannot have halo edges");
    if (s.dev.deform) return fail(LBM_EINVAL, "domains with pulsating bodies cannot have halo edges");
    if ((reinterpret_cast<uintptr_t>(recv) | reinterpret_cast<uintptr_t>(send)) % elem_size(b->storage))
      return fail(LBM_EINVAL, "halo buffers must be aligned to the element size");
  }
  LBM_CUDA(cudaStreamSynchronize(b->st));
  if (recv) {
    // the linked-edge read of the sweep, with the caller's buffer as a one-column lattice
    edge = LBM_NEIGHBOR;
    s.dev.nb_nx[side] = 1;
    s.dev.nb_pitch[side] = 1;
    s.dev.nb_lat[side][0] = recv;
    s.dev.nb_lat[side][1] = recv;
    s.halo_send[side] = send;
    link = -2;
  } else {
    edge = side == 0 ? s.p.west : s.p.east;
    s.dev.nb_nx[side] = 0;
    s.dev.nb_pitch[side] = 0;
    s.dev.nb_lat[side][0] = nullptr;
    s.dev.nb_lat[side][1] = nullptr;
    s.halo_send[side] = nullptr;
    link = -1;
  }
  LBM_CUDA(cudaMemcpyAsync(b->d_doms + slot, &s.dev, sizeof(DomDev), cudaMemcpyHostToDevice, b->st));
  LBM_CUDA(cudaStreamSynchronize(b->st));
  return LBM_OK;
}

lbm_status lbm_batch_pack_halos(lbm_batch *b) {
  Range range("lbm_batch_pack_halos");
  if (!b) return fail(LBM_EINVAL, "batch is NULL");
  HaloPack pack{};
  pack.elem = static_cast<int32_t>(elem_size(b->storage));
  int max_ny = 0;
  for (const Slot &s : b->slots) {
    if (!s.used) continue;
    for (int side = 0; side < 2; ++side) {
      if (!s.halo_send[side]) continue;
      if (pack.n == kMaxHaloItems) {
        LBM_CUDA(launch_halo_pack(b->st, pack, max_ny));
        b->launches++;
        pack.n = 0;
        max_ny = 0;
      }
      pack.item[pack.n++] = HaloItem{s.dev.lat[s.parity], s.halo_send[side], s.p.ny, s.pitch,
                                     side == 1 ? s.p.nx - 1 : 0, side};
      max_ny = std::max(max_ny, s.p.ny);
    }
  }
  if (pack.n > 0) {
    LBM_CUDA(launch_halo_pack(b->st, pack, max_ny));
    b->launches++;
  }
  return LBM_OK;
}

lbm_status lbm_batch_evict(lbm_batch *b, int32_t slot) {
  lbm_status rc = check_slot(b, slot);
  if (rc != LBM_OK) return rc;
  Slot &s = b->slots[slot];
  LBM_CUDA(cudaStreamSynchronize(b->st));
  // a linked partner gets its own edge rule back
  if (s.link_west >= 0) {
    Slot &P = b->slots[s.link_west];
    P.dev.east = P.p.east;
    P.link_east = -1;
    LBM_CUDA(cudaMemcpyAsync(b->d_doms + s.link_west, &P.dev, sizeof(DomDev), cudaMemcpyHostToDevice, b->st));
  }
  if (s.link_east >= 0) {
    Slot &P = b->slots[s.link_east];
    P.dev.west = P.p.west;
    P.link_west = -1;
    LBM_CUDA(cudaMemcpyAsync(b->d_doms + s.link_east, &P.dev, sizeof(DomDev), cudaMemcpyHostToDevice, b->st));
  }
  LBM_CUDA(cudaStreamSynchronize(b->st));
  release_memory(b, s);
  s = Slot();
  b->dirty = true;
  return LBM_OK;
}

lbm_status lbm_batch_capture(lbm_batch *b) {
  Range range("lbm_batch_capture");
  if (!b) return fail(LBM_EINVAL, "batch is NULL");
  if (b->graph_steps <= 0) return LBM_OK;  // the batch steps with direct launches
  if (b->dirty) {
    lbm_status rc = rebuild_lists(b);
    if (rc != LBM_OK) return rc;
  }
  if (!b->graph) return capture_graph(b);
  return LBM_OK;
}

lbm_status lbm_batch_inject(lbm_batch *b, int32_t slot, int32_t kind) {
  if (!b) return fail(LBM_EINVAL, "batch is NULL");
  switch (kind) {
    case LBM_INJECT_NONE:
    case LBM_INJECT_WAIT_TIMEOUT: {
      const int want = kind == LBM_INJECT_WAIT_TIMEOUT ? 1 : 0;
      if (want != b->inject) {
        b->inject = want;
        drop_graph(b);  // a captured graph holds the launch arguments
      }
      return LBM_OK;
    }
    case LBM_INJECT_UNSTABLE: {
      lbm_status rc = check_slot(b, slot);
      if (rc != LBM_OK) return rc;
      static const int32_t kUnstable = 1;
      // the status word is only ever OR-ed: a plain write would race with the sweep's
      // atomics, so the host stores the bit in stream order (no sweep runs meanwhile)
      LBM_CUDA(cudaMemcpyAsync(b->slots[slot].dev.status, &kUnstable, sizeof(int32_t),
                               cudaMemcpyHostToDevice, b->st));
      LBM_CUDA(cudaStreamSynchronize(b->st));
      return LBM_OK;
    }
  }
  return fail(LBM_EINVAL, "unknown injection kind %d", kind);
}

lbm_status lbm_batch_autotune(lbm_batch *b, int32_t reps, double *best_us) {
  Range range("lbm_batch_autotune");
  if (!b) return fail(LBM_EINVAL, "batch is NULL");
  return autotune(b, reps, best_us);
}

lbm_status lbm_batch_set_grouped_admission(lbm_batch *b, int32_t on) {
  if (!b) return fail(LBM_EINVAL, "batch is NULL");
  if (on != 0 && on != 1) return fail(LBM_EINVAL, "on must be 0 or 1");
  b->group_admit = on != 0;
  return LBM_OK;
}

lbm_status lbm_batch_set_tile(lbm_batch *b, int32_t vec, int32_t warps, int32_t rows,
                              int32_t pipeline) {
  if (!b) return fail(LBM_EINVAL, "batch is NULL");
  return set_config(b, vec, warps, rows, pipeline);
}

lbm_status lbm_batch_get_tile(lbm_batch *b, int32_t *vec, int32_t *warps, int32_t *rows,
                              int32_t *pipeline) {
  if (!b) return fail(LBM_EINVAL, "batch is NULL");
  if (vec) *vec = b->vec;
  if (warps) *warps = b->warps;
  if (rows) *rows = b->rows;
  if (pipeline) *pipeline = b->pipe;
  return LBM_OK;
}

lbm_status lbm_batch_info(lbm_batch *b, int32_t *resident, int64_t *cells, int64_t *launches,
                          size_t *bytes) {
  if (!b) return fail(LBM_EINVAL, "batch is NULL");
  int r = 0;
  long long c = 0;
  for (const Slot &s : b->slots)
    if (s.used) {
      ++r;
      c += static_cast<long long>(s.p.nx) * s.p.ny;
    }
  if (resident) *resident = r;
  if (cells) *cells = c;
  if (launches) *launches = b->launches;
  if (bytes) *bytes = b->bytes_in_use;
  return LBM_OK;
}

lbm_status lbm_batch_destroy(lbm_batch *b) {
  destroy(b);
  return LBM_OK;
}

// ---- single domain: a batch with one slot and an unbounded step target ------------------

lbm_status lbm_domain_create(const lbm_params *p, const uint8_t *mask, const lbm_geometry *geom,
                             const lbm_body *bodies, int32_t nbodies, void *cuda_stream,
                             lbm_alloc_fn alloc, lbm_free_fn free_fn, void *alloc_ctx,
                             lbm_domain **out) {
  if (!out) return fail(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  lbm_status rc = validate(p, nbodies);
  if (rc != LBM_OK) return rc;
  lbm_batch *b = nullptr;
  rc = create(1, 0, p->storage, 32, cuda_stream, alloc, free_fn, alloc_ctx, &b);
  if (rc != LBM_OK) return rc;
  int slot = -1;
  rc = admit(b, p, mask, geom, bodies, nbodies, std::numeric_limits<long long>::max(), &slot);
  if (rc != LBM_OK) {
    destroy(b);
    return rc;
  }
  lbm_domain *d = new (std::nothrow) lbm_domain();
  if (!d) {
    destroy(b);
    return fail(LBM_ENOMEM, "host allocation failed");
  }
  d->b = b;
  // resolve lbm_moments_noalloc's staging array on this device now (with lazy module
  // loading, its module and the array's memory are loaded here), so that the
  // allocation-free call itself loads nothing; a failure is retried by that call
  int dev = 0;
  double *scratch = nullptr;
  if (cudaGetDevice(&dev) == cudaSuccess && noalloc_scratch_on(dev, &scratch) != LBM_OK)
    cudaGetLastError();
  *out = d;
  return LBM_OK;
}

lbm_status lbm_step(lbm_domain *d, int64_t nsteps) {
  Range range("lbm_step");
  if (!d) return fail(LBM_EINVAL, "domain is NULL");
  if (nsteps < 0) return fail(LBM_EINVAL, "nsteps must be >= 0");
  long long n = 0;
  return run(d->b, nsteps, &n);
}

lbm_status lbm_forces(lbm_domain *d, double *out, int64_t max_entries, int64_t *written) {
  if (!d) return fail(LBM_EINVAL, "domain is NULL");
  long long w = 0;
  int done = 0;
  lbm_status rc = poll(d->b, 0, out, max_entries, &w, &done);
  if (written) *written = w;
  return rc;
}

lbm_status lbm_moments(lbm_domain *d, double *rho, double *ux, double *uy) {
  Range range("lbm_moments");
  if (!d) return fail(LBM_EINVAL, "domain is NULL");
  return moments(d->b, 0, rho, ux, uy);
}

lbm_status lbm_get_populations(lbm_domain *d, void *out, size_t bytes) {
  if (!d || !out) return fail(LBM_EINVAL, "domain or out is NULL");
  return populations(d->b, 0, out, nullptr, bytes);
}

lbm_status lbm_set_populations(lbm_domain *d, const void *in, size_t bytes) {
  if (!d) return fail(LBM_EINVAL, "domain is NULL");
  return populations(d->b, 0, nullptr, in, bytes);
}

lbm_status lbm_get_mask(lbm_domain *d, uint8_t *out) {
  if (!d) return fail(LBM_EINVAL, "domain is NULL");
  return get_mask(d->b, 0, out);
}

lbm_status lbm_steps_done(lbm_domain *d, int64_t *steps) {
  if (!d) return fail(LBM_EINVAL, "domain is NULL");
  if (steps) *steps = d->b->slots[0].done;
  return LBM_OK;
}

lbm_status lbm_set_steps_done(lbm_domain *d, int64_t steps) {
  if (!d) return fail(LBM_EINVAL, "domain is NULL");
  return lbm_batch_set_steps_done(d->b, 0, steps);
}

lbm_status lbm_set_dynamics(lbm_domain *d, int32_t body, const lbm_body_dynamics *dyn) {
  if (!d) return fail(LBM_EINVAL, "domain is NULL");
  return lbm_batch_set_dynamics(d->b, 0, body, dyn);
}

lbm_status lbm_set_deformation(lbm_domain *d, int32_t body, double amplitude, double rate) {
  if (!d) return fail(LBM_EINVAL, "domain is NULL");
  return lbm_batch_set_deformation(d->b, 0, body, amplitude, rate);
}

lbm_status lbm_body_state(lbm_domain *d, double *out) {
  if (!d) return fail(LBM_EINVAL, "domain is NULL");
  return lbm_batch_body_state(d->b, 0, out);
}

lbm_status lbm_coupled_state(lbm_domain *d, double *out) {
  if (!d) return fail(LBM_EINVAL, "domain is NULL");
  return lbm_batch_coupled_state(d->b, 0, out);
}

lbm_status lbm_restore_coupled(lbm_domain *d, int64_t steps, const double *in) {
  if (!d) return fail(LBM_EINVAL, "domain is NULL");
  return lbm_batch_restore_coupled(d->b, 0, steps, in);
}

lbm_status lbm_domain_destroy(lbm_domain *d) {
  if (!d) return LBM_OK;
  destroy(d->b);
  delete d;
  return LBM_OK;
}

}  // extern "C"

// ======================================================================================
// Moments export without any device allocation.
//
// lbm_moments stages its three output fields in a device buffer it allocates for the
// call. Some callers cannot let a library allocate at that point: an application that
// has handed every byte of device memory to its own arena (a training or serving
// process whose caching allocator holds the GPU), a monitoring tap polled from a loop
// where an allocation's implicit device synchronisation or latency is not acceptable,
// or code that must keep the device footprint fixed after start-up. lbm_moments_noalloc
// stages the fields in one fixed file-scope device array instead, sized for domains of
// up to kNoAllocMaxNodes nodes; every GPU that loads this library holds that array
// (3 * 2^18 doubles = 6 MiB) until the process exits.

namespace lbm {
namespace {

constexpr size_t kNoAllocMaxNodes = size_t(1) << 18;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_moments_scratch[3 * kNoAllocMaxNodes];

std::mutex g_scratch_mu;
double *g_scratch_addr[kNoAllocMaxDevices] = {};

}  // namespace

// Device address of g_moments_scratch on `dev` (which must be current). In host code
// the array's name is only a host-side stand-in, so the address is looked up once per
// device with cudaGetSymbolAddress and cached.
lbm_status noalloc_scratch_on(int dev, double **out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(LBM_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_moments_scratch);
    if (e != cudaSuccess)
      return fail(LBM_ECUDA, "cudaGetSymbolAddress(g_moments_scratch) failed: %s", cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[dev];
  return LBM_OK;
}

}  // namespace lbm

extern "C" lbm_status lbm_moments_noalloc(lbm_domain *d, double *rho, double *ux, double *uy) {
  if (!d) return fail(LBM_EINVAL, "domain is NULL");
  lbm_batch *b = d->b;
  const Slot &s = b->slots[0];
  const size_t cells = static_cast<size_t>(s.p.nx) * s.p.ny;
  if (cells > kNoAllocMaxNodes)
    return fail(LBM_EINVAL,
                "lbm_moments_noalloc: domain has %zu nodes, more than the %zu its fixed staging "
                "array holds; use lbm_moments",
                cells, kNoAllocMaxNodes);
  // the domain's device must be the current one: the staging address is per device
  cudaPointerAttributes attr{};
  LBM_CUDA(cudaPointerGetAttributes(&attr, s.dev.lat[0]));
  int cur = -1;
  LBM_CUDA(cudaGetDevice(&cur));
  if (attr.device != cur)
    return fail(LBM_EINVAL, "domain lives on device %d but device %d is current", attr.device, cur);
  double *tmp = nullptr;
  lbm_status rc = noalloc_scratch_on(cur, &tmp);
  if (rc != LBM_OK) return rc;
  LBM_CUDA(launch_moments_sized(b->storage, b->st, b->d_doms, s.p.nx, s.p.ny, s.parity, tmp,
                                tmp + cells, tmp + 2 * cells));
  double *outs[3] = {rho, ux, uy};
  for (int q = 0; q < 3; ++q)
    if (outs[q])
      LBM_CUDA(cudaMemcpyAsync(outs[q], tmp + q * cells, sizeof(double) * cells, cudaMemcpyDefault, b->st));
  LBM_CUDA(cudaStreamSynchronize(b->st));
  int status = 0;
  rc = read_status(b, s, &status);
  if (rc != LBM_OK) return rc;
  if (status & 2) return fail(LBM_ETIMEOUT, "a sweep gave up waiting for its row copies");
  if (status & 1) return fail(LBM_EUNSTABLE, "domain diverged");
  return LBM_OK;
}
