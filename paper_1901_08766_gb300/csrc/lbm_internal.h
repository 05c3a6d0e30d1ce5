// Internal types shared by the CUDA kernels and the host runtime of the TRT-LBM-VP
// library. Not part of the public ABI (include/lbm.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cmath>

#include <cuda_runtime.h>

#include "../../include/lbm.h"

namespace lbm {

constexpr int kQ = 9;
constexpr int kPitchAlign = 64;  // row pitch in elements is a multiple of this
constexpr int kMaxBodies = 255;
constexpr int kMaxMovingShapes = 64;  // geometry kept on the device by a moving domain
constexpr int kMaxMovingBodies = 8;

// Per-domain constants of the collision in one precision (filled on the host).
// FP16-shifted storage holds kF16Scale (f - w rho0): values up to 65504 / 1024 = 64
// (rho below about 145) and full FP16 precision down to 2^-24 = 6e-8.
constexpr float kF16Scale = 1024.0f;

template <typename T> struct CellConst {
  T omp, omm;        // omega+ = 1/tau_s, omega- = 1/tau_a
  T hp, hm;          // omega+/2, omega-/2
  T one_m_omp;       // 1 - omega+
  T inv_2eta1;       // 1 / (2 eta + 1)
  T rho0;            // rho0 times the storage scale (compute space)
  T pw0, pw1, pw2;   // omega+ * w for the rest, axis and diagonal classes
  T mw1, mw2;        // 3 omega- * w for the axis and diagonal classes
  T kw0, kw1, kw2;   // (1 - omega+/2) * w per class (Guo symmetric part)
  T qw1, qw2;        // 3 (1 - omega-/2) * w per class (Guo antisymmetric part)
  T wr0, wr1, wr2;   // w * rho0 per class: the shift of the shifted compute variables
  T ghost[kQ];       // inlet populations in compute space, as a stored node would hold them
};

// Per-domain static description, resident in device memory (one per batch slot).
struct ShapeDev;
struct PlacedShape;

struct DomDev {
  void *lat[2];            // lattice A/B: [9][ny][pitch] elements of the storage type
  uint8_t *mask;           // [ny][pitch] body id, 0 = fluid
  double *bodies;          // [nbodies][5]: cx, cy, vx, vy, omega (centres at the current step)
  float *bodies_f;         // the same table rounded to FP32 (FP32-compute storages)
  const int32_t *solid;    // solid nodes (j * pitch + i), grouped by body, row-major
  const int32_t *solid_off;// [nbodies + 1] offsets into solid
  void *fvp[2];            // F_VP of solid nodes, [ny][pitch] pairs in compute precision, one
                           // field per parity of the lattice the sweep read: a step's force
                           // reduction reads one while the next step's sweep writes the other
  double *ring;            // force ring [cap][nbodies][2]
  int32_t *status;         // bit 0: unstable; bit 1: a bounded device-side wait ran out
  int32_t nx, ny, pitch;
  int32_t west, east, south, north;
  int32_t nbodies, force_every, force_cap;
  double omega_p, omega_m;  // 1/tau_s, 1/tau_a
  double inv_2eta1;         // 1 / (2 eta + 1)
  double rho0;
  double ghost[kQ];         // inlet populations f^eq(rho0, u_in) (minus w rho0 if storage is shifted)
  CellConst<float> cf;      // collision constants for FP32 compute
  CellConst<double> cd;     // collision constants for FP64 compute
  // moving domains (prescribed translation; null / 0 otherwise)
  const ShapeDev *shapes;   // [nshapes] reference geometry (step index 0)
  PlacedShape *placed;      // [nshapes] moving domains: each shape at the next step index,
                            // written once per step before the move kernel reads it
  const float4 *shapes_f;   // [nshapes] FP32 centre x, y and extent (shape_extent) of each
  const double *centre0;    // [nbodies][2] reference centres
  double *rowsum[2];        // [ny][nbodies][3] per-row sums of -F_VP and the step they belong to,
                            // one table per lattice parity (as the F_VP fields)
  int32_t nshapes, moving;
  // slab decomposition: global column of local column 0, and the lattices of linked
  // neighbour domains ([0] west, [1] east; used where the edge is LBM_NEIGHBOR)
  int32_t x0;
  int32_t nb_nx[2], nb_pitch[2];
  void *nb_lat[2][2];  // [side][lattice A/B]
  // coupled bodies of a moving domain (fluid-structure coupling; null / 0 otherwise)
  double *fsi;              // [2][nbodies][6] body state of step n in [n & 1]: x, y, vx, vy
                            // and the force of step n - 1 (Fx, Fy)
  const double *fsi_par;    // [nbodies][8]: mass, k_x, k_y, c_x, c_y, free_x, free_y, coupled
  int32_t fsi_on;           // some body of the domain is coupled
  int32_t fsi_pad;
  // deforming bodies: [nbodies][2] amplitude a and rate nu of the pulsation
  // s(n) = 1 + a sin(nu n) (moving domains; null otherwise); the dilation rate kappa = s'/s
  // of the current step in FP64 and FP32 ([nbodies] each, every domain, zero for rigid
  // bodies); bit b of `deform`: body b + 1 pulsates
  const double *dpar;
  double *kappa;
  float *kappa_f;
  // turning or pulsating bodies: cos theta, sin theta and the scale s of step index m in
  // [m & 1][nbodies][3] (written one step ahead by the body-table update)
  double *turn;
  uint32_t deform;
  int32_t deform_pad;
};

// Per-domain dynamic state, uploaded at the start of each batch run.
struct DomDyn {
  long long step0;     // steps done when the run started
  long long step_end;  // the domain stops before this step count
  int32_t parity;      // lattice holding g at step0
  int32_t pad;
};

// One sweep tile: a warp-wide strip (32 * vec cells) by (warps * rows) rows.
struct TileDev {
  int32_t dom, x0, y0, pad;
};

// One force-reduction item: (slot, body id) and the body's range in the solid list, or
// (rows = 1, moving domains) the range of rows of the per-row sums.
struct ForceItem {
  int32_t dom, body, beg, end, rows, pad;
};

// One row of a moving domain for the geometry update.
struct MoveRow {
  int32_t dom, j;
};

// A row of a moving domain that a shape reaches at index n or n + 1 (the move kernels'
// list): its domain and row, and its column intervals at n and at n + 1 (lo > hi: none).
struct BusyRow {
  int32_t dom, j, olo, ohi, nlo, nhi;
};

// Device-side counters of a batch.
struct Counters {
  int32_t ntiles;
  int32_t nforce;
  long long run_base;  // steps completed in the current run (advanced by the graphs)
  int32_t nmove;       // rows of moving domains
  int32_t nmovedom;    // moving domains, listed after their rows
  // work items of the direct sweep, taken by warps in turn: the next item and the warps
  // that have run out; the last warp to run out resets both for the next launch
  int32_t item_next, item_done;
  // the move kernels' list of busy rows: its length, and the blocks of the second launch
  // that have finished (the last one empties the list)
  int32_t nbusy, busy_done;
};

struct SweepArgs {
  const DomDev *doms;
  const DomDyn *dyn;
  const TileDev *tiles;
  const Counters *ctr;
  int32_t rows;  // rows per warp
  // host-side failure injection (tests of the error paths; no GPU fault): bit 0 makes the
  // TMA-staged sweep report its first row wait as timed out after that wait has completed
  int32_t inject;
};

struct ShapeDev {
  int32_t kind, body;
  double cx, cy, radius, chord, thickness, ca, sa;  // ca, sa = cos/sin(aoa) from the host
};

// A shape at one step index with the FP32 copies of the move kernel's circle pre-test.
struct PlacedShape {
  ShapeDev s;
  float fcx, fcy, fr2;  // centre and squared radius in FP32
  int32_t fast;         // a circle within the pre-test's bounds
};

// Largest distance of a shape's node from its reference point: the radius of a circle;
// for a NACA section (reference at the quarter chord) 3/4 of the chord along it plus the
// largest half thickness across it, 5 |t| c max(poly) < 5 |t| c (0.2969 + 0.2843) < 3 |t| c,
// and never less than the chord.
__host__ __device__ inline double shape_extent(const ShapeDev &s) {
  if (s.kind == LBM_SHAPE_CIRCLE) return s.radius;
  return fmax(s.chord, 0.75 * s.chord + 3.0 * fabs(s.thickness) * s.chord);
}

// One domain of a batched admission (lbm_batch_admit_many): where its mask, lattices and
// solid-node list live, its geometry, and the position of its rows in the flat row list
// of all admitted domains (rows row0 .. row0 + ny - 1).
struct AdmitDev {
  uint8_t *mask;
  void *lat[2];
  int32_t *counts;         // [nbodies + 1][ny] per-row node counts of each body id
  const int32_t *row_off;  // [nbodies][ny] offsets of each body's nodes of a row in `solid`
  int32_t *solid;          // the domain's solid-node list
  const ShapeDev *shapes;
  int32_t nshapes, nx, ny, pitch, nbodies, x0, row0, bad;  // bad: largest unknown body id
  double rho0, u0x, u0y;
};

// One halo edge to pack (slab decomposition over devices): the populations of the three
// directions that cross the edge outward, taken from column `col` of the current lattice
// `lat` ([9][ny][pitch]), written to `send` ([9][ny], those three planes only). east:
// the east edge (directions 1, 5, 8 from the last column), else the west edge (3, 6, 7
// from column 0).
struct HaloItem {
  const void *lat;
  void *send;
  int32_t ny, pitch, col, east;
};
constexpr int kMaxHaloItems = 64;  // halo edges packed by one launch
struct HaloPack {
  HaloItem item[kMaxHaloItems];
  int32_t n, elem;  // items, element size in bytes
};

// A span of device memory to fill (batched admission): a copy of `bytes` from src, or
// zeros when src is null.
struct FillSeg {
  void *dst;
  const void *src;
  size_t bytes;
};

// Kernel launchers (one translation unit per storage type for the sweep).
cudaError_t launch_forces(int storage, int grid, cudaStream_t st, const DomDev *doms,
                          const DomDyn *dyn, const ForceItem *items, const Counters *ctr,
                          int s);
void fill_cell_const(DomDev &d, int storage);
// the message lbm_last_error returns (shared by the 2D and 3D entry points)
void set_last_error(const char *msg);
cudaError_t launch_advance(cudaStream_t st, Counters *ctr, int k);
// moving domains, step s: the rows a shape reaches at its index n or n + 1 listed in busy
// (needs only the shapes, so it may run beside the sweep) ...
cudaError_t launch_move_cull(int grid, cudaStream_t st, const DomDev *doms, const DomDyn *dyn,
                             const MoveRow *rows, const Counters *ctr, BusyRow *busy, int s);
// ... then, after the sweep, a warp per listed row: its -F_VP sums over the mask the
// sweep used, then its mask at n + 1, and the body centres of n + 1
cudaError_t launch_move_rows(int grid, cudaStream_t st, const DomDev *doms, const DomDyn *dyn,
                             const MoveRow *rows, const Counters *ctr, BusyRow *busy, int s, int storage);
// moving domains (rows: the move list, whose ctr->nmove rows are followed by one entry
// per moving domain): every shape at the index after step s, for the move kernel of
// step s; grid: blocks striding over the domains
cudaError_t launch_shape_table(int grid, cudaStream_t st, const DomDev *doms, const DomDyn *dyn,
                               const MoveRow *rows, const Counters *ctr, int s);
// the mask and body centres of one moving domain at step index n
cudaError_t launch_place(cudaStream_t st, const DomDev *dom_dev, int nx, int ny, int pitch, long long n);
// coupled bodies: advance their state with the force of the step just reduced, then the
// next step's mask of the rows of domains with coupled bodies
cudaError_t launch_fsi(int grid, cudaStream_t st, const DomDev *doms, const DomDyn *dyn,
                       const MoveRow *rows, const Counters *ctr, int s);
cudaError_t launch_rasterize(cudaStream_t st, uint8_t *mask, int nx, int ny, int pitch,
                             const ShapeDev *shapes, int nshapes, int x0);
cudaError_t launch_init(int storage, cudaStream_t st, void *lat, int nx, int ny, int pitch,
                        double rho0, double ux, double uy);
cudaError_t launch_row_counts(cudaStream_t st, const uint8_t *mask, int nx, int ny, int pitch,
                              int nbodies, int32_t *counts /* [nbodies+1][ny] */,
                              int32_t *bad_id);
cudaError_t launch_row_scatter(cudaStream_t st, const uint8_t *mask, int nx, int ny, int pitch,
                               int nbodies, const int32_t *row_off /* [nbodies][ny] */,
                               int32_t *solid);
cudaError_t launch_moments_sized(int storage, cudaStream_t st, const DomDev *dom, int nx,
                                 int ny, int parity, double *rho, double *ux, double *uy);
// batched admission over the flat row list of n domains (rows: total rows)
cudaError_t launch_admit_raster_count(cudaStream_t st, AdmitDev *ad, int n, int rows);
cudaError_t launch_admit_scatter(cudaStream_t st, const AdmitDev *ad, int n, int rows, int max_bodies);
cudaError_t launch_admit_init(int storage, cudaStream_t st, const AdmitDev *ad, int n, int rows);
cudaError_t launch_fill(cudaStream_t st, const FillSeg *segs, int nseg);
cudaError_t launch_halo_pack(cudaStream_t st, const HaloPack &pack, int max_ny);

// per-storage sweep launchers (one translation unit each); def: a resident domain has
// pulsating bodies (the direct sweep's instantiation with the kappa term of U_O)
cudaError_t launch_sweep_f64(int vec, int pipe, int grid, int warps, cudaStream_t st,
                             const SweepArgs &a, int s, bool def);
cudaError_t launch_sweep_f32(int vec, int pipe, int grid, int warps, cudaStream_t st,
                             const SweepArgs &a, int s, bool def);
cudaError_t launch_sweep_f16s(int vec, int pipe, int grid, int warps, cudaStream_t st,
                             const SweepArgs &a, int s, bool def);
cudaError_t launch_sweep_bf16s(int vec, int pipe, int grid, int warps, cudaStream_t st,
                             const SweepArgs &a, int s, bool def);
int max_blocks_f64(int vec, int pipe, int warps);
int max_blocks_f32(int vec, int pipe, int warps);
int max_blocks_f16s(int vec, int pipe, int warps);
int max_blocks_bf16s(int vec, int pipe, int warps);

}  // namespace lbm
