/*
 * lbm.h — C ABI of the GB300 TRT-LBM-VP library (libpaper_1901_08766_gb300.so).
 *
 * The library advances 2D D2Q9 flows past obstacles with the coupled two-relaxation-
 * time lattice Boltzmann / volume-penalization method of Cui, Wang, Yao, Liu and Yu
 * (arXiv:1901.08766). One time step is one fused CUDA sweep per domain: pull-stream
 * the populations (Eq. streaming), form rho and u* (Eq. rho, Eq. rho*velocity-star),
 * penalize solid nodes (Eq. d-V, Eq. force-density, Eq. velocity-r), and collide with
 * the TRT operator plus the split Guo forcing term (Eq. TRT-collision, Eq.
 * collision-modified). The force on each body (Sec. 3, drag and lift sums) is
 * reduced in FP64 every step into a device ring.
 *
 * Conventions for every call:
 *  - Every function returns lbm_status; nothing aborts, throws or traps across the
 *    ABI. lbm_last_error() gives a thread-local description of the last failure.
 *  - Lattice units: dx = dy = dt = 1, c_s^2 = 1/3. Node (i, j) sits at (i, j),
 *    i in [0, nx) along the flow, j in [0, ny) upward.
 *  - Populations are ordered alpha = 0..8 as in Eq. (D2Q9): rest, (1,0), (0,1),
 *    (-1,0), (0,-1), (1,1), (-1,1), (-1,-1), (1,-1).
 *  - The library owns all device memory it allocates (populations, mask, force
 *    ring); it allocates through the caller's lbm_alloc_fn (e.g. PyTorch's caching
 *    allocator), or through cudaMallocAsync when none is given. The caller owns every
 *    host buffer and every pointer it passes in; inputs are copied at the call.
 *  - Work is enqueued on the cudaStream_t given at creation and is asynchronous,
 *    except the calls documented as synchronising (they return host results).
 *  - A domain or batch is used from one host thread at a time.
 */
#ifndef PAPER_1901_08766_GB300_LBM_H
#define PAPER_1901_08766_GB300_LBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,    /* invalid argument or parameter combination */
  LBM_ENOMEM = 2,    /* device or host allocation failed */
  LBM_ECUDA = 3,     /* a CUDA runtime call failed (text in lbm_last_error) */
  LBM_EUNSTABLE = 4, /* a domain diverged: rho <= 0.01, rho >= 100 or not finite (sticky) */
  LBM_ETIMEOUT = 5,  /* a bounded device-side wait ran out (sticky per domain) */
  LBM_EBUSY = 6,     /* no free slot / over the memory budget / force ring full */
  LBM_ENOTFOUND = 7  /* unknown slot */
} lbm_status;

/* Population storage. Collision and penalization run in FP64 for LBM_F64 and in FP32
 * otherwise (LBM_F32 rounds to nearest even). LBM_BF16S stores f_alpha - w_alpha rho0
 * and LBM_F16S stores 1024 (f_alpha - w_alpha rho0) (shifted by the rest weights, so
 * that storage keeps the small deviations; the power-of-two scale keeps deviations down
 * to 6e-8 in FP16's normal range, and values up to 64, i.e. rho below about 145, fit).
 * Both round stochastically with counter-based random bits keyed by the step index and
 * the node, so that the stored value is exact in expectation; the rest population is
 * stored as the node's pulled mass minus the eight rounded moving populations, so that
 * rounding keeps each node's mass (Eq. (rho)) within one unit of the rest population.
 * The paper stores FP64 only: this rounding rule is the library's. */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16S = 2, LBM_BF16S = 3 } lbm_storage;

/* Domain-edge rules. x edges: west PERIODIC or INLET_EQ (ghost populations at
 * f^eq(rho0, u_in)); east PERIODIC or OUTFLOW_ZG (zero gradient: the missing
 * populations are read from the last column). y edges: PERIODIC or FREE_SLIP
 * (specular reflection, walls half a cell outside the first and last rows). Both
 * edges of an axis are periodic or neither is. The x rule is applied first.
 * NEIGHBOR (x edges, set only by lbm_batch_link_x): the pull across the edge reads the
 * adjacent column of another resident domain of the batch (slab decomposition of one
 * grid). */
typedef enum { LBM_PERIODIC = 0, LBM_INLET_EQ = 1, LBM_OUTFLOW_ZG = 2, LBM_FREE_SLIP = 3,
               LBM_NEIGHBOR = 4 } lbm_edge;

/* Rigid body k (1-based id in the mask): obstacle velocity
 * U_O(x) = (vx, vy) + omega * z x (x - (cx, cy))  (Eq. boundary-condition, Sec. 2.2).
 * ref_length (D or chord) is carried for force coefficients only. */
typedef struct {
  double cx, cy, vx, vy, omega, ref_length;
} lbm_body;

typedef enum {
  LBM_SHAPE_CIRCLE = 0,          /* chi = 1 where |x - c|^2 <  r^2 */
  LBM_SHAPE_ANNULUS_OUTSIDE = 1, /* chi = 1 where |x - c|^2 >  r^2 (Couette outer wall) */
  LBM_SHAPE_NACA4 = 2            /* NACA 00tt, quarter chord at c, nose-up aoa > 0 */
} lbm_shape_kind;

/* One obstacle shape of the mask function chi (Eq. mask function); tested at node
 * positions in FP64. body is the id written where chi = 1 (1..255); later shapes
 * overwrite earlier ones. NACA half thickness: 5 t c (0.2969 sqrt(x) - 0.1260 x -
 * 0.3516 x^2 + 0.2843 x^3 - 0.1015 x^4), x = x'/c, inside when 0 <= x' <= c and
 * |y'| <= y_t. */
typedef struct {
  int32_t kind, body;
  double cx, cy, radius;
  double chord, thickness, aoa_rad;
} lbm_shape;

typedef struct {
  const lbm_shape *shapes; /* host array */
  int32_t nshapes;
} lbm_geometry;

/* Problem parameters (Sec. 2: grid, nu or tau, Lambda, eta, U_in, initial state). */
typedef struct {
  int32_t nx, ny;         /* grid size, each >= 3 */
  double nu;              /* > 0: tau_plus = nu / c_s^2 + 1/2; else tau_plus is used */
  double tau_plus;        /* symmetric relaxation time tau_s, > 1/2 */
  double magic_lambda;    /* Lambda = (tau_s - 1/2)(tau_a - 1/2) > 0 */
  double eta;             /* penalization parameter, > 0 */
  double rho0;            /* reference density (> 0) */
  double u_in_x, u_in_y;  /* inlet velocity of an INLET_EQ west edge */
  double u0_x, u0_y;      /* uniform initial velocity: g = f^eq(rho0, u0) everywhere */
  int32_t west, east, south, north; /* lbm_edge */
  int32_t storage;        /* lbm_storage */
  int32_t force_every;    /* record body forces every k-th step (0: never) */
  int32_t force_capacity; /* force-ring entries kept on the device (0: 8192) */
  int32_t moving;         /* 1: the bodies move (prescribed translation): at step index n
                           * body k is centred at c_k + V_k n and its shapes are translated
                           * by V_k n (chi(x, t), U_O(x, t) of Sec. 2.2; rotation acts through
                           * U_O only). 2: the bodies also turn their shapes: body k has
                           * turned by theta = omega_k n about its centre c_k + V_k n, a shape
                           * whose reference point (circle centre, NACA quarter chord) is
                           * offset by d from c_k sits at c_k + V_k n + R(theta) d, and a NACA
                           * section's angle of attack is aoa - theta; sin and cos of theta are
                           * evaluated in FP64 by a fixed sequence of rounded operations
                           * (reduction by pi/2 split in three parts, Taylor series to r^17),
                           * within 2 ulp of the exact values for |theta| < 1.3e7. Coupled
                           * bodies need moving = 1. Needs device geometry (no host mask), at
                           * most 64 shapes and 8 bodies. 0: fixed mask. */
  int32_t x_origin;       /* global column of local column 0: a domain that is one slab of
                           * a larger grid rasterises its shapes and evaluates U_O at the
                           * global position (i + x_origin, j), so slabs reproduce the
                           * undivided grid bit for bit. 0 for an undivided domain. With
                           * 16-bit storage it must be divisible by 8: the stochastic
                           * rounding bits are keyed by global 8-column groups. */
} lbm_params;

typedef void *(*lbm_alloc_fn)(size_t bytes, void *ctx);
typedef void (*lbm_free_fn)(void *ptr, void *ctx);

typedef struct lbm_domain lbm_domain;
typedef struct lbm_batch lbm_batch;

/* Fill p with defaults: 64x64, nu = 0.1, Lambda = 3/16, eta = 1e-4, rho0 = 1, periodic,
 * FP32 storage, forces every step, 8192-entry ring. */
LBM_API void lbm_params_default(lbm_params *p);

LBM_API const char *lbm_status_string(lbm_status s);
LBM_API const char *lbm_last_error(void);

/* Device bytes one domain with these parameters occupies (populations x2, mask,
 * solid-node list bound, force ring). Used for admission by memory budget. */
LBM_API size_t lbm_domain_bytes(const lbm_params *p, int32_t nbodies);

/* ---- single domain ---------------------------------------------------------------- */

/* Create a domain on the current CUDA device.
 *  body_mask_host: nx*ny bytes, row-major [ny][nx], 0 = fluid, k = body k; or NULL to
 *                  rasterise `geom` on the device (Eq. mask function).
 *  bodies:         host array of nbodies rigid bodies (nbodies <= 255; every mask id
 *                  must be <= nbodies).
 *  cuda_stream:    cudaStream_t all work is ordered on (NULL: legacy default stream).
 *  alloc/free/ctx: device allocator (both NULL: cudaMallocAsync/cudaFreeAsync).
 * Initial state: g = f^eq(rho0, u0) at every node (step (1) of the algorithm).
 * Synchronises once (the solid-node count sizes the force reducer's list). */
LBM_API lbm_status lbm_domain_create(const lbm_params *p, const uint8_t *body_mask_host,
                             const lbm_geometry *geom, const lbm_body *bodies,
                             int32_t nbodies, void *cuda_stream, lbm_alloc_fn alloc,
                             lbm_free_fn free_fn, void *alloc_ctx, lbm_domain **out);

/* Advance nsteps time steps (steps (2)-(6), repeated). Asynchronous: divergence is
 * reported by the next synchronising call (lbm_forces, lbm_moments). Returns
 * LBM_EBUSY, doing nothing, if the undrained force entries would exceed the ring. */
LBM_API lbm_status lbm_step(lbm_domain *d, int64_t nsteps);

/* Drain recorded body forces into host `out` as [entries][nbodies][2] doubles (force
 * ON body k: -sum of F_VP over its nodes, Sec. 3 drag/lift sums with the sign read
 * as the force on the body). Copies min(available, max_entries) oldest entries and
 * sets *written. Synchronises the stream. Returns LBM_EUNSTABLE if diverged. */
LBM_API lbm_status lbm_forces(lbm_domain *d, double *out, int64_t max_entries, int64_t *written);

/* Macroscopic fields of the current state, [ny][nx] FP64 each: rho and u = u* + du of
 * the streamed populations (Eq. rho, Eq. velocity-r). Host or device pointers; any
 * may be NULL. Synchronises the stream. */
LBM_API lbm_status lbm_moments(lbm_domain *d, double *rho, double *ux, double *uy);

/* Raw current populations in the storage type, [9][ny][nx] (element size 8, 4, 2, 2
 * for F64, F32, F16S, BF16S; F16S holds 1024 (f - w rho0), BF16S f - w rho0). bytes must equal
 * 9*nx*ny*element size. Host or device pointers. Synchronise the stream. */
LBM_API lbm_status lbm_get_populations(lbm_domain *d, void *out, size_t bytes);
LBM_API lbm_status lbm_set_populations(lbm_domain *d, const void *in, size_t bytes);

/* lbm_moments without any device allocation, for callers that cannot let the library
 * allocate when they read the fields: an application whose own arena or caching
 * allocator owns all device memory, a monitoring loop that cannot afford an
 * allocation's latency or implicit device synchronisation, or code that must keep its
 * device footprint fixed after start-up. The paper has no counterpart; this is a
 * service of the library.
 *  - Same outputs as lbm_moments (host or device pointers, any may be NULL; synchronises).
 *  - The fields are staged in one fixed device array owned by the library, 3 * 2^18
 *    doubles (6 MiB), which every GPU that loads the library holds until exit; domains
 *    with more than 2^18 = 262144 nodes are rejected with LBM_EINVAL.
 *  - lbm_domain_create looks up the array's device address for its device (once per
 *    device; with CUDA's lazy module loading that is also when the array's 6 MiB are
 *    taken), so calls on such a domain load nothing. Should that look-up have failed,
 *    the first call retries it (for the current device, which must be the domain's):
 *    make that first call before any stream capture.
 *  - Every call, from any domain, reuses the same array; calls whose work overlaps on the
 *    GPU (different streams, no ordering between them) race on it and must be serialised
 *    by the caller. Each call overwrites every value it reads back, so nothing needs to
 *    start at zero. */
LBM_API lbm_status lbm_moments_noalloc(lbm_domain *d, double *rho, double *ux, double *uy);

/* The body-id mask chi of Eq. (mask function) as used by the sweep, [ny][nx] bytes,
 * 0 = fluid, k = body k. Host or device pointer. Synchronises the stream. */
LBM_API lbm_status lbm_get_mask(lbm_domain *d, uint8_t *out);

/* Steps done so far (the step index of the next step). */
LBM_API lbm_status lbm_steps_done(lbm_domain *d, int64_t *steps);

/* Sets the step index (steps >= 0). The step index keys the random bits of the 16-bit
 * storages' rounding and the force-series entries, so a run resumed from saved
 * populations reproduces the uninterrupted run bit for bit when the index is restored
 * with them. Force entries not yet read by lbm_forces are discarded. LBM_EINVAL for a
 * negative index. No counterpart in the paper (a checkpoint facility). */
LBM_API lbm_status lbm_set_steps_done(lbm_domain *d, int64_t steps);

LBM_API lbm_status lbm_domain_destroy(lbm_domain *d);

/* ---- batches of uneven domains (continuous batching) ----------------------------------- */

/* A batch advances many domains of one storage type together: each time step is one
 * persistent launch over a tile work list covering every resident domain, plus one
 * force-reduction launch; steps are replayed from captured CUDA graphs. Unless a domain
 * has coupled bodies, the force reduction of a step runs on a second stream of the
 * library's beside the next step's sweep; every call returns with that stream joined to
 * cuda_stream, so work ordered after a call on cuda_stream sees its results.
 *  max_domains:      slot count (1..4096).
 *  hbm_budget_bytes: admission limit on the sum of lbm_domain_bytes (0: no limit).
 *  graph_steps:      steps per captured graph (0: no graphs, one launch per kernel).
 * The sweep starts with the tile the autotuner picks on a 64-domain batch of uneven
 * cylinder-pair domains: 16-bit storage (vec 8, 12 warps, 4 rows, pipeline 4), FP32
 * (4, 16, 4, 0), FP64 (2, 4, 4, 0); lbm_batch_set_tile / lbm_batch_autotune change it. */
LBM_API lbm_status lbm_batch_create(int32_t max_domains, size_t hbm_budget_bytes, int32_t storage,
                            int32_t graph_steps, void *cuda_stream, lbm_alloc_fn alloc,
                            lbm_free_fn free_fn, void *alloc_ctx, lbm_batch **out);

/* Admit one domain (p->storage must equal the batch's) that will run `nsteps` steps.
 * Mask from body_mask_host or rasterised from geom as in lbm_domain_create. Returns
 * LBM_EBUSY (nothing admitted) if no slot is free or the budget would be exceeded.
 * Synchronises once. */
LBM_API lbm_status lbm_batch_admit(lbm_batch *b, const lbm_params *p, const uint8_t *body_mask_host,
                           const lbm_geometry *geom, const lbm_body *bodies, int32_t nbodies,
                           int64_t nsteps, int32_t *slot);

/* Admit n fixed-geometry domains at once, each rasterised on the device from its
 * geometry (no host masks, no moving domains: use lbm_batch_admit for those): the same
 * state, slots and results as n calls of lbm_batch_admit, with one rasterise/count, one
 * solid-list, one initial-state and two copy launches over the rows of all of them and
 * two synchronisations in all (one to size the solid-node lists from the per-row
 * counts, one at the end), instead of two per domain. params, geoms, nbodies, nsteps:
 * arrays of n; bodies: n pointers to each domain's body table (may be NULL where
 * nbodies is 0). slots[i] receives domain i's slot. All or none: on any error nothing is
 * admitted and every allocation is given back. LBM_EBUSY when fewer than n slots are free
 * or the memory budget would be exceeded; LBM_EINVAL as lbm_batch_admit, with the
 * domain's index in the message. Memory: for n >= 2 the domains' blocks come from one
 * allocation and their solid-node lists from another (two allocator calls in all); an
 * evicted domain's share is returned, and leaves the memory budget, when the last domain
 * of the group leaves. No counterpart in the paper (admission scheduling). */
LBM_API lbm_status lbm_batch_admit_many(lbm_batch *b, int32_t n, const lbm_params *params,
                                        const lbm_geometry *geoms, const lbm_body *const *bodies,
                                        const int32_t *nbodies, const int64_t *nsteps, int32_t *slots);

/* Whether lbm_batch_admit_many takes two allocations for all of its domains (on = 1, the
 * default: fewer allocator calls; a group's memory returns, and leaves the budget, when
 * its last domain leaves) or two per domain (on = 0: each domain's memory returns at its
 * eviction, as after lbm_batch_admit; for a server under a memory budget, whose requests
 * end at different times). Applies to later admissions. No counterpart in the paper. */
LBM_API lbm_status lbm_batch_set_grouped_admission(lbm_batch *b, int32_t on);

/* Advance every resident, unfinished domain by up to max_steps steps; a domain stops
 * at its own nsteps. *steps_run = steps actually run (<= max_steps). Asynchronous.
 * Returns LBM_EBUSY (nothing run) if a domain's force ring cannot hold the entries. */
LBM_API lbm_status lbm_batch_run(lbm_batch *b, int64_t max_steps, int64_t *steps_run);

/* Drain a slot's recorded forces (as lbm_forces); *done = 1 once the slot has run all
 * its steps and its forces are drained. Synchronises the stream. */
LBM_API lbm_status lbm_batch_poll(lbm_batch *b, int32_t slot, double *out, int64_t max_entries,
                          int64_t *written, int32_t *done);

/* lbm_batch_poll for n slots with one synchronisation: their entries and status words
 * reach pinned host memory by asynchronous copies (for n >= 4, one copy launch gathers
 * them into device staging, read back by one transfer): outs[i] receives up to
 * max_entries[i] entries of slot slots[i], [entries][nbodies][2] FP64, written[i] their
 * number, done[i] as lbm_batch_poll, status[i] the slot's own state (LBM_OK, LBM_EUNSTABLE
 * or LBM_ETIMEOUT; a failed slot's entries are still drained). Returns LBM_EINVAL or
 * LBM_ENOTFOUND (nothing drained) for a bad argument, LBM_ENOMEM if the pinned or device
 * staging cannot grow, LBM_ECUDA if a copy fails. No counterpart in the paper (host I/O). */
LBM_API lbm_status lbm_batch_poll_many(lbm_batch *b, int32_t n, const int32_t *slots,
                                       double *const *outs, const int64_t *max_entries,
                                       int64_t *written, int32_t *done, int32_t *status);

/* Per-slot access, as the single-domain calls of the same name. Synchronise. */
LBM_API lbm_status lbm_batch_moments(lbm_batch *b, int32_t slot, double *rho, double *ux, double *uy);
LBM_API lbm_status lbm_batch_get_populations(lbm_batch *b, int32_t slot, void *out, size_t bytes);
LBM_API lbm_status lbm_batch_set_populations(lbm_batch *b, int32_t slot, const void *in, size_t bytes);
LBM_API lbm_status lbm_batch_steps_done(lbm_batch *b, int32_t slot, int64_t *steps);
/* As lbm_set_steps_done; also LBM_EINVAL beyond the slot's admitted step count. */
LBM_API lbm_status lbm_batch_set_steps_done(lbm_batch *b, int32_t slot, int64_t steps);
LBM_API lbm_status lbm_batch_get_mask(lbm_batch *b, int32_t slot, uint8_t *out);

/* Advance every resident, unfinished domain by up to `steps` real time steps launched
 * one kernel at a time (no graphs), bracketing each force and sweep launch with CUDA
 * events on the batch stream. Outputs the mean duration per launch in microseconds
 * (any may be NULL) and the steps run. Synchronises the stream. */
LBM_API lbm_status lbm_batch_profile(lbm_batch *b, int32_t steps, double *sweep_us,
                                     double *force_us, int64_t *steps_run);

/* Slab decomposition of one grid along x: link two resident domains so that the west
 * slab's east edge pulls the first column of the east slab and the east slab's west edge
 * pulls the last column of the west slab (streaming across the cut, Eq. streaming; both
 * read the same time level, as the undivided grid does). The pair needs the same ny and
 * y edges, the same steps done and admitted (they step together in every run) and the
 * same storage (one batch). With lbm_params.x_origin set to each slab's first global
 * column, the slabs reproduce the undivided grid bit for bit (tested); each reports the
 * force on its part of a body. Linking a domain to itself in both directions is the
 * periodic edge. Evicting a slab restores its partner's own edge rule. LBM_EINVAL if the
 * domains do not match or an edge is linked already. No counterpart in the paper. */
LBM_API lbm_status lbm_batch_link_x(lbm_batch *b, int32_t west_slot, int32_t east_slot);

/* Free a slot and its device memory. */
LBM_API lbm_status lbm_batch_evict(lbm_batch *b, int32_t slot);

/* Halo edges: one grid cut into slabs over several devices (or batches). Streaming
 * (Eq. streaming) across a cut pulls, at the same time level, the neighbouring slab's
 * column next to the cut. Only the three populations that cross the cut are needed:
 * e_x = +1 (directions 1, 5, 8) eastward and e_x = -1 (3, 6, 7) westward, for every row.
 * lbm_batch_set_halo turns the x edge `side` (0 west, 1 east) of a slot into a halo
 * edge fed from caller-owned device buffers, both [9][ny] elements of the batch's
 * storage type (element (a, j) at a * ny + j):
 *   recv: read by every later sweep as the column beyond the edge; the caller fills
 *         planes 1, 5, 8 (west edge) or 3, 6, 7 (east edge) before every step with the
 *         neighbour's send buffer for this cut;
 *   send: written by lbm_batch_pack_halos with this slot's own column at the edge,
 *         planes 3, 6, 7 (west edge, column 0) or 1, 5, 8 (east edge, column nx - 1).
 * Per step: lbm_batch_pack_halos, the exchange (device copies, peer copies or NCCL
 * send/recv, ordered on or after the batch stream), then lbm_batch_run of one step. The
 * slabs' x_origin values place each slab in the grid (shapes, obstacle velocities and
 * the 16-bit rounding keyed by global columns), so the slabs reproduce the undivided
 * grid bit for bit. recv = send = NULL restores the edge given at admission. The buffers
 * stay the caller's (not freed by the library) and must outlive their use. LBM_EINVAL if
 * the edge is linked to a slot (lbm_batch_link_x), the slot has coupled or pulsating
 * bodies, or only one buffer is given. No counterpart in the paper (its method is local,
 * Sec. 2.2, which is what lets a grid be cut). */
LBM_API lbm_status lbm_batch_set_halo(lbm_batch *b, int32_t slot, int32_t side, void *recv, void *send);
/* Enqueue on the batch stream the packing of every halo edge's send buffer from the
 * current state (one launch for up to 64 edges). Asynchronous. */
LBM_API lbm_status lbm_batch_pack_halos(lbm_batch *b);

/* Build the work lists of the resident slots and capture the CUDA graph of graph_steps
 * steps now, so that the next lbm_batch_run of at least graph_steps steps replays it
 * instead of capturing it first (capture is host work of a few milliseconds; do it
 * outside latency- or time-critical regions). No step is run. A graph stays valid
 * until the membership of the batch or its tile shape changes. No-op when graph_steps
 * is 0. No counterpart in the paper (launch scheduling). */
LBM_API lbm_status lbm_batch_capture(lbm_batch *b);

/* Host-side failure injection, for tests of the error paths; no GPU fault, trap or hang
 * is raised. No counterpart in the paper.
 *   LBM_INJECT_NONE: clear the injection of later sweep launches.
 *   LBM_INJECT_UNSTABLE: set the slot's "unstable" status bit from the host, in stream
 *     order, as if its sweep had seen a density out of range; the next poll, forces or
 *     moments call of the slot returns LBM_EUNSTABLE (sticky).
 *   LBM_INJECT_WAIT_TIMEOUT: every later launch of the shared-memory-staged sweep
 *     (pipeline 1) takes its timeout path at its first row, after that row's bulk
 *     copies have completed and after waiting for the copies of the row it prefetched,
 *     so no copy is in flight when the block exits; the slots it covered report
 *     LBM_ETIMEOUT (sticky). Other pipelines ignore it.
 * `slot` is used by LBM_INJECT_UNSTABLE only. A captured graph is rebuilt when the
 * injection changes. LBM_EINVAL for an unknown kind, LBM_ENOTFOUND for a free slot. */
typedef enum { LBM_INJECT_NONE = 0, LBM_INJECT_UNSTABLE = 1, LBM_INJECT_WAIT_TIMEOUT = 2 } lbm_inject;
LBM_API lbm_status lbm_batch_inject(lbm_batch *b, int32_t slot, int32_t kind);

/* Time each sweep tile shape (cells per thread, warps per block, rows per warp, row
 * pipeline) on the
 * resident domains for `reps` launches each, keep the fastest and rebuild the work
 * list and graphs. The timing launches write only the spare lattice, so the state is
 * untouched. *best_us receives the best time per sweep launch (may be NULL). */
LBM_API lbm_status lbm_batch_autotune(lbm_batch *b, int32_t reps, double *best_us);

/* Set the sweep tile shape explicitly: vec = cells per thread (F64 1|2, F32 2|4,
 * F16S/BF16S 4|8), warps = warps per block (1..16), rows = rows per warp (1..16),
 * pipeline = 0 (rows read straight into registers), 1 (rows staged through shared
 * memory by bulk asynchronous copies, one row ahead), 2 (the next row's loads issued
 * into a second register set before the current row is updated; at most 8 warps per
 * block), 3 or 4 (as 0, compiled for 20 or 24 resident warps per SM: at most 10 or 12
 * warps per block, fewer registers per thread). Results do not depend on it. */
LBM_API lbm_status lbm_batch_set_tile(lbm_batch *b, int32_t vec, int32_t warps, int32_t rows,
                                      int32_t pipeline);
LBM_API lbm_status lbm_batch_get_tile(lbm_batch *b, int32_t *vec, int32_t *warps, int32_t *rows,
                                      int32_t *pipeline);

/* Resident slots and cells, and kernel launches issued since creation (sweeps, force
 * reductions, graph replays count each captured kernel). Any output may be NULL. */
LBM_API lbm_status lbm_batch_info(lbm_batch *b, int32_t *resident, int64_t *cells,
                          int64_t *kernel_launches, size_t *bytes_in_use);

LBM_API lbm_status lbm_batch_destroy(lbm_batch *b);

/* ---- Fluid-structure coupling (moving domains) -----------------------------------------
 * The paper prescribes the obstacle velocity U_O (Sec. 2.2) for rigid obstacles; here a
 * body of a moving domain may instead respond to its force. It is a rigid body of mass M
 * on springs (k_x, k_y) anchored at its initial centre x0, with dampers (c_x, c_y). After
 * every step each free axis advances by semi-implicit Euler with dt = 1, in FP64, each
 * operation rounded in this order:
 *     Fm = (F_n + F_{n-1}) / 2,   v <- v + (Fm - k (x - x0) - c v) / M,   x <- x + v,
 * F_n the force on the body of step n (-sum of F_VP over its nodes, Eq. hydrodynamic
 * force), F_{-1} = 0. The two-step mean cancels a component of F_n that alternates every
 * step (with eta -> 0 the penalization reflects the interior fluid velocity about U_O);
 * driven by F_n alone a body diverges. An axis that is not free keeps its velocity. The
 * next step's mask, centre and U_O = V + omega x (x - c) use the new state (omega stays as
 * given); shapes translate with the centre. The coupling is explicit: a spring-mounted
 * cylinder is stable at five times the mass of the fluid it displaces and more, not at
 * two (the instability is reported as LBM_EUNSTABLE once the density leaves its range). */
typedef struct {
  double mass;              /* M > 0 */
  double stiffness[2];      /* k_x, k_y >= 0 */
  double damping[2];        /* c_x, c_y >= 0 */
  int32_t free_axis[2];     /* 1: the axis responds to the force, 0: it keeps its velocity */
} lbm_body_dynamics;

/* Give body `body` (1-based) of a slot dynamics. The slot must be a moving domain that
 * records the force of every step (force_every = 1), has not stepped yet and is not
 * linked; LBM_EINVAL otherwise (the domain is unchanged). Such a slot cannot change its
 * step index afterwards (lbm_batch_set_steps_done to another index is LBM_EINVAL) nor be
 * linked. Synchronises. */
LBM_API lbm_status lbm_batch_set_dynamics(lbm_batch *b, int32_t slot, int32_t body,
                                          const lbm_body_dynamics *dyn);
LBM_API lbm_status lbm_set_dynamics(lbm_domain *d, int32_t body, const lbm_body_dynamics *dyn);

/* ---- Deforming obstacles (moving domains) ----------------------------------------------
 * Sec. 2.2 lets the mask chi and U_O depend on time; here a body of a moving domain may
 * pulsate about its centre: at step index n its shapes are scaled by
 *     s(n) = 1 + a sin(nu n),   |a| < 1,
 * radii and NACA chords by s(n) (the thickness ratio is kept) and each shape's offset d from
 * the body's reference centre to s(n) d (s(n) R(theta) d in a rotating domain), and U_O at
 * its nodes adds the velocity of that dilation, kappa(n) (x - c), kappa = s'/s =
 * a nu cos(nu n) / s(n), in FP64 in that order (sin and cos as for rotating domains). Set
 * before the first step of a moving slot that is not linked and has no coupled body
 * (LBM_EINVAL otherwise); it re-places the slot's mask at index 0. Synchronises. */
LBM_API lbm_status lbm_batch_set_deformation(lbm_batch *b, int32_t slot, int32_t body, double amplitude,
                                             double rate);
LBM_API lbm_status lbm_set_deformation(lbm_domain *d, int32_t body, double amplitude, double rate);

/* The body table of the slot's current step into host `out`, [nbodies][5] doubles: centre
 * x, y, velocity x, y, angular velocity (for coupled bodies the integrated state; for
 * prescribed motion c + V n). Synchronises. */
LBM_API lbm_status lbm_batch_body_state(lbm_batch *b, int32_t slot, double *out);
LBM_API lbm_status lbm_body_state(lbm_domain *d, double *out);

/* Checkpoint of a slot with coupled bodies: the full state of its current step into host
 * `out`, [nbodies][6] doubles (x, y, vx, vy and the force of the previous step Fx, Fy;
 * rows of bodies without dynamics are zero). Synchronises. */
LBM_API lbm_status lbm_batch_coupled_state(lbm_batch *b, int32_t slot, double *out);
LBM_API lbm_status lbm_coupled_state(lbm_domain *d, double *out);

/* Resume a slot with coupled bodies at step index `steps` (with its populations restored
 * by lbm_batch_set_populations): `in` is a state written by lbm_batch_coupled_state at
 * that index. Sets the step index, the bodies' state and table, and the mask of that
 * geometry; undrained force entries are dropped. The resumed run repeats the original
 * bit for bit. LBM_EINVAL if the slot has no coupled body or steps is outside
 * [0, admitted steps]. Synchronises. */
LBM_API lbm_status lbm_batch_restore_coupled(lbm_batch *b, int32_t slot, int64_t steps, const double *in);
LBM_API lbm_status lbm_restore_coupled(lbm_domain *d, int64_t steps, const double *in);

/* ---- 3D: D3Q19 / D3Q15 TRT-LBM-VP (single domain) ------------------------------------
 * The paper's closing remark: the method extends to 3D by replacing D2Q9 with D3Q15 or
 * D3Q19. This is the step of Sec. 2.2 with either lattice. D3Q19: e_0 = 0; e_1..6 = +x,
 * -x, +y, -y, +z, -z; e_7..18 the face diagonals (+x+y, -x-y, +x-y, -x+y, +x+z, -x-z,
 * +x-z, -x+z, +y+z, -y-z, +y-z, -y+z); weights 1/3, 1/18, 1/36. D3Q15: e_0..6 as D3Q19;
 * e_7..14 the cube corners (+x+y+z, -x-y-z, +x+y-z, -x-y+z, +x-y+z, -x+y-z, -x+y+z,
 * +x-y-z); weights 2/9, 1/9, 1/72. Directions 2m-1 and 2m are opposite. Populations
 * [Q][nz][ny][nx] (Q = 19 or 15); storage types, their rounding and the F16S scale as
 * for 2D. Edges: x as in 2D (PERIODIC / INLET_EQ west, PERIODIC / OUTFLOW_ZG east); y (south,
 * north) and z (bottom, top) PERIODIC or FREE_SLIP; rules applied x, then y, then z.
 * U_O = V + omega x (x - c) with an angular velocity vector. */
typedef struct {
  int32_t nx, ny, nz;       /* grid size, each >= 3 */
  double nu;                /* > 0: tau_plus = nu / c_s^2 + 1/2; else tau_plus is used */
  double tau_plus, magic_lambda, eta, rho0;
  double u_in[3];           /* inlet velocity of an INLET_EQ west edge */
  double u0[3];             /* uniform initial velocity */
  int32_t west, east, south, north, bottom, top; /* lbm_edge */
  int32_t storage;          /* lbm_storage */
  int32_t force_every;      /* record body forces every k-th step (0: never) */
  int32_t force_capacity;   /* force-ring entries kept on the device (0: 8192) */
  int32_t lattice;          /* 19 (or 0): D3Q19; 15: D3Q15 */
  int32_t moving;           /* 0 or 1: bodies translate with their velocities (at most 8 bodies,
                               64 shapes, |V| <= 1 per axis): body k is centred at
                               c_k + V_k n at step index n, its shapes translated by V_k n,
                               the mask recomputed after every step; positions are not
                               wrapped at periodic edges */
} lbm3_params;

typedef struct {
  double c[3], v[3], w[3];  /* centre, velocity, angular velocity */
  double ref_length;        /* for force coefficients only */
} lbm3_body;

typedef enum { LBM3_SHAPE_SPHERE = 0,      /* chi = 1 where |x - c|^2 < r^2 */
               LBM3_SHAPE_CYLINDER_Z = 1   /* chi = 1 where (x - cx)^2 + (y - cy)^2 < r^2 */
} lbm3_shape_kind;

typedef struct {
  int32_t kind, body;       /* body id 1..255 written where chi = 1; later shapes overwrite */
  double c[3], radius;
} lbm3_shape;

typedef struct lbm3_domain lbm3_domain;

/* Defaults: 32^3, nu = 0.1, Lambda = 3/16, eta = 1e-4, rho0 = 1, periodic, FP32,
 * forces every step, 8192-entry ring. */
LBM_API void lbm3_params_default(lbm3_params *p);

/* Device bytes of one 3D domain (populations x2, mask, F_VP field, bodies, force sums,
 * ring). */
LBM_API size_t lbm3_domain_bytes(const lbm3_params *p, int32_t nbodies);

/* Create a 3D domain on the current device: the mask is rasterised on the device from
 * `shapes` (FP64 predicates at node positions), g = f^eq(rho0, u0). Allocation and
 * stream as lbm_domain_create. Synchronises once. */
LBM_API lbm_status lbm3_domain_create(const lbm3_params *p, const lbm3_shape *shapes,
                                      int32_t nshapes, const lbm3_body *bodies, int32_t nbodies,
                                      void *cuda_stream, lbm_alloc_fn alloc, lbm_free_fn free_fn,
                                      void *alloc_ctx, lbm3_domain **out);

/* Advance nsteps time steps (asynchronous; LBM_EBUSY, doing nothing, if the undrained
 * force entries would exceed the ring). */
LBM_API lbm_status lbm3_step(lbm3_domain *d, int64_t nsteps);

/* Drain recorded forces into host `out` as [entries][nbodies][3] doubles (force ON body
 * k: -sum of F_VP over its nodes). Synchronises. LBM_EUNSTABLE if diverged. */
LBM_API lbm_status lbm3_forces(lbm3_domain *d, double *out, int64_t max_entries, int64_t *written);

/* rho and u = u* + du of the current state, [nz][ny][nx] FP64 each (host or device
 * pointers, any may be NULL). Synchronises. */
LBM_API lbm_status lbm3_moments(lbm3_domain *d, double *rho, double *ux, double *uy, double *uz);

/* Raw populations [Q][nz][ny][nx] in the storage type; bytes must equal
 * Q nx ny nz element size (Q = 19 or 15). Synchronise. */
LBM_API lbm_status lbm3_get_populations(lbm3_domain *d, void *out, size_t bytes);
LBM_API lbm_status lbm3_set_populations(lbm3_domain *d, const void *in, size_t bytes);

/* The body-id mask [nz][ny][nx]; steps done so far. */
LBM_API lbm_status lbm3_get_mask(lbm3_domain *d, uint8_t *out);
LBM_API lbm_status lbm3_steps_done(lbm3_domain *d, int64_t *steps);

/* Set the step index (>= 0), e.g. with populations restored by lbm3_set_populations: the
 * 16-bit storages draw their rounding bits from the step index, so a resumed run repeats
 * the original one bit for bit. Undrained force entries are dropped; later entries
 * count from the new index. Synchronises. */
LBM_API lbm_status lbm3_set_steps_done(lbm3_domain *d, int64_t steps);

/* Coupled bodies in 3D: the 2D fluid-structure coupling above on three axes. Body k of a
 * moving domain with dynamics is a rigid body of mass M on springs (k_x, k_y, k_z)
 * anchored at its initial centre, with dampers (c_x, c_y, c_z); after every step each free
 * axis advances, in FP64 and rounded in this order,
 *     Fm = (F_n + F_{n-1}) / 2,   v <- v + (Fm - k (x - x0) - c v) / M,   x <- x + v,
 * F_n its force of step n (-sum of F_VP over its nodes), F_{-1} = 0; an axis that is not
 * free keeps its velocity. The next step's mask, centre and U_O use the new state (omega
 * stays as given); its shapes translate with the centre, by (x - x0). The |V| <= 1 limit
 * of prescribed motion does not apply to it. */
typedef struct {
  double mass;              /* M > 0 */
  double stiffness[3];      /* k >= 0 per axis */
  double damping[3];        /* c >= 0 per axis */
  int32_t free_axis[3];     /* 1: the axis responds to the force, 0: it keeps its velocity */
} lbm3_body_dynamics;

/* Give body `body` (1-based) dynamics. The domain must be moving, record the force of
 * every step (force_every = 1) and not have stepped yet; LBM_EINVAL otherwise (the domain is
 * unchanged). Such a domain changes its step index only through lbm3_restore_coupled
 * (lbm3_set_steps_done to another index is LBM_EINVAL). Synchronises. */
LBM_API lbm_status lbm3_set_dynamics(lbm3_domain *d, int32_t body, const lbm3_body_dynamics *dyn);

/* A body of a moving 3D domain pulsating about its centre, as lbm_batch_set_deformation in
 * 2D: shapes scaled by s(n) = 1 + a sin(nu n) (|a| < 1), radii and each shape's offset from
 * the body's reference centre; U_O adds kappa (x - c), kappa = a nu cos(nu n) / s(n). The
 * dilation is isotropic, so the body must be made of spheres. Set before the first step,
 * not with coupled bodies (LBM_EINVAL otherwise); it re-places the mask at index 0.
 * Synchronises. */
LBM_API lbm_status lbm3_set_deformation(lbm3_domain *d, int32_t body, double amplitude, double rate);

/* The body table of the current step into host `out`, [nbodies][9] doubles: centre,
 * velocity, angular velocity (coupled bodies: the integrated state; prescribed motion:
 * c + V n). Synchronises. */
LBM_API lbm_status lbm3_body_state(lbm3_domain *d, double *out);

/* Checkpoint of a domain with coupled bodies: the state of its current step into host
 * `out`, [nbodies][9] doubles (x[3], v[3] and the previous step's force F[3]; rows of
 * bodies without dynamics are zero). Synchronises. LBM_EINVAL if no body is coupled. */
LBM_API lbm_status lbm3_coupled_state(lbm3_domain *d, double *out);

/* Resume at step index `steps` >= 0 (populations restored by lbm3_set_populations): `in`
 * is a state written by lbm3_coupled_state at that index. Sets the step index, the bodies'
 * state and table and the mask of that geometry; undrained force entries are dropped. The
 * resumed run repeats the original bit for bit. LBM_EINVAL if no body is coupled.
 * Synchronises. */
LBM_API lbm_status lbm3_restore_coupled(lbm3_domain *d, int64_t steps, const double *in);

/* Run `steps` steps bracketing the sweep and the force reduction of each with CUDA
 * events; mean microseconds per launch (either output may be NULL). */
LBM_API lbm_status lbm3_profile(lbm3_domain *d, int32_t steps, double *sweep_us, double *force_us);

/* The 3D sweep's register budget: pipeline 0 (16-bit storage: 16 resident warps per SM at
 * 128 registers; FP32/FP64: 12 warps at 168), 3 or 4 (16-bit storage only: 20 or 24
 * resident warps per SM at 102 or 85 registers). A new domain starts at pipeline 3 for
 * 16-bit D3Q15 and 0 otherwise (the faster on a 384 x 128 x 128 sphere channel). With
 * 16-bit storage the sweep's warps
 * take strips from a device counter, otherwise every (grid warps)-th strip. Results do
 * not depend on it. LBM_EINVAL for another value or a pipeline the storage does not
 * have. */
LBM_API lbm_status lbm3_set_tile(lbm3_domain *d, int32_t pipeline);
LBM_API lbm_status lbm3_get_tile(lbm3_domain *d, int32_t *pipeline);

/* Time each pipeline the storage has on the domain for `reps` sweep launches each (two
 * more untimed) and keep the fastest. The timing launches read the current lattice and
 * write only the spare one, so the state is untouched. *best_us receives the best time
 * per sweep launch (may be NULL). Synchronises. */
LBM_API lbm_status lbm3_autotune(lbm3_domain *d, int32_t reps, double *best_us);

LBM_API lbm_status lbm3_domain_destroy(lbm3_domain *d);

/* ---- batches of 3D domains --------------------------------------------------------------
 * A 3D batch advances many fixed-geometry 3D domains of one storage type and one lattice
 * together (the 2D batch's recipe for Sec. 2.2's 3D step): each time step is one
 * persistent sweep launch per group of up to 16 domains with steps left, whose warps take
 * strips of every domain of the group from one device counter (the domains' parameters
 * travel in the launch's), then one force-reduction launch per group. Every result is
 * that of the same domain run alone (lbm3_step), bit for bit.
 *  max_domains: slots (1..4096); hbm_budget_bytes: admission limit on the sum of
 *  lbm3_domain_bytes (0: none); storage, lattice (19 or 15) of every domain; memory from the
 *  allocator callbacks (both NULL: stream-ordered cudaMallocAsync), launches on
 *  cuda_stream. LBM_EINVAL for an argument out of range. */
typedef struct lbm3_batch lbm3_batch;
LBM_API lbm_status lbm3_batch_create(int32_t max_domains, size_t hbm_budget_bytes, int32_t storage,
                                     int32_t lattice, void *cuda_stream, lbm_alloc_fn alloc,
                                     lbm_free_fn free_fn, void *alloc_ctx, lbm3_batch **out);

/* Admit a domain (arguments as lbm3_domain_create) that runs `nsteps` steps; *slot
 * receives its slot. LBM_EINVAL for another storage or lattice than the batch's, or a
 * moving domain (p->moving != 0); LBM_EBUSY when every slot is taken or the budget would
 * be exceeded. Synchronises. */
LBM_API lbm_status lbm3_batch_admit(lbm3_batch *b, const lbm3_params *p, const lbm3_shape *shapes,
                                    int32_t nshapes, const lbm3_body *bodies, int32_t nbodies,
                                    int64_t nsteps, int32_t *slot);

/* Enqueue up to max_steps steps of every resident domain with steps left (asynchronous);
 * *steps_run receives the steps enqueued (0: nothing left). LBM_EBUSY, enqueueing
 * nothing, if a domain's undrained force entries would exceed its ring. */
LBM_API lbm_status lbm3_batch_run(lbm3_batch *b, int64_t max_steps, int64_t *steps_run);

/* Drain a slot's force entries as lbm3_forces does ([entry][body][3], FP64, into host
 * memory); *done = 1 once the slot reached its step target. Synchronises.
 * LBM_EUNSTABLE if the domain diverged; LBM_ENOTFOUND for a free slot. */
LBM_API lbm_status lbm3_batch_poll(lbm3_batch *b, int32_t slot, double *out, int64_t max_entries,
                                   int64_t *written, int32_t *done);

/* The slot's domain, for lbm3_get_populations, lbm3_set_populations, lbm3_moments,
 * lbm3_get_mask and lbm3_steps_done. It stays owned by the batch: do not step, destroy
 * or change its step index through the lbm3_* calls. */
LBM_API lbm_status lbm3_batch_domain(lbm3_batch *b, int32_t slot, lbm3_domain **out);

/* Free a slot and its device memory (synchronises). LBM_ENOTFOUND for a free slot. */
LBM_API lbm_status lbm3_batch_evict(lbm3_batch *b, int32_t slot);

/* The batched sweep's register budget, as lbm3_set_tile (a new batch takes pipeline 3
 * for 16-bit D3Q15, 0 otherwise). Results do not depend on it. */
LBM_API lbm_status lbm3_batch_set_tile(lbm3_batch *b, int32_t pipeline);

/* Resident slots and cells, kernel launches enqueued by lbm3_batch_run, bytes admitted
 * and the current pipeline. Any output may be NULL. */
LBM_API lbm_status lbm3_batch_info(lbm3_batch *b, int32_t *resident, int64_t *cells,
                                   int64_t *launches, size_t *bytes, int32_t *pipeline);

/* Destroy the batch and every resident domain (synchronises). NULL is a no-op. */
LBM_API lbm_status lbm3_batch_destroy(lbm3_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* PAPER_1901_08766_GB300_LBM_H */
