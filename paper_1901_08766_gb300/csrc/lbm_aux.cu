// Auxiliary kernels of the TRT-LBM-VP library: geometry -> mask rasteriser (Eq. mask
// function), initial state (step (1)), solid-node lists, the FP64 body-force reducer
// (Sec. 3 drag and lift sums) and the moments export.
#include "lbm_cell.cuh"
#include "lbm_turn.cuh"

namespace lbm {

// ---- rasteriser ------------------------------------------------------------------------
// Node (i, j) is tested at (i, j) in FP64 with explicitly rounded operations (no
// contraction), so the predicate takes the same decision as a plain IEEE evaluation of
// the same expressions on the host.

__device__ __forceinline__ double naca_half_thickness(double xc, double t, double chord) {
  const double s = __dsqrt_rn(xc);
  double p = __dadd_rn(__dmul_rn(-0.1015, xc), 0.2843);
  p = __dsub_rn(__dmul_rn(p, xc), 0.3516);
  p = __dsub_rn(__dmul_rn(p, xc), 0.1260);
  p = __dmul_rn(p, xc);
  return __dmul_rn(__dmul_rn(__dmul_rn(5.0, t), chord), __dadd_rn(__dmul_rn(0.2969, s), p));
}

__device__ __forceinline__ bool inside(const ShapeDev &s, double x, double y) {
  if (s.kind == LBM_SHAPE_CIRCLE || s.kind == LBM_SHAPE_ANNULUS_OUTSIDE) {
    const double dx = __dsub_rn(x, s.cx), dy = __dsub_rn(y, s.cy);
    const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    const double r2 = __dmul_rn(s.radius, s.radius);
    return s.kind == LBM_SHAPE_CIRCLE ? (d2 < r2) : (d2 > r2);
  }
  if (s.kind == LBM_SHAPE_NACA4) {
    const double qc = __dmul_rn(0.25, s.chord);
    const double lex = __dsub_rn(s.cx, __dmul_rn(qc, s.ca));
    const double ley = __dadd_rn(s.cy, __dmul_rn(qc, s.sa));
    const double dx = __dsub_rn(x, lex), dy = __dsub_rn(y, ley);
    const double xp = __dsub_rn(__dmul_rn(dx, s.ca), __dmul_rn(dy, s.sa));
    const double yp = __dadd_rn(__dmul_rn(dx, s.sa), __dmul_rn(dy, s.ca));
    if (!(xp >= 0.0 && xp <= s.chord)) return false;
    const double yt = naca_half_thickness(__ddiv_rn(xp, s.chord), s.thickness, s.chord);
    return fabs(yp) <= yt;
  }
  return false;
}

__global__ void rasterize_kernel(uint8_t *mask, int nx, int ny, int pitch,
                                 const ShapeDev *shapes, int nshapes, int x0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= pitch || j >= ny) return;
  uint8_t b = 0;
  if (i < nx) {
    for (int k = 0; k < nshapes; ++k)
      if (inside(shapes[k], double(i + x0), double(j))) b = static_cast<uint8_t>(shapes[k].body);
  }
  mask[static_cast<size_t>(j) * pitch + i] = b;
}

cudaError_t launch_rasterize(cudaStream_t st, uint8_t *mask, int nx, int ny, int pitch,
                             const ShapeDev *shapes, int nshapes, int x0) {
  dim3 grid((pitch + 255) / 256, ny);
  rasterize_kernel<<<grid, 256, 0, st>>>(mask, nx, ny, pitch, shapes, nshapes, x0);
  return cudaGetLastError();
}

// ---- moving domains (prescribed translation, turning and pulsating shapes) ------------------
// chi(x, t) and U_O(x, t) of a domain whose bodies translate (Sec. 2.2): at step index n
// body k is centred at c_k + V_k n and each of its shapes is translated by V_k n (turned
// by omega_k n about the centre in a rotating domain, scaled by s_k(n) for a pulsating
// body: shape_turned below). The
// step from n to n + 1 uses the geometry of index n; after its sweep, one warp per row
// (a fixed mapping, so the result does not depend on the launch) first sums -F_VP over
// the row's nodes of each body under the mask the sweep used (FP64, lane-strided then a
// fixed shuffle tree; the force kernel adds the rows in order), then rewrites the row's
// mask for index n + 1. Both touch only the columns that some shape reaches (its
// reference point within radius or chord + 1) at index n or n + 1: nothing else can be
// solid (a turning or pulsating shape: within its grown reach of the body centre). Each
// node is read and rewritten by the same lane. The warp of row 0 moves the body table.
// Positions are c + V n with explicitly rounded FP64 operations, as a plain evaluation on
// the host computes them.

constexpr int kMoveWarps = 8;

__device__ __forceinline__ double moved(double c0, double v, long long n) {
  return __dadd_rn(c0, __dmul_rn(v, static_cast<double>(n)));
}

// Shape s0 of a domain at index n (translated with its body) and its column interval in
// row j: a node farther than the shape's reach from its reference point is outside it
// (lo > hi: the row misses the shape; the outside-annulus kind spans every column).
__device__ __forceinline__ bool coupled(const DomDev &D, int body) {
  return D.fsi_on && body >= 1 && body <= D.nbodies && D.fsi_par[8 * (body - 1) + 7] != 0.0;
}

// a shape of a coupled body, its body's centre at (cx, cy): translated by the centre's
// displacement from the reference centre
__device__ __forceinline__ ShapeDev shape_about(const DomDev &D, const ShapeDev &s0, double cx, double cy) {
  ShapeDev s = s0;
  s.cx = __dadd_rn(s0.cx, __dsub_rn(cx, D.centre0[2 * (s0.body - 1)]));
  s.cy = __dadd_rn(s0.cy, __dsub_rn(cy, D.centre0[2 * (s0.body - 1) + 1]));
  return s;
}

__device__ __forceinline__ bool deforms(const DomDev &D, int body) {
  return D.deform != 0u && body >= 1 && body <= D.nbodies && ((D.deform >> ((body - 1) & 31)) & 1u);
}

// scale s(n) = 1 + a sin(nu n) of pulsating body b (0-based)
__device__ __forceinline__ double pulse_scale(const DomDev &D, int b, long long n, double *kappa) {
  const double a = D.dpar[2 * b], nu = D.dpar[2 * b + 1];
  double sn, cs;
  turn_sincos(__dmul_rn(nu, static_cast<double>(n)), sn, cs);
  const double sc = __dadd_rn(1.0, __dmul_rn(a, sn));
  if (kappa) *kappa = __ddiv_rn(__dmul_rn(__dmul_rn(a, nu), cs), sc);  // s'/s
  return sc;
}

// A rotating domain (moving = 2) turns body b's shapes by theta = omega n about its
// centre c0 + V n, and a pulsating body scales them by s(n) about it: the reference point
// offset d from c0 goes to s(n) R(theta) d, radii and chords to s(n) times theirs, a NACA
// section's (cos, sin) of its angle of attack to those of aoa - theta.
// cos theta, sin theta and the scale of body b (0-based) at step index n, evaluated
__device__ __forceinline__ void turn_of(const DomDev &D, int b, long long n, double &cs, double &sn, double &sc) {
  cs = 1.0;
  sn = 0.0;
  sc = 1.0;
  if (D.moving == 2) turn_sincos(__dmul_rn(D.bodies[5 * b + 4], static_cast<double>(n)), sn, cs);
  if (deforms(D, b + 1)) sc = pulse_scale(D, b, n, nullptr);
}

// The same, stored one step ahead: the body-table update of index m writes index m + 1
// into slot (m + 1) & 1, while the move kernel of the step to m reads slot m & 1
__device__ __forceinline__ void store_turn(const DomDev &D, int b, long long m) {
  double *t = D.turn + (static_cast<size_t>(m & 1) * D.nbodies + b) * 3;
  turn_of(D, b, m, t[0], t[1], t[2]);
}

// table: read cos, sin and scale from the one-step-ahead table (the move kernel's index
// n + 1), else evaluate them (admission, step-index changes)
__device__ __forceinline__ ShapeDev shape_turned(const DomDev &D, const ShapeDev &s0, long long n, bool table) {
  ShapeDev s = s0;
  const int b = s0.body - 1;
  const double *bt = D.bodies + 5 * b;  // vx, vy at 2, 3
  double cs, sn, sc;
  if (table) {
    const double *t = D.turn + (static_cast<size_t>(n & 1) * D.nbodies + b) * 3;
    cs = t[0];
    sn = t[1];
    sc = t[2];
  } else {
    turn_of(D, b, n, cs, sn, sc);
  }
  const double c0x = D.centre0[2 * b], c0y = D.centre0[2 * b + 1];
  const double dx = __dsub_rn(s0.cx, c0x), dy = __dsub_rn(s0.cy, c0y);
  double rx = dx, ry = dy;
  if (D.moving == 2) {
    rx = __dsub_rn(__dmul_rn(cs, dx), __dmul_rn(sn, dy));
    ry = __dadd_rn(__dmul_rn(sn, dx), __dmul_rn(cs, dy));
    s.ca = __dadd_rn(__dmul_rn(s0.ca, cs), __dmul_rn(s0.sa, sn));
    s.sa = __dsub_rn(__dmul_rn(s0.sa, cs), __dmul_rn(s0.ca, sn));
  }
  if (deforms(D, s0.body)) {
    rx = __dmul_rn(sc, rx);
    ry = __dmul_rn(sc, ry);
    s.radius = __dmul_rn(sc, s0.radius);
    s.chord = __dmul_rn(sc, s0.chord);
  }
  s.cx = __dadd_rn(moved(c0x, bt[2], n), rx);
  s.cy = __dadd_rn(moved(c0y, bt[3], n), ry);
  return s;
}

__device__ __forceinline__ ShapeDev shape_at(const DomDev &D, const ShapeDev &s0, long long n, bool table = false) {
  ShapeDev s = s0;
  if ((D.moving == 2 || deforms(D, s0.body)) && s0.body >= 1 && s0.body <= D.nbodies)
    return shape_turned(D, s0, n, table);
  if (coupled(D, s0.body)) {
    const double *st = D.fsi + (static_cast<size_t>(n & 1) * D.nbodies + (s0.body - 1)) * 6;
    return shape_about(D, s0, st[0], st[1]);
  }
  if (s0.body >= 1 && s0.body <= D.nbodies) {
    const double *b = D.bodies + 5 * (s0.body - 1);
    s.cx = moved(s0.cx, b[2], n);
    s.cy = moved(s0.cy, b[3], n);
  }
  return s;
}

__device__ __forceinline__ void shape_cols(const ShapeDev &s, int nx, int x0, int j, int &lo, int &hi) {
  lo = 0;
  hi = nx - 1;
  if (s.kind == LBM_SHAPE_ANNULUS_OUTSIDE) return;
  const double reach = shape_extent(s) + 1.0;
  if (fabs(double(j) - s.cy) > reach) {
    lo = 1;
    hi = 0;
    return;
  }
  // clamped in FP64 first, so that a shape far outside converts safely
  const double lcx = s.cx - double(x0);  // local column of the reference point
  const double dlo = fmin(fmax(floor(lcx - reach), -1.0), double(nx));
  const double dhi = fmin(fmax(ceil(lcx + reach), -1.0), double(nx));
  lo = max(0, static_cast<int>(dlo));
  hi = min(nx - 1, static_cast<int>(dhi));
}

// A shape placed for one row: its geometry, column interval, and the FP32 copies the
// circle pre-test of inside_row uses (converted once per row, not per node: the
// conversions and FP64 compares ran on the FP64 pipe, the move kernel's bottleneck).
struct RowShape {
  ShapeDev s;
  int lo, hi;
  float fcx, fcy, fr2;  // centre and squared radius in FP32
  int fast;             // a circle within the pre-test's bounds
};

// The column interval of shape s0 at index n in row j from FP32 positions with a margin
// of 2 cells: conservative (it contains every node within the shape's reach) while
// positions stay below 10^6 cells and n below 2^24, where the FP32 position error is
// below 0.15 cell. Rows far from every shape thereby cost no FP64 work.
__device__ __forceinline__ void shape_cols_f32(const DomDev &D, int k, long long n, float fn, int j,
                                               int &lo, int &hi) {
  const ShapeDev &s0 = D.shapes[k];
  const float4 f = D.shapes_f[k];  // FP32 centre and extent (no FP64 conversions here)
  lo = 0;
  hi = D.nx - 1;
  if (s0.kind == LBM_SHAPE_ANNULUS_OUTSIDE) return;
  float cx, cy, turn = 0.f;
  if (coupled(D, s0.body)) {
    const ShapeDev s = shape_at(D, s0, n);
    cx = float(s.cx - double(D.x0));
    cy = float(s.cy);
  } else if ((D.moving == 2 || deforms(D, s0.body)) && s0.body >= 1 && s0.body <= D.nbodies) {
    // a turning or pulsating shape stays within (1 + |a|) times its offset from the body
    // centre and (1 + |a|) times its size: cull about the centre with the reach grown by
    // both (no trigonometry here)
    const int b = s0.body - 1;
    cx = (float(D.centre0[2 * b]) - float(D.x0)) + float(D.bodies[5 * b + 2]) * fn;
    cy = float(D.centre0[2 * b + 1]) + float(D.bodies[5 * b + 3]) * fn;
    const float ox = float(s0.cx - D.centre0[2 * b]), oy = float(s0.cy - D.centre0[2 * b + 1]);
    const float grow = deforms(D, s0.body) ? fabsf(float(D.dpar[2 * b])) : 0.f;
    turn = (1.0f + grow) * sqrtf(ox * ox + oy * oy) + grow * f.z + 0.01f;
  } else {
    float vx = 0.f, vy = 0.f;
    if (s0.body >= 1 && s0.body <= D.nbodies) {  // the FP32 copy of the body table
      vx = D.bodies_f[5 * (s0.body - 1) + 2];
      vy = D.bodies_f[5 * (s0.body - 1) + 3];
    }
    cx = (f.x - float(D.x0)) + vx * fn;
    cy = f.y + vy * fn;
  }
  const float reach = f.z + 2.0f + turn;
  if (!(fabsf(float(j) - cy) <= reach)) {
    lo = 1;
    hi = 0;
    return;
  }
  const float flo = fminf(fmaxf(floorf(cx - reach), -1.0f), float(D.nx));
  const float fhi = fminf(fmaxf(ceilf(cx + reach), -1.0f), float(D.nx));
  lo = max(0, static_cast<int>(flo));
  hi = min(D.nx - 1, static_cast<int>(fhi));
}

// The FP32 copies of a row shape's geometry (after r.s is set).
__device__ __forceinline__ void prep_row_shape(RowShape &r) {
  const ShapeDev &s = r.s;
  r.fast = s.kind == LBM_SHAPE_CIRCLE && fabs(s.cx) < 4096.0 && fabs(s.cy) < 4096.0 && s.radius < 100.0;
  r.fcx = float(s.cx);
  r.fcy = float(s.cy);
  r.fr2 = float(s.radius) * float(s.radius);
}

// inside() with an FP32 pre-test for circles: a node whose FP32 squared distance is
// farther than 0.5 from r^2 is decided there, the others take the exact FP64 predicate.
// With centres below 4096 in magnitude (FP32 position error <= 1.2e-4) and radii below
// 100 (|dx|, |dy| <= r + 2 in the column interval), the FP32 error of d^2 is below
// 2 (|dx| + |dy|) 1.2e-4 + 3 d^2 2^-24 < 0.06, so the FP32 decision is the exact one.
__device__ __forceinline__ bool inside_row(const RowShape &r, int i, int j) {
  if (r.fast) {
    const float dx = float(i) - r.fcx, dy = float(j) - r.fcy;
    const float d2 = dx * dx + dy * dy;
    if (d2 < r.fr2 - 0.5f) return true;
    if (d2 > r.fr2 + 0.5f) return false;
  }
  return inside(r.s, double(i), double(j));
}

// Body ids of row j over columns [c0, c1] at the geometry held in rs (warp-wide).
__device__ void write_ids(const DomDev &D, int j, int c0, int c1, int lane, const RowShape *rs) {
  uint8_t *row = D.mask + static_cast<size_t>(j) * D.pitch;
  for (int i = c0 + lane; i <= c1; i += 32) {
    uint8_t id = 0;
    if (i < D.nx)
      for (int k = 0; k < D.nshapes; ++k)
        if (i >= rs[k].lo && i <= rs[k].hi && inside_row(rs[k], i + D.x0, j))
          id = static_cast<uint8_t>(rs[k].s.body);
    row[i] = id;
  }
}

// The whole mask row j at index n (admission and step-index changes).
__device__ void place_row(const DomDev &D, int j, long long n, int lane, RowShape *rs) {
  for (int k = lane; k < D.nshapes; k += 32) {
    rs[k].s = shape_at(D, D.shapes[k], n);
    prep_row_shape(rs[k]);
    shape_cols(rs[k].s, D.nx, D.x0, j, rs[k].lo, rs[k].hi);
  }
  __syncwarp();
  write_ids(D, j, 0, D.pitch - 1, lane, rs);
  __syncwarp();
}

// Body centres at index n (the warp of row 0).
__device__ void place_centres(const DomDev &D, long long n, int lane) {
  if (lane < D.nbodies) {
    double *b = D.bodies + 5 * lane;
    if (coupled(D, lane + 1)) {
      const double *st = D.fsi + (static_cast<size_t>(n & 1) * D.nbodies + lane) * 6;
      for (int e = 0; e < 4; ++e) {
        b[e] = st[e];
        D.bodies_f[5 * lane + e] = float(st[e]);
      }
      return;
    }
    const double cx = moved(D.centre0[2 * lane], b[2], n), cy = moved(D.centre0[2 * lane + 1], b[3], n);
    b[0] = cx;
    b[1] = cy;
    D.bodies_f[5 * lane] = float(cx);
    D.bodies_f[5 * lane + 1] = float(cy);
    if (deforms(D, lane + 1)) {  // the dilation rate of step n
      double kp;
      pulse_scale(D, lane, n, &kp);
      D.kappa[lane] = kp;
      D.kappa_f[lane] = float(kp);
    }
    if (D.moving == 2 || deforms(D, lane + 1)) store_turn(D, lane, n + 1);  // one step ahead
  }
}

// Rows of moving domains, in two launches. The first culls every row (one thread per
// row, FP32 column intervals at n and n + 1) and appends the rows a shape reaches at
// either index, with their intervals, to a list; the second gives each listed row a
// warp for the exact work: the row's -F_VP sums over the mask the sweep used, then its
// mask at index n + 1. (One launch that culled 32 rows per warp and then walked its busy
// rows one after another took as long as its longest walk.) The list's order does not
// matter: each row writes only its own sums and mask row. The culling reads only the
// shapes, so it runs beside the sweep, in 64-thread blocks (at most 64 registers: the
// room one block has on an SM next to the sweep's two).
constexpr int kCullThreads = 64;
__global__ void __launch_bounds__(kCullThreads)
move_cull_kernel(const DomDev *doms, const DomDyn *dyn, const MoveRow *rows, const Counters *ctr,
                 BusyRow *busy, int s) {
  Counters *c = const_cast<Counters *>(ctr);
  const int lane = threadIdx.x & 31;
  const int nrows = ctr->nmove;
  const long long run_base = ctr->run_base;
  const int stride = gridDim.x * blockDim.x;
  // warp-uniform bounds: every lane takes part in the ballot
  for (int base = blockIdx.x * blockDim.x + threadIdx.x - lane; base < nrows; base += stride) {
    const int q = base + lane;
    int olo = 1, ohi = 0, nlo = 1, nhi = 0;
    bool is_busy = false;
    MoveRow mr{0, 0};
    if (q < nrows) {
      mr = rows[q];
      const DomDev &D = doms[mr.dom];
      const DomDyn dy = dyn[mr.dom];
      const long long n = dy.step0 + run_base + s;  // the sweep just computed step n + 1
      if (n < dy.step_end) {
        const bool fsi = D.fsi_on != 0;
        const float fn0 = float(n), fn1 = float(n + 1);
        olo = D.nx; ohi = -1; nlo = D.nx; nhi = -1;
        for (int k = 0; k < D.nshapes; ++k) {
          int lo, hi;
          shape_cols_f32(D, k, n, fn0, mr.j, lo, hi);
          if (lo <= hi) { olo = min(olo, lo); ohi = max(ohi, hi); }
          if (fsi) continue;
          shape_cols_f32(D, k, n + 1, fn1, mr.j, lo, hi);
          if (lo <= hi) { nlo = min(nlo, lo); nhi = max(nhi, hi); }
        }
        // row 0 also moves the body centres (domains without coupled bodies)
        is_busy = olo <= ohi || nlo <= nhi || (mr.j == 0 && !fsi);
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, is_busy);
    if (m != 0u) {
      int at = 0;
      if (lane == 0) at = atomicAdd(&c->nbusy, __popc(m));
      at = __shfl_sync(0xffffffffu, at, 0) + __popc(m & ((1u << lane) - 1u));
      if (is_busy) busy[at] = BusyRow{mr.dom, mr.j, olo, ohi, nlo, nhi};
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kMoveWarps * 32, 4)
move_rows_kernel(const DomDev *doms, const DomDyn *dyn, const MoveRow *rows, const Counters *ctr,
                 const BusyRow *busy, int s) {
  __shared__ RowShape shapes[kMoveWarps][kMaxMovingShapes];
  Counters *c = const_cast<Counters *>(ctr);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  RowShape *rs = shapes[warp];
  const int nbusy = ctr->nbusy;
  const long long run_base = ctr->run_base;
  // consecutive list entries (the consecutive rows a body crosses) go to warps of
  // different blocks, so the busy rows spread over the SMs
  for (int w = warp * static_cast<int>(gridDim.x) + blockIdx.x; w < nbusy; w += gridDim.x * kMoveWarps) {
    const BusyRow br = busy[w];
    const int jolo = br.olo, johi = br.ohi, jnlo = br.nlo, jnhi = br.nhi;
    const DomDev &D = doms[br.dom];
    const DomDyn dy = dyn[br.dom];
    const long long n = dy.step0 + run_base + s;
    const int j = br.j;
    // (a domain with coupled bodies takes only the row sums here: its next geometry
    // depends on the force, and fsi_kernel places it after the force reduction)
    const bool fsi = D.fsi_on != 0;
    const uint8_t *mrow = D.mask + static_cast<size_t>(j) * D.pitch;
    if (D.force_every > 0 && (n + 1) % D.force_every == 0 && jolo <= johi) {
      // -F_VP of each body over the row's solid nodes (all inside the old interval),
      // with the step index as a tag: the force kernel adds only the entries of its
      // step, so rows (or bodies) without solid nodes here need no entry
      // the F_VP field the sweep of step n wrote (the parity of the lattice it read)
      const int par = (dy.parity + static_cast<int>((run_base + s) & 1)) & 1;
      const T *fv = static_cast<const T *>(D.fvp[par]) + 2 * static_cast<size_t>(j) * D.pitch;
      unsigned present = 0u;  // bit b: body b has a node in the interval
      for (int i = jolo + lane; i <= johi; i += 32) present |= 1u << (mrow[i] & 31);
      present = __reduce_or_sync(0xffffffffu, present) & ~1u;
      while (present) {
        const int body = __ffs(present) - 1;
        present &= present - 1;
        double fx = 0.0, fy = 0.0;
        for (int i = jolo + lane; i <= johi; i += 32)
          if (mrow[i] == body) {
            fx -= double(fv[2 * i]);
            fy -= double(fv[2 * i + 1]);
          }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          fx += __shfl_down_sync(0xffffffffu, fx, off);
          fy += __shfl_down_sync(0xffffffffu, fy, off);
        }
        if (lane == 0) {
          double *r = D.rowsum[par] + (static_cast<size_t>(j) * D.nbodies + (body - 1)) * 3;
          r[0] = fx;
          r[1] = fy;
          r[2] = static_cast<double>(n);
        }
      }
    }
    __syncwarp();
    if (fsi) continue;
    // the mask changes only where a shape reaches at either index: the shapes at
    // n + 1 with their column intervals in this row, then their ids over the union
    const int c0 = min(jolo, jnlo), c1 = max(johi, jnhi);
    if (c0 <= c1) {
      for (int k = lane; k < D.nshapes; k += 32) {
        shape_cols_f32(D, k, n + 1, float(n + 1), j, rs[k].lo, rs[k].hi);
        if (rs[k].lo <= rs[k].hi) {  // the shape at n + 1, placed once for all rows
          const PlacedShape &t = D.placed[k];
          rs[k].s = t.s;
          rs[k].fcx = t.fcx;
          rs[k].fcy = t.fcy;
          rs[k].fr2 = t.fr2;
          rs[k].fast = t.fast;
        }
      }
      __syncwarp();
      write_ids(D, j, c0, c1, lane, rs);
    }
    __syncwarp();
    if (j == 0) place_centres(D, n + 1, lane);
  }
  // the last block to finish empties the list for the next step (every block read its
  // length before finishing)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&c->busy_done, 1) == static_cast<int>(gridDim.x) - 1) {
      c->nbusy = 0;
      c->busy_done = 0;
    }
  }
}

// One axis of a coupled body after step n, driven by the mean of the forces of steps n
// and n - 1 (Fp), which cancels the force component that alternates every step (the
// penalized interior's velocity is reflected about U_O each step):
// v <- v + ((F + Fp) / 2 - k (x - x0) - c v) / M, then x <- x + v (semi-implicit Euler,
// dt = 1), each operation rounded as written; an axis that is not free keeps its velocity.
__device__ __forceinline__ void fsi_axis(double F, double Fp, double k, double c, double M, bool free_axis,
                                         double x0, double &x, double &v) {
  if (free_axis) {
    const double Fm = __dmul_rn(__dadd_rn(F, Fp), 0.5);
    double t = __dsub_rn(Fm, __dmul_rn(k, __dsub_rn(x, x0)));
    t = __dsub_rn(t, __dmul_rn(c, v));
    v = __dadd_rn(v, __ddiv_rn(t, M));
  }
  x = __dadd_rn(x, v);
}

// Coupled bodies after step n (launched after the force reduction, which wrote the
// force of step n into ring entry n): every warp advances the bodies of its domain
// from the state of index n (the same operations give the same values in every warp),
// then rewrites its row's mask at index n + 1 where a shape reaches at n or n + 1; the
// warp of row 0 stores the new state (the other parity, so that no warp reads a value
// another warp has replaced) and the body table the next sweep uses.
__global__ void __launch_bounds__(kMoveWarps * 32)
fsi_kernel(const DomDev *doms, const DomDyn *dyn, const MoveRow *rows, const Counters *ctr, int s) {
  __shared__ RowShape shapes[kMoveWarps][kMaxMovingShapes];
  __shared__ double cen[kMoveWarps][kMaxMovingBodies][2];  // centres at index n + 1
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  RowShape *rs = shapes[warp];
  const int nrows = ctr->nmove;
  const long long run_base = ctr->run_base;
  // consecutive rows to warps of different blocks (as in move_rows_kernel)
  for (int q = warp * static_cast<int>(gridDim.x) + blockIdx.x; q < nrows; q += gridDim.x * kMoveWarps) {
    const MoveRow mr = rows[q];
    const DomDev &D = doms[mr.dom];
    if (!D.fsi_on) continue;
    const DomDyn dy = dyn[mr.dom];
    const long long n = dy.step0 + run_base + s;
    if (n >= dy.step_end) continue;
    const int j = mr.j;
    if (lane < D.nbodies) {
      double *b = D.bodies + 5 * lane;
      if (coupled(D, lane + 1)) {
        const double *par = D.fsi_par + 8 * lane;
        const double *st = D.fsi + (static_cast<size_t>(n & 1) * D.nbodies + lane) * 6;
        const double *F = D.ring + (static_cast<size_t>(n % D.force_cap) * D.nbodies + lane) * 2;
        double x = st[0], y = st[1], vx = st[2], vy = st[3];
        const double fx = F[0], fy = F[1];
        fsi_axis(fx, st[4], par[1], par[3], par[0], par[5] != 0.0, D.centre0[2 * lane], x, vx);
        fsi_axis(fy, st[5], par[2], par[4], par[0], par[6] != 0.0, D.centre0[2 * lane + 1], y, vy);
        cen[warp][lane][0] = x;
        cen[warp][lane][1] = y;
        if (j == 0) {
          double *nst = D.fsi + (static_cast<size_t>((n + 1) & 1) * D.nbodies + lane) * 6;
          const double v6[6] = {x, y, vx, vy, fx, fy};
          for (int e = 0; e < 6; ++e) nst[e] = v6[e];
          for (int e = 0; e < 4; ++e) {
            b[e] = v6[e];
            D.bodies_f[5 * lane + e] = float(v6[e]);
          }
        }
      } else if (j == 0) {
        const double cx = moved(D.centre0[2 * lane], b[2], n + 1), cy = moved(D.centre0[2 * lane + 1], b[3], n + 1);
        b[0] = cx;
        b[1] = cy;
        D.bodies_f[5 * lane] = float(cx);
        D.bodies_f[5 * lane + 1] = float(cy);
      }
    }
    __syncwarp();
    // the row's shapes at n + 1 and the columns they or the shapes at n reach (FP64)
    int c0 = D.nx, c1 = -1;
    for (int k = lane; k < D.nshapes; k += 32) {
      const ShapeDev &s0 = D.shapes[k];
      int lo, hi;
      shape_cols(shape_at(D, s0, n), D.nx, D.x0, j, lo, hi);
      if (lo <= hi) { c0 = min(c0, lo); c1 = max(c1, hi); }
      rs[k].s = coupled(D, s0.body) ? shape_about(D, s0, cen[warp][s0.body - 1][0], cen[warp][s0.body - 1][1])
                                    : shape_at(D, s0, n + 1);
      prep_row_shape(rs[k]);
      shape_cols(rs[k].s, D.nx, D.x0, j, rs[k].lo, rs[k].hi);
      if (rs[k].lo <= rs[k].hi) { c0 = min(c0, rs[k].lo); c1 = max(c1, rs[k].hi); }
    }
    c0 = __reduce_min_sync(0xffffffffu, c0);
    c1 = __reduce_max_sync(0xffffffffu, c1);
    __syncwarp();
    if (c0 <= c1) write_ids(D, j, c0, c1, lane, rs);
    __syncwarp();
  }
}

cudaError_t launch_fsi(int grid, cudaStream_t st, const DomDev *doms, const DomDyn *dyn,
                       const MoveRow *rows, const Counters *ctr, int s) {
  fsi_kernel<<<grid, kMoveWarps * 32, 0, st>>>(doms, dyn, rows, ctr, s);
  return cudaGetLastError();
}

// Every shape of a moving domain at the index after step s (block: one domain, thread:
// one shape), as each busy row of the move kernel placed it before: its FP64 position
// and the FP32 copies of the pre-test, computed once per step instead of once per row
// (that FP64 work ran on every busy row). Domains with coupled bodies are placed by
// fsi_kernel after their force reduction.
__global__ void __launch_bounds__(kMaxMovingShapes)
shape_table_kernel(const DomDev *doms, const DomDyn *dyn, const MoveRow *rows, const Counters *ctr, int s) {
  const MoveRow *movedoms = rows + ctr->nmove;
  const int ndom = ctr->nmovedom;
  for (int q = blockIdx.x; q < ndom; q += gridDim.x) {
    const int d = movedoms[q].dom;
    const DomDev &D = doms[d];
    if (D.fsi_on != 0) continue;
    const DomDyn dy = dyn[d];
    const long long n = dy.step0 + ctr->run_base + s;  // as in the move kernels
    if (n >= dy.step_end) continue;
    for (int k = threadIdx.x; k < D.nshapes; k += blockDim.x) {
      RowShape r;
      r.s = shape_at(D, D.shapes[k], n + 1, true);
      prep_row_shape(r);
      D.placed[k] = PlacedShape{r.s, r.fcx, r.fcy, r.fr2, r.fast};
    }
  }
}

cudaError_t launch_shape_table(int grid, cudaStream_t st, const DomDev *doms, const DomDyn *dyn,
                               const MoveRow *rows, const Counters *ctr, int s) {
  shape_table_kernel<<<grid, kMaxMovingShapes, 0, st>>>(doms, dyn, rows, ctr, s);
  return cudaGetLastError();
}

cudaError_t launch_move_cull(int grid, cudaStream_t st, const DomDev *doms, const DomDyn *dyn,
                             const MoveRow *rows, const Counters *ctr, BusyRow *busy, int s) {
  move_cull_kernel<<<grid, kCullThreads, 0, st>>>(doms, dyn, rows, ctr, busy, s);
  return cudaGetLastError();
}

cudaError_t launch_move_rows(int grid, cudaStream_t st, const DomDev *doms, const DomDyn *dyn,
                             const MoveRow *rows, const Counters *ctr, BusyRow *busy, int s, int storage) {
  if (storage == LBM_F64)
    move_rows_kernel<double><<<grid, kMoveWarps * 32, 0, st>>>(doms, dyn, rows, ctr, busy, s);
  else
    move_rows_kernel<float><<<grid, kMoveWarps * 32, 0, st>>>(doms, dyn, rows, ctr, busy, s);
  return cudaGetLastError();
}

// Mask and centres of one moving domain at index n (admission, step-index changes).
__global__ void __launch_bounds__(kMoveWarps * 32) place_kernel(const DomDev *dom, long long n) {
  __shared__ RowShape shapes[kMoveWarps][kMaxMovingShapes];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const DomDev &D = *dom;
  for (int j = blockIdx.x * kMoveWarps + warp; j < D.ny; j += gridDim.x * kMoveWarps) {
    place_row(D, j, n, lane, shapes[warp]);
    if (j == 0) place_centres(D, n, lane);
  }
}

cudaError_t launch_place(cudaStream_t st, const DomDev *dom_dev, int nx, int ny, int pitch, long long n) {
  (void)nx;
  (void)pitch;
  place_kernel<<<(ny + kMoveWarps - 1) / kMoveWarps, kMoveWarps * 32, 0, st>>>(dom_dev, n);
  return cudaGetLastError();
}

// ---- initial state: g = f^eq(rho0, u0) at every node, padding zero ----------------------

template <int S>
__global__ void init_kernel(typename Codec<S>::E *lat, int nx, int ny, int pitch, double rho0,
                            double ux, double uy) {
  using Cd = Codec<S>;
  using E = typename Cd::E;
  // 16-byte stores: rows start on 16-byte boundaries (the pitch is a multiple of 64
  // elements, the lattice starts on a 256-byte boundary)
  constexpr int kPer = 16 / static_cast<int>(sizeof(E));
  const int wd = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  const int a = blockIdx.z;
  if (wd >= pitch / kPer || j >= ny) return;
  const double w = a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  const double eu = ex_of(a) * ux + ey_of(a) * uy;
  const double usq = ux * ux + uy * uy;
  // Eq. (feq) with c_s^2 = 1/3; shifted storage keeps f^eq - w rho0 (times its scale)
  const double dev = rho0 * w * (3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
  const E val = Cd::enc(typename Cd::T(Cd::kStoreShifted ? dev * Cd::kScale : rho0 * w + dev));
  union {
    uint4 v;
    E e[kPer];
  } u;
#pragma unroll
  for (int q = 0; q < kPer; ++q) u.e[q] = wd * kPer + q < nx ? val : E(0);
  reinterpret_cast<uint4 *>(lat + (static_cast<size_t>(a) * ny + j) * pitch)[wd] = u.v;
}

cudaError_t launch_init(int storage, cudaStream_t st, void *lat, int nx, int ny, int pitch,
                        double rho0, double ux, double uy) {
  const int per = storage == LBM_F64 ? 2 : (storage == LBM_F32 ? 4 : 8);  // elements per 16 bytes
  dim3 grid((pitch / per + 127) / 128, ny, kQ);
  switch (storage) {
    case LBM_F64: init_kernel<LBM_F64><<<grid, 128, 0, st>>>(static_cast<double *>(lat), nx, ny, pitch, rho0, ux, uy); break;
    case LBM_F32: init_kernel<LBM_F32><<<grid, 128, 0, st>>>(static_cast<float *>(lat), nx, ny, pitch, rho0, ux, uy); break;
    case LBM_F16S: init_kernel<LBM_F16S><<<grid, 128, 0, st>>>(static_cast<uint16_t *>(lat), nx, ny, pitch, rho0, ux, uy); break;
    case LBM_BF16S: init_kernel<LBM_BF16S><<<grid, 128, 0, st>>>(static_cast<uint16_t *>(lat), nx, ny, pitch, rho0, ux, uy); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---- solid-node lists -----------------------------------------------------------------
// The force reducer sums F_VP over each body's nodes in one fixed order: body by body,
// row-major within a body. The list is built in two row-parallel passes: per-row counts
// of every body id, an exclusive scan on the host, then one block per (row, body)
// writing the row's nodes of that body at its offset in column order.

// counts[b * ny + j] = nodes of body id b in row j (b = 0 counts fluid); *bad_id > 0 if
// an id exceeds nbodies.
__global__ void row_counts_kernel(const uint8_t *mask, int nx, int ny, int pitch, int nbodies,
                                  int32_t *counts, int32_t *bad_id) {
  __shared__ int32_t hist[256];
  const int j = blockIdx.x;
  for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  const uint8_t *row = mask + static_cast<size_t>(j) * pitch;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) atomicAdd(&hist[row[i]], 1);
  __syncthreads();
  for (int b = threadIdx.x; b < 256; b += blockDim.x) {
    const int c = hist[b];
    if (b <= nbodies) counts[static_cast<size_t>(b) * ny + j] = c;
    else if (c > 0) atomicMax(bad_id, b);
  }
}

cudaError_t launch_row_counts(cudaStream_t st, const uint8_t *mask, int nx, int ny, int pitch,
                              int nbodies, int32_t *counts, int32_t *bad_id) {
  row_counts_kernel<<<ny, 256, 0, st>>>(mask, nx, ny, pitch, nbodies, counts, bad_id);
  return cudaGetLastError();
}

// Block (j, b-1): the nodes of body b in row j, in column order, at row_off[(b-1)*ny + j].
__global__ void row_scatter_kernel(const uint8_t *mask, int nx, int ny, int pitch,
                                   const int32_t *row_off, int32_t *solid) {
  const int j = blockIdx.x;
  const int body = blockIdx.y + 1;
  __shared__ int32_t warp_tot[32];
  __shared__ int32_t base;
  if (threadIdx.x == 0) base = row_off[static_cast<size_t>(body - 1) * ny + j];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint8_t *row = mask + static_cast<size_t>(j) * pitch;
  for (int i0 = 0; i0 < nx; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    const bool hit = i < nx && row[i] == body;
    const unsigned bal = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) before += warp_tot[w];
      total += warp_tot[w];
    }
    if (hit) solid[base + before + __popc(bal & ((1u << lane) - 1u))] = j * pitch + i;
    __syncthreads();
    if (threadIdx.x == 0) base += total;
    __syncthreads();
  }
}

cudaError_t launch_row_scatter(cudaStream_t st, const uint8_t *mask, int nx, int ny, int pitch,
                               int nbodies, const int32_t *row_off, int32_t *solid) {
  if (nbodies <= 0) return cudaSuccess;
  row_scatter_kernel<<<dim3(ny, nbodies), 256, 0, st>>>(mask, nx, ny, pitch, row_off, solid);
  return cudaGetLastError();
}

// ---- batched admission ------------------------------------------------------------------
// The same rasteriser, per-row counts, solid-node lists and initial state as above, for
// many domains in one launch each: block r of a launch takes row r of the flat row list
// of all admitted domains (domain d owns rows row0 .. row0 + ny - 1).

__device__ __forceinline__ int admit_domain_of(const AdmitDev *ad, int n, int r) {
  int lo = 0, hi = n - 1;  // the last domain with row0 <= r
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ad[mid].row0 <= r) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Mask row j (all pitch columns, padding zero) from the domain's shapes, then its per-row
// node counts of every body id. One warp per row of the flat list, eight rows per block.
// Only the columns within some shape's reach (shape_cols) take the FP64 predicate; the
// rest are fluid. A lane writes four columns with one 32-bit store (rows start on
// 64-byte boundaries: the pitch is a multiple of 64).
constexpr int kAdmitCull = 64;        // shapes per domain whose column intervals are culled
constexpr int kAdmitRowsPerBlock = 8;  // rows (warps) per block of the rasteriser

__global__ void __launch_bounds__(32 * kAdmitRowsPerBlock) admit_raster_count_kernel(AdmitDev *ad, int n, int rows) {
  __shared__ int32_t hist_s[kAdmitRowsPerBlock][256];
  __shared__ int lo_s[kAdmitRowsPerBlock][kAdmitCull], hi_s[kAdmitRowsPerBlock][kAdmitCull];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * kAdmitRowsPerBlock + warp;
  if (r >= rows) return;  // warp-uniform; the warps of a block do not synchronise
  int32_t *hist = hist_s[warp];
  int *lo = lo_s[warp], *hi = hi_s[warp];
  for (int b = lane; b < 256; b += 32) hist[b] = 0;
  AdmitDev &A = ad[admit_domain_of(ad, n, r)];
  const int j = r - A.row0;
  const bool cull = A.nshapes <= kAdmitCull;
  if (cull)
    for (int k = lane; k < A.nshapes; k += 32) shape_cols(A.shapes[k], A.nx, A.x0, j, lo[k], hi[k]);
  __syncwarp();
  uint8_t *row = A.mask + static_cast<size_t>(j) * A.pitch;
  int fluid = 0;
  for (int c0 = 4 * lane; c0 < A.pitch; c0 += 4 * 32) {
    uint32_t word = 0;
    for (int q = 0; q < 4; ++q) {
      const int i = c0 + q;
      if (i >= A.nx) break;
      uint32_t b = 0;
      for (int k = 0; k < A.nshapes; ++k) {
        if (cull && (i < lo[k] || i > hi[k])) continue;
        if (inside(A.shapes[k], double(i + A.x0), double(j))) b = static_cast<uint8_t>(A.shapes[k].body);
      }
      if (b == 0) ++fluid;
      else atomicAdd(&hist[b], 1);
      word |= b << (8 * q);
    }
    *reinterpret_cast<uint32_t *>(row + c0) = word;
  }
  for (int o = 16; o > 0; o >>= 1) fluid += __shfl_xor_sync(0xffffffffu, fluid, o);
  __syncwarp();
  if (lane == 0) hist[0] = fluid;
  __syncwarp();
  for (int b = lane; b < 256; b += 32) {
    const int cnt = hist[b];
    if (b <= A.nbodies) A.counts[static_cast<size_t>(b) * A.ny + j] = cnt;
    else if (cnt > 0) atomicMax(&A.bad, b);
  }
}

cudaError_t launch_admit_raster_count(cudaStream_t st, AdmitDev *ad, int n, int rows) {
  if (rows <= 0) return cudaSuccess;
  admit_raster_count_kernel<<<(rows + kAdmitRowsPerBlock - 1) / kAdmitRowsPerBlock, 32 * kAdmitRowsPerBlock, 0, st>>>(
      ad, n, rows);
  return cudaGetLastError();
}

// The nodes of each body in row r of the flat list, in column order, at the row's offset
// in the body's part of the solid list (as row_scatter_kernel). One warp per row, eight
// rows per block; a row without nodes of a body (its count) is not scanned for it.
__global__ void __launch_bounds__(32 * kAdmitRowsPerBlock) admit_scatter_kernel(const AdmitDev *ad, int n, int rows) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * kAdmitRowsPerBlock + warp;
  if (r >= rows) return;  // warp-uniform
  const AdmitDev &A = ad[admit_domain_of(ad, n, r)];
  const int j = r - A.row0;
  const uint8_t *row = A.mask + static_cast<size_t>(j) * A.pitch;
  for (int body = 1; body <= A.nbodies; ++body) {
    if (A.counts[static_cast<size_t>(body) * A.ny + j] == 0) continue;
    int base = A.row_off[static_cast<size_t>(body - 1) * A.ny + j];
    for (int i0 = 0; i0 < A.nx; i0 += 32) {
      const int i = i0 + lane;
      const bool hit = i < A.nx && row[i] == body;
      const unsigned bal = __ballot_sync(0xffffffffu, hit);
      if (hit) A.solid[base + __popc(bal & ((1u << lane) - 1u))] = j * A.pitch + i;
      base += __popc(bal);
    }
  }
}

cudaError_t launch_admit_scatter(cudaStream_t st, const AdmitDev *ad, int n, int rows, int max_bodies) {
  if (rows <= 0 || max_bodies <= 0) return cudaSuccess;
  admit_scatter_kernel<<<(rows + kAdmitRowsPerBlock - 1) / kAdmitRowsPerBlock, 32 * kAdmitRowsPerBlock, 0, st>>>(
      ad, n, rows);
  return cudaGetLastError();
}

static_assert(kPitchAlign % 16 == 0, "16-byte row stores need pitches of 16 elements");

// Block r: row r of every direction of lattice A set to f^eq(rho0, u0) as init_kernel
// does, with 16-byte stores (a row starts on a 16-byte boundary: lattices start on
// 256-byte boundaries and the pitch is a multiple of 64 elements). Of lattice B only the
// words holding padding columns (x >= nx) are zeroed: the first sweep writes every node
// of it before anything reads one, and the padding stays as every lattice keeps it.
template <int S>
__global__ void admit_init_kernel(const AdmitDev *ad, int n) {
  using Cd = Codec<S>;
  using E = typename Cd::E;
  constexpr int kPer = 16 / static_cast<int>(sizeof(E));
  __shared__ int dsh;
  __shared__ E val_s[kQ];
  if (threadIdx.x == 0) dsh = admit_domain_of(ad, n, blockIdx.x);
  __syncthreads();
  const AdmitDev &A = ad[dsh];
  const int j = blockIdx.x - A.row0;
  if (threadIdx.x < kQ) {
    const int a = threadIdx.x;
    const double w = a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    const double eu = ex_of(a) * A.u0x + ey_of(a) * A.u0y;
    const double usq = A.u0x * A.u0x + A.u0y * A.u0y;
    const double dev = A.rho0 * w * (3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
    val_s[a] = Cd::enc(typename Cd::T(Cd::kStoreShifted ? dev * Cd::kScale : A.rho0 * w + dev));
  }
  __syncthreads();
  const int words = A.pitch / kPer;
  for (int t = threadIdx.x; t < kQ * words; t += blockDim.x) {
    const int a = t / words, wd = t - a * words;
    const size_t off = (static_cast<size_t>(a) * A.ny + j) * A.pitch;
    const E val = val_s[a];
    union {
      uint4 v;
      E e[kPer];
    } u;
#pragma unroll
    for (int q = 0; q < kPer; ++q) u.e[q] = wd * kPer + q < A.nx ? val : E(0);
    reinterpret_cast<uint4 *>(static_cast<E *>(A.lat[0]) + off)[wd] = u.v;
    if ((wd + 1) * kPer > A.nx)
      reinterpret_cast<uint4 *>(static_cast<E *>(A.lat[1]) + off)[wd] = make_uint4(0u, 0u, 0u, 0u);
  }
}

cudaError_t launch_admit_init(int storage, cudaStream_t st, const AdmitDev *ad, int n, int rows) {
  if (rows <= 0) return cudaSuccess;
  const int grid = rows;
  switch (storage) {
    case LBM_F64: admit_init_kernel<LBM_F64><<<grid, 256, 0, st>>>(ad, n); break;
    case LBM_F32: admit_init_kernel<LBM_F32><<<grid, 256, 0, st>>>(ad, n); break;
    case LBM_F16S: admit_init_kernel<LBM_F16S><<<grid, 256, 0, st>>>(ad, n); break;
    case LBM_BF16S: admit_init_kernel<LBM_BF16S><<<grid, 256, 0, st>>>(ad, n); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Fill each span: a copy from its source, or zeros (16-byte words where both ends are
// aligned, bytes otherwise). Block (x, k) strides over span k.
__global__ void fill_kernel(const FillSeg *segs, int nseg) {
  for (int k = blockIdx.y; k < nseg; k += gridDim.y) {
    unsigned char *d = static_cast<unsigned char *>(segs[k].dst);
    const unsigned char *src = static_cast<const unsigned char *>(segs[k].src);
    const size_t bytes = segs[k].bytes;
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    const size_t t0 = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(d) | reinterpret_cast<uintptr_t>(src) | bytes) & 15) == 0;
    if (vec) {
      uint4 *dv = reinterpret_cast<uint4 *>(d);
      const uint4 *sv = reinterpret_cast<const uint4 *>(src);
      for (size_t i = t0; i < bytes / 16; i += stride) dv[i] = src ? sv[i] : make_uint4(0u, 0u, 0u, 0u);
    } else {
      for (size_t i = t0; i < bytes; i += stride) d[i] = src ? src[i] : 0;
    }
  }
}

cudaError_t launch_fill(cudaStream_t st, const FillSeg *segs, int nseg) {
  if (nseg <= 0) return cudaSuccess;
  fill_kernel<<<dim3(32, nseg < 65535 ? nseg : 65535), 256, 0, st>>>(segs, nseg);
  return cudaGetLastError();
}

// ---- halo edges (slab decomposition over devices) -------------------------------------
// Block (x, k) copies rows x*256 .. of halo item k: the three populations that leave the
// domain through that edge, from the edge column into the send buffer's planes.
template <typename E>
__global__ void halo_pack_kernel(const __grid_constant__ HaloPack pack) {
  const HaloItem &it = pack.item[blockIdx.y];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= it.ny) return;
  const E *lat = static_cast<const E *>(it.lat);
  E *send = static_cast<E *>(it.send);
  const size_t plane = static_cast<size_t>(it.ny) * it.pitch;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    // east edge: e_x = +1 (1, 5, 8); west edge: e_x = -1 (3, 6, 7)
    const int a = it.east ? (q == 0 ? 1 : (q == 1 ? 5 : 8)) : (q == 0 ? 3 : (q == 1 ? 6 : 7));
    send[static_cast<size_t>(a) * it.ny + j] = lat[a * plane + static_cast<size_t>(j) * it.pitch + it.col];
  }
}

cudaError_t launch_halo_pack(cudaStream_t st, const HaloPack &pack, int max_ny) {
  if (pack.n <= 0) return cudaSuccess;
  const dim3 grid((max_ny + 255) / 256, pack.n);
  switch (pack.elem) {
    case 2: halo_pack_kernel<uint16_t><<<grid, 256, 0, st>>>(pack); break;
    case 4: halo_pack_kernel<uint32_t><<<grid, 256, 0, st>>>(pack); break;
    case 8: halo_pack_kernel<unsigned long long><<<grid, 256, 0, st>>>(pack); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---- body forces -------------------------------------------------------------------------
// The sweep of step n+1 writes F_VP of every solid node (Eq. force-density) to the
// domain's F_VP field; this kernel, launched after it, sums -F_VP over each body's
// nodes (Sec. 3, drag and lift sums, read as the force on the body) into the force
// ring. One block per (slot, body) item: each thread accumulates a strided subset of
// the body's row-major node list in FP64, then a fixed shuffle + shared-memory tree,
// so the sum order depends only on the node list, not on the tiling or the batch.

// Small blocks at no more than 32 registers: one fits on an SM beside the direct sweep's
// two 384-thread blocks at 80 registers (61,440 of 65,536), so the reduction of step n
// runs while the sweep of step n + 1 does.
constexpr int kForceThreads = 128;

template <int S>
__global__ void __launch_bounds__(kForceThreads, 16)
forces_kernel(const DomDev *doms, const DomDyn *dyn, const ForceItem *items, const Counters *ctr,
              int s) {
  using T = typename Codec<S>::T;
  const int nitems = ctr->nforce;
  const long long run_base = ctr->run_base;
  __shared__ double red[2][kForceThreads / 32];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const ForceItem item = items[it];
    const DomDev &D = doms[item.dom];
    const DomDyn dy = dyn[item.dom];
    // the F_VP field the sweep of this step wrote (the parity of the lattice it read)
    const int par = (dy.parity + static_cast<int>((run_base + s) & 1)) & 1;
    const T *fv = static_cast<const T *>(D.fvp[par]);
    const int32_t *solid = D.solid;
    const int force_every = D.force_every;
    // the node indices do not depend on the step: their loads overlap the checks below
    const int q0 = item.beg + threadIdx.x;
    const int32_t lin0 = (!item.rows && q0 < item.end) ? __ldg(solid + q0) : 0;
    const long long n = dy.step0 + run_base + s;  // the sweep just computed step n + 1
    if (n >= dy.step_end || force_every <= 0) continue;
    if ((n + 1) % force_every != 0) continue;
    double fx = 0.0, fy = 0.0;
    if (item.rows) {
      // moving domain: the per-row sums of -F_VP, rows in order per thread
      for (int q = q0; q < item.end; q += blockDim.x) {
        const double *r = D.rowsum[par] + (static_cast<size_t>(q) * D.nbodies + (item.body - 1)) * 3;
        if (r[2] == static_cast<double>(n)) {  // written for this step
          fx += r[0];
          fy += r[1];
        }
      }
    } else {
      for (int q = q0; q < item.end; q += blockDim.x) {
        const size_t lin = static_cast<size_t>(q == q0 ? lin0 : __ldg(solid + q));
        fx -= double(fv[2 * lin]);
        fy -= double(fv[2 * lin + 1]);
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      fx += __shfl_down_sync(0xffffffffu, fx, off);
      fy += __shfl_down_sync(0xffffffffu, fy, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
      red[0][warp] = fx;
      red[1][warp] = fy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sx = 0.0, sy = 0.0;
      for (int w = 0; w < kForceThreads / 32; ++w) {
        sx += red[0][w];
        sy += red[1][w];
      }
      const long long e = (n + 1) / D.force_every - 1;  // entry index of step n + 1
      double *slot = D.ring + (static_cast<size_t>(e % D.force_cap) * D.nbodies + (item.body - 1)) * 2;
      slot[0] = sx;
      slot[1] = sy;
    }
    __syncthreads();
  }
}

cudaError_t launch_forces(int storage, int grid, cudaStream_t st, const DomDev *doms,
                          const DomDyn *dyn, const ForceItem *items, const Counters *ctr, int s) {
  switch (storage) {
    case LBM_F64: forces_kernel<LBM_F64><<<grid, kForceThreads, 0, st>>>(doms, dyn, items, ctr, s); break;
    case LBM_F32: forces_kernel<LBM_F32><<<grid, kForceThreads, 0, st>>>(doms, dyn, items, ctr, s); break;
    case LBM_F16S: forces_kernel<LBM_F16S><<<grid, kForceThreads, 0, st>>>(doms, dyn, items, ctr, s); break;
    case LBM_BF16S: forces_kernel<LBM_BF16S><<<grid, kForceThreads, 0, st>>>(doms, dyn, items, ctr, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Advance the device step counter of a run by k steps (last node of a captured graph).
__global__ void advance_kernel(Counters *ctr, int k) { ctr->run_base += k; }

cudaError_t launch_advance(cudaStream_t st, Counters *ctr, int k) {
  advance_kernel<<<1, 1, 0, st>>>(ctr, k);
  return cudaGetLastError();
}

// ---- moments export ------------------------------------------------------------------------

template <int S>
__global__ void moments_kernel(const DomDev *dom, int parity, double *rho, double *ux, double *uy) {
  using Cd = Codec<S>;
  using T = typename Cd::T;
  const DomDev &D = *dom;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= D.nx || j >= D.ny) return;
  const void *src = D.lat[parity];
  const CellConst<T> &C = cell_const<T>(D);
  T x[kQ];
#pragma unroll
  for (int a = 0; a < kQ; ++a) x[a] = pull_scalar<S>(D, src, a, i, j);
  const int b = D.mask[static_cast<size_t>(j) * D.pitch + i];
  T uox = T(0), uoy = T(0);
  if (b) body_velocity<true>(D, b, i, j, uox, uoy);
  const NodeMacro<T> m = node_macro<T, Cd::kShiftCompute, true>(x, C, b != 0, uox, uoy);
  const size_t c = static_cast<size_t>(j) * D.nx + i;
  if (rho) rho[c] = double(m.rho * (T(1) / T(Cd::kScale)));  // unscaled (power of two: exact)
  if (ux) ux[c] = double(m.ux);
  if (uy) uy[c] = double(m.uy);
}

template <int S>
cudaError_t launch_moments_t(cudaStream_t st, const DomDev *dom, int nx, int ny, int parity,
                             double *rho, double *ux, double *uy) {
  dim3 grid((nx + 127) / 128, ny);
  moments_kernel<S><<<grid, 128, 0, st>>>(dom, parity, rho, ux, uy);
  return cudaGetLastError();
}

cudaError_t launch_moments_sized(int storage, cudaStream_t st, const DomDev *dom, int nx, int ny,
                                 int parity, double *rho, double *ux, double *uy) {
  switch (storage) {
    case LBM_F64: return launch_moments_t<LBM_F64>(st, dom, nx, ny, parity, rho, ux, uy);
    case LBM_F32: return launch_moments_t<LBM_F32>(st, dom, nx, ny, parity, rho, ux, uy);
    case LBM_F16S: return launch_moments_t<LBM_F16S>(st, dom, nx, ny, parity, rho, ux, uy);
    case LBM_BF16S: return launch_moments_t<LBM_BF16S>(st, dom, nx, ny, parity, rho, ux, uy);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lbm
