// 3D TRT-LBM-VP (D3Q19 / D3Q15): moments, initial state, rasteriser, moving, coupled and
// pulsating bodies, force reductions and the single-domain runtime (the C ABI lbm3_* of
// include/lbm.h). The sweep kernel and the node update are in lbm3d.cuh; the sweep is
// instantiated per storage by lbm3d_sweep_<storage>.cu.
#include "lbm3d.cuh"

namespace lbm {
namespace d3 {

// Scalar pull with the edge rules (moments export).
template <int Q, int S>
__device__ __forceinline__ typename Codec<S>::T pull3(const Dom3 &D, const void *lat, int a, int i, int j, int k) {
  using Cd = Codec<S>;
  using E = typename Cd::E;
  int sx = i - ex3<Q>(a);
  if (sx < 0) {
    if (D.west == LBM_INLET_EQ) return const3<typename Cd::T>(D).ghost[a];
    sx += D.nx;
  } else if (sx > D.nx - 1) {
    sx = D.east == LBM_OUTFLOW_ZG ? D.nx - 1 : sx - D.nx;
  }
  int sa, sy, sz;
  src_row3<Q>(D, a, j, k, sa, sy, sz);
  const E *p = static_cast<const E *>(lat);
  typename Cd::T x = Cd::dec(p[((static_cast<size_t>(sa) * D.nz + sz) * D.ny + sy) * D.pitch + sx]);
  if (Cd::kShiftCompute && !Cd::kStoreShifted) x -= shift3(const3<typename Cd::T>(D), a);
  return x;
}

template <int Q, int S>
__global__ void moments3_kernel(const Dom3 *dom, int par, double *rho, double *ux, double *uy, double *uz) {
  using Cd = Codec<S>;
  using T = typename Cd::T;
  const Dom3 &D = *dom;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  if (i >= D.nx) return;
  T x[Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) x[a] = pull3<Q, S>(D, D.lat[par], a, i, j, k);
  const int b = D.mask[(static_cast<size_t>(k) * D.ny + j) * D.pitch + i];
  T uo[3] = {T(0), T(0), T(0)};
  // kappa exists only in moving domains: the dilation term only where a body pulsates
  if (b) {
    if (D.deform) body_velocity3<true>(D, b, i, j, k, uo);
    else body_velocity3<false>(D, b, i, j, k, uo);
  }
  const Macro3<T> m = macro3<Q, T, Cd::kShiftCompute, true>(x, const3<T>(D), b != 0, uo);
  const size_t c = (static_cast<size_t>(k) * D.ny + j) * D.nx + i;
  if (rho) rho[c] = double(m.rho * (T(1) / T(Cd::kScale)));
  if (ux) ux[c] = double(m.u[0]);
  if (uy) uy[c] = double(m.u[1]);
  if (uz) uz[c] = double(m.u[2]);
}

template <int Q, int S>
__global__ void init3_kernel(typename Codec<S>::E *lat, int nx, int nrows, int pitch, double rho0,
                             double u0x, double u0y, double u0z) {
  using Cd = Codec<S>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  if (i >= pitch) return;
  const double w = w3<Q>(a == 0 ? 0 : (a < 7 ? 1 : 2));
  const double eu = ex3<Q>(a) * u0x + ey3<Q>(a) * u0y + ez3<Q>(a) * u0z;
  const double usq = u0x * u0x + u0y * u0y + u0z * u0z;
  const double dev = rho0 * w * (3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
  double val = Cd::kStoreShifted ? dev * Cd::kScale : rho0 * w + dev;
  if (i >= nx) val = 0.0;
  const typename Cd::E e = Cd::enc(typename Cd::T(val));
  for (int row = blockIdx.z; row < nrows; row += gridDim.z)  // row = k * ny + j
    lat[(static_cast<size_t>(a) * nrows + row) * pitch + i] = e;
}

// sphere / z-cylinder predicates in FP64 with explicit roundings (the plain IEEE order)
struct Shape3Dev {
  int32_t kind, body;
  double c[3], radius;
};

__device__ __forceinline__ bool inside3(const Shape3Dev &s, int i, int j, int k) {
  const double dx = __dsub_rn(double(i), s.c[0]), dy = __dsub_rn(double(j), s.c[1]);
  double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  if (s.kind == LBM3_SHAPE_SPHERE) {
    const double dz = __dsub_rn(double(k), s.c[2]);
    d2 = __dadd_rn(d2, __dmul_rn(dz, dz));
  }
  return d2 < __dmul_rn(s.radius, s.radius);
}

// Where the shapes of a moving domain are at a step index: bodies9 [nb][9] (velocity at
// 3..5); for coupled bodies (bit body - 1 of `coupled`) the state rows of that index, xs
// [8][9] (centre at 0..2), and the reference centres c0 [8][3].
struct Place3 {
  const double *bodies9;
  int nb;
  uint32_t coupled;
  const double *xs, *c0;
  uint32_t deform;     // bit b: body b + 1 pulsates ([8][2] amplitude and rate in dpar)
  const double *dpar;
};

// scale s(n) = 1 + a sin(nu n) of a pulsating body (a, nu at p[0], p[1]); kappa = s'/s
__device__ __forceinline__ double pulse3(const double *p, long long n, double *kappa) {
  double sn, cs;
  turn_sincos(__dmul_rn(p[1], static_cast<double>(n)), sn, cs);
  const double sc = __dadd_rn(1.0, __dmul_rn(p[0], sn));
  if (kappa) *kappa = __ddiv_rn(__dmul_rn(__dmul_rn(p[0], p[1]), cs), sc);
  return sc;
}

// shape s0 at step index n: translated with its body's velocity by V n, or, for a coupled
// body, by its integrated centre minus its reference centre, x - x0 (explicit roundings);
// n = 0 and the initial state give the reference shape exactly
__device__ __forceinline__ Shape3Dev shape3_at(const Shape3Dev &s0, const Place3 &pl, long long n) {
  Shape3Dev s = s0;
  if (s0.body < 1 || s0.body > pl.nb) return s;
  const int b = s0.body - 1;
  if (pl.coupled >> b & 1u) {
    for (int d = 0; d < 3; ++d) s.c[d] = __dadd_rn(s0.c[d], __dsub_rn(pl.xs[9 * b + d], pl.c0[3 * b + d]));
  } else if (pl.deform >> b & 1u) {
    // a pulsating body: the offset from its reference centre and the radius scaled by s(n)
    const double sc = pulse3(pl.dpar + 2 * b, n, nullptr);
    const double *v = pl.bodies9 + 9 * b + 3;
    for (int d = 0; d < 3; ++d)
      s.c[d] = __dadd_rn(__dadd_rn(pl.c0[3 * b + d], __dmul_rn(v[d], double(n))),
                         __dmul_rn(sc, __dsub_rn(s0.c[d], pl.c0[3 * b + d])));
    s.radius = __dmul_rn(sc, s0.radius);
  } else if (n != 0) {
    const double *v = pl.bodies9 + 9 * b + 3;
    for (int d = 0; d < 3; ++d) s.c[d] = __dadd_rn(s0.c[d], __dmul_rn(v[d], double(n)));
  }
  return s;
}

__global__ void rasterize3_kernel(uint8_t *mask, int nx, int ny, int nz, int pitch, const Shape3Dev *shapes,
                                  int nshapes, Place3 pl, long long n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  if (i >= pitch) return;
  uint8_t id = 0;
  if (i < nx)
    for (int q = 0; q < nshapes; ++q) {
      const Shape3Dev s = shape3_at(shapes[q], pl, n);
      if (inside3(s, i, j, k)) id = static_cast<uint8_t>(s.body);
    }
  mask[(static_cast<size_t>(k) * ny + j) * pitch + i] = id;
}

// the state row of coupled body b at step index n (x at 0..2, v at 3..5, F_{n-1} at 6..8)
__device__ __forceinline__ double *fsi_row3(const Dom3 &D, int b, long long n) {
  return D.fsi + (static_cast<size_t>(n & 1) * kMaxMoving3 + b) * 9;
}

// centre of body b along axis d at step index n: a coupled body's integrated state, else
// c0 + V n (explicit roundings, as the oracle's plain evaluation)
__device__ __forceinline__ double centre3(const Dom3 &D, int b, int d, long long n) {
  if (D.coupled >> b & 1u) return fsi_row3(D, b, n)[d];
  return __dadd_rn(D.centre0[3 * b + d], __dmul_rn(D.bodies[9 * b + 3 + d], double(n)));
}

// body table at step index n (centres; coupled bodies also their velocities), FP64 and
// FP32, for bodies b = b0, b0 + stride, ...
__device__ __forceinline__ void place_bodies3(const Dom3 &D, long long n, int b0, int stride) {
  for (int b = b0; b < D.nbodies; b += stride) {
    if (D.deform >> b & 1u) {  // the dilation rate of step n
      double kp;
      pulse3(D.dpar + 2 * b, n, &kp);
      D.kappa[b] = kp;
      D.kappa_f[b] = float(kp);
    }
    const bool cpl = D.coupled >> b & 1u;
    const double *st = cpl ? fsi_row3(D, b, n) : nullptr;
    for (int d = 0; d < 3; ++d) {
      const double c = centre3(D, b, d, n);
      D.bodies[9 * b + d] = c;
      D.bodies_f[9 * b + d] = float(c);
      if (cpl) {
        D.bodies[9 * b + 3 + d] = st[3 + d];
        D.bodies_f[9 * b + 3 + d] = float(st[3 + d]);
      }
    }
  }
}

__global__ void centres3_kernel(const Dom3 *dom, long long n) { place_bodies3(*dom, n, threadIdx.x, blockDim.x); }

// Node ranges of body b's box at step index n, grown by `grow` nodes (inclusive; empty if
// some hi < lo): the box its shapes reach about its centre c0 + V n.
struct Box3 {
  int lo[3], hi[3];
};

__device__ __forceinline__ Box3 body_box3(const Dom3 &D, int b, long long n, int grow) {
  Box3 B;
  const int N[3] = {D.nx, D.ny, D.nz};
  for (int d = 0; d < 3; ++d) {
    const float h = D.mbox[b][d];
    if (h < 0.f) {
      B.lo[d] = 0;
      B.hi[d] = N[d] - 1;
      continue;
    }
    const double c = centre3(D, b, d, n);
    // clamped to [-1, N] in FP64 first, so that a body far outside converts safely
    const double lo = fmin(fmax(floor(c - double(h)) - grow, -1.0), double(N[d]));
    const double hi = fmax(fmin(ceil(c + double(h)) + grow, double(N[d])), -1.0);
    B.lo[d] = max(0, static_cast<int>(lo));
    B.hi[d] = min(N[d] - 1, static_cast<int>(hi));
  }
  return B;
}

__device__ __forceinline__ bool box_empty(const Box3 &B) {
  return B.hi[0] < B.lo[0] || B.hi[1] < B.lo[1] || B.hi[2] < B.lo[2];
}

// One axis of a coupled body after step n, driven by the mean of the forces of steps n
// and n - 1, (F + Fp) / 2 (it cancels the force component that alternates every step):
// v <- v + (Fm - k (x - x0) - c v) / M, then x <- x + v (semi-implicit Euler, dt = 1),
// each operation rounded as written; an axis that is not free keeps its velocity.
__device__ __forceinline__ void fsi3_axis(double F, double Fp, double k, double c, double M, bool free_axis,
                                          double x0, double &x, double &v) {
  if (free_axis) {
    const double Fm = __dmul_rn(__dadd_rn(F, Fp), 0.5);
    double t = __dsub_rn(Fm, __dmul_rn(k, __dsub_rn(x, x0)));
    t = __dsub_rn(t, __dmul_rn(c, v));
    v = __dadd_rn(v, __ddiv_rn(t, M));
  }
  x = __dadd_rn(x, v);
}

constexpr int kMaxMoveBlocks3 = 256;  // blocks per body of the moving-domain kernels, at most
constexpr int kMaxShapes3 = 64;    // shapes of a moving 3D domain
constexpr int kMoveThreads3 = 256;

// Forces of a moving domain at step index n (the sweep just computed step n + 1): per
// body, the rows of its box at n (where all its nodes of step n lie) split over
// the launch's blocks (at most kMaxMoveBlocks3, sized to the box), one warp per row, -F_VP of the nodes with its id; each block's sum
// (fixed tree) goes to a partial slot, and the last block of the body adds the partials
// in block order into the ring entry and, for a coupled body, advances its state to n + 1
// from that force. Deterministic: the box depends on the state of index n only.
template <typename T>
__global__ void __launch_bounds__(kMoveThreads3)
mforce3_kernel(const __grid_constant__ Dom3 dom, long long n, long long entry) {
  const Dom3 &D = dom;  // kernel parameter: no dependent loads of the domain's fields
  const int b = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const Box3 B = body_box3(D, b, n, 0);
  const int ny_b = B.hi[1] - B.lo[1] + 1, nz_b = B.hi[2] - B.lo[2] + 1;
  const int nrows = (ny_b > 0 && nz_b > 0 && B.hi[0] >= B.lo[0]) ? ny_b * nz_b : 0;
  double f[3] = {0.0, 0.0, 0.0};
  for (int r = blockIdx.x * (kMoveThreads3 / 32) + warp; r < nrows; r += gridDim.x * (kMoveThreads3 / 32)) {
    const int j = B.lo[1] + r % ny_b, k = B.lo[2] + r / ny_b;
    const size_t row = static_cast<size_t>(k) * D.ny + j;
    const uint8_t *m = D.mask + row * D.pitch;
    const T *fv = static_cast<const T *>(D.fvp) + 3 * row * D.pitch;
    for (int i = B.lo[0] + lane; i <= B.hi[0]; i += 32) {
      // mask byte and F_VP loaded together (in bounds for every node of the box)
      const uint8_t id = m[i];
      const T v0 = fv[3 * i], v1 = fv[3 * i + 1], v2 = fv[3 * i + 2];
      if (id == b + 1) {
        f[0] -= double(v0);
        f[1] -= double(v1);
        f[2] -= double(v2);
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
    for (int e = 0; e < 3; ++e) f[e] += __shfl_down_sync(0xffffffffu, f[e], off);
  __shared__ double red[3][kMoveThreads3 / 32];
  __shared__ bool last;
  if (lane == 0)
    for (int e = 0; e < 3; ++e) red[e][warp] = f[e];
  __syncthreads();
  if (threadIdx.x == 0) {
    double *part = D.mpart + (static_cast<size_t>(b) * kMaxMoveBlocks3 + blockIdx.x) * 3;
    for (int e = 0; e < 3; ++e) {
      double t = 0.0;
      for (int w = 0; w < kMoveThreads3 / 32; ++w) t += red[e][w];
      part[e] = t;
    }
    __threadfence();
    last = atomicAdd(D.mcount + b, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last block: thread q loads partial q (all at once), then a fixed tree over q
  double t[3] = {0.0, 0.0, 0.0};
  if (threadIdx.x < gridDim.x)
    for (int e = 0; e < 3; ++e) t[e] = __ldcg(D.mpart + (static_cast<size_t>(b) * kMaxMoveBlocks3 + threadIdx.x) * 3 + e);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
    for (int e = 0; e < 3; ++e) t[e] += __shfl_down_sync(0xffffffffu, t[e], off);
  __syncthreads();
  if (lane == 0)
    for (int e = 0; e < 3; ++e) red[e][warp] = t[e];
  __syncthreads();
  if (threadIdx.x != 0) return;
  double *slot = D.ring + (static_cast<size_t>(entry % D.force_cap) * D.nbodies + b) * 3;
  double F[3];
  for (int e = 0; e < 3; ++e) {
    double x = 0.0;
    for (int w = 0; w < kMoveThreads3 / 32; ++w) x += red[e][w];
    slot[e] = x;
    F[e] = x;
  }
  D.mcount[b] = 0u;
  if (D.coupled >> b & 1u) {
    const double *par = D.fsi_par + 12 * b;  // M, k[3], c[3], free[3]
    const double *st = fsi_row3(D, b, n);
    double *nst = fsi_row3(D, b, n + 1);
    for (int e = 0; e < 3; ++e) {
      double x = st[e], v = st[3 + e];
      fsi3_axis(F[e], st[6 + e], par[1 + e], par[4 + e], par[0], par[7 + e] != 0.0, D.centre0[3 * b + e], x, v);
      nst[e] = x;
      nst[3 + e] = v;
      nst[6 + e] = F[e];
    }
  }
}

// The mask of a moving domain at step index n + 1, after the forces of step n: per body,
// the nodes of its box at n grown by one node (|V| <= 1 per axis, so the box at n + 1 lies
// inside; a coupled body: the union of its boxes at n and n + 1), ids from every shape at
// n + 1 (later shapes overwrite earlier ones), one warp per row. Boxes of different bodies
// may overlap: they write the same ids there. Block (0, 0) then moves the body table to
// n + 1 (no other block reads it).
// inside3 with an FP32 pre-test: a node whose FP32 squared distance is farther than 0.5
// from r^2 is decided there, the others take the exact FP64 predicate. With centres below
// 4096 in magnitude (FP32 position error <= 2.5e-4) and radii below 100 (|dx|, |dy|, |dz|
// <= r + 3 for nodes near the sphere or cylinder), the FP32 error of d^2 is below
// 2 (|dx| + |dy| + |dz|) 2.5e-4 + 4 d^2 2^-24 < 0.2, so the FP32 decision is the exact one.
__device__ __forceinline__ bool inside3_fast(const Shape3Dev &s, const float (&cf)[3], int i, int j, int k) {
  if (fabs(s.c[0]) < 4096.0 && fabs(s.c[1]) < 4096.0 && fabs(s.c[2]) < 4096.0 && s.radius < 100.0) {
    const float dx = float(i) - cf[0], dy = float(j) - cf[1];
    float d2 = dx * dx + dy * dy;
    if (s.kind == LBM3_SHAPE_SPHERE) {
      const float dz = float(k) - cf[2];
      d2 += dz * dz;
    }
    const float r2 = float(s.radius) * float(s.radius);
    if (d2 < r2 - 0.5f) return true;
    if (d2 > r2 + 0.5f) return false;
  }
  return inside3(s, i, j, k);
}

__global__ void __launch_bounds__(kMoveThreads3) mmove3_kernel(const __grid_constant__ Dom3 dom, long long n) {
  const Dom3 &D = dom;
  const int b = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // every shape at n + 1, translated once per block (FP64, explicit roundings)
  __shared__ Shape3Dev sh[kMaxShapes3];
  __shared__ float shc[kMaxShapes3][3];
  const Place3 pl{D.bodies, D.nbodies, D.coupled, D.fsi ? fsi_row3(D, 0, n + 1) : nullptr, D.centre0, D.deform,
                  D.dpar};
  for (int q = threadIdx.x; q < D.nshapes; q += blockDim.x) {
    sh[q] = shape3_at(D.shapes[q], pl, n + 1);
    for (int d = 0; d < 3; ++d) shc[q][d] = float(sh[q].c[d]);
  }
  __syncthreads();
  Box3 B;
  if (D.coupled >> b & 1u) {
    B = body_box3(D, b, n, 0);
    const Box3 B1 = body_box3(D, b, n + 1, 0);
    if (box_empty(B)) B = B1;
    else if (!box_empty(B1))
      for (int d = 0; d < 3; ++d) {
        B.lo[d] = min(B.lo[d], B1.lo[d]);
        B.hi[d] = max(B.hi[d], B1.hi[d]);
      }
  } else {
    B = body_box3(D, b, n, 1);
  }
  const int ny_b = B.hi[1] - B.lo[1] + 1, nz_b = B.hi[2] - B.lo[2] + 1;
  const int nrows = (ny_b > 0 && nz_b > 0 && B.hi[0] >= B.lo[0]) ? ny_b * nz_b : 0;
  for (int r = blockIdx.x * (kMoveThreads3 / 32) + warp; r < nrows; r += gridDim.x * (kMoveThreads3 / 32)) {
    const int j = B.lo[1] + r % ny_b, k = B.lo[2] + r / ny_b;
    uint8_t *m = D.mask + (static_cast<size_t>(k) * D.ny + j) * D.pitch;
    for (int i = B.lo[0] + lane; i <= B.hi[0]; i += 32) {
      uint8_t id = 0;
      for (int q = 0; q < D.nshapes; ++q)
        if (inside3_fast(sh[q], shc[q], i, j, k)) id = static_cast<uint8_t>(sh[q].body);
      m[i] = id;
    }
  }
  if (blockIdx.x == 0 && blockIdx.y == 0) place_bodies3(D, n + 1, threadIdx.x, blockDim.x);
}

// Body forces of step index n (the sweep just computed step n + 1): one warp per listed
// row sums -F_VP per body over the row's solid column range (lane-strided, fixed shuffle
// tree); the last block to finish then adds the rows in list order (thread-strided, fixed
// tree) into the ring entry. The result does not depend on which block finishes last.
constexpr int kRowsThreads = 256;

// The force entry `entry` of a domain D (Dom3, or Rows3Dom in a batch): block bx of gx
// sums -F_VP per body over every gx-th group of its rows (one warp per row), the last
// block to finish adds the row sums in row order into the ring.
template <typename T, typename DomT>
__device__ __forceinline__ void rows3_run(const DomT &D, long long entry, int bx, int gx) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wg = (bx * static_cast<int>(blockDim.x) + static_cast<int>(threadIdx.x)) >> 5;
  const int nw = (gx * static_cast<int>(blockDim.x)) >> 5;
  for (int q = wg; q < D.nfrows; q += nw) {
    const int4 it = D.frows[q];
    const size_t row = static_cast<size_t>(it.x);
    const uint8_t *m = D.mask + row * D.pitch;
    const T *fv = static_cast<const T *>(D.fvp) + 3 * row * D.pitch;
    for (int body = 1; body <= D.nbodies; ++body) {
      double f[3] = {0.0, 0.0, 0.0};
      for (int i = it.y + lane; i < it.z; i += 32) {
        const uint8_t id = m[i];  // mask byte and F_VP loaded together
        const T v0 = fv[3 * i], v1 = fv[3 * i + 1], v2 = fv[3 * i + 2];
        if (id == body) {
          f[0] -= double(v0);
          f[1] -= double(v1);
          f[2] -= double(v2);
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1)
        for (int e = 0; e < 3; ++e) f[e] += __shfl_down_sync(0xffffffffu, f[e], off);
      if (lane == 0)
        for (int e = 0; e < 3; ++e) D.rowsum[(static_cast<size_t>(q) * D.nbodies + body - 1) * 3 + e] = f[e];
    }
  }
  __shared__ bool last;
  __shared__ double red[3][kRowsThreads / 32];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(D.rows_done, 1u) == static_cast<unsigned>(gx) - 1u;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int body = 1; body <= D.nbodies; ++body) {
    double f[3] = {0.0, 0.0, 0.0};
    int q = threadIdx.x;
    // four rows' sums loaded at once, added in row order (the order of the plain loop)
    for (; q + 3 * static_cast<int>(blockDim.x) < D.nfrows; q += 4 * blockDim.x) {
      double v[4][3];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        for (int e = 0; e < 3; ++e)
          v[u][e] = __ldcg(D.rowsum + (static_cast<size_t>(q + u * blockDim.x) * D.nbodies + body - 1) * 3 + e);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        for (int e = 0; e < 3; ++e) f[e] += v[u][e];
    }
    for (; q < D.nfrows; q += blockDim.x)
      for (int e = 0; e < 3; ++e) f[e] += __ldcg(D.rowsum + (static_cast<size_t>(q) * D.nbodies + body - 1) * 3 + e);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
      for (int e = 0; e < 3; ++e) f[e] += __shfl_down_sync(0xffffffffu, f[e], off);
    if (lane == 0)
      for (int e = 0; e < 3; ++e) red[e][warp] = f[e];
    __syncthreads();
    if (threadIdx.x == 0) {
      double *slot = D.ring + (static_cast<size_t>(entry % D.force_cap) * D.nbodies + body - 1) * 3;
      for (int e = 0; e < 3; ++e) {
        double t = 0.0;
        for (int w = 0; w < kRowsThreads / 32; ++w) t += red[e][w];
        slot[e] = t;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *D.rows_done = 0u;
}

template <typename T>
__global__ void __launch_bounds__(kRowsThreads) rows3_kernel(const __grid_constant__ Dom3 dom, long long entry) {
  rows3_run<T>(dom, entry, blockIdx.x, gridDim.x);
}

// What the force reduction of a batch reads of one domain.
struct Rows3Dom {
  const int4 *frows;
  const uint8_t *mask;
  const void *fvp;
  double *rowsum, *ring;
  uint32_t *rows_done;
  long long entry;  // the ring entry this launch writes
  int32_t pitch, nfrows, nbodies, force_cap;
};

struct Rows3Args {
  Rows3Dom dom[kGroup3];
  int32_t ndom;
};

// The force entries of up to kGroup3 domains of a batch: blocks (bx, d) reduce domain d
// as rows3_kernel's gridDim.x blocks would; a domain without solid rows gets a zero entry.
template <typename T>
__global__ void __launch_bounds__(kRowsThreads) rows3_batch_kernel(const __grid_constant__ Rows3Args args) {
  const Rows3Dom &D = args.dom[blockIdx.y];
  if (D.nfrows == 0) {
    if (blockIdx.x == 0 && threadIdx.x < 3 * D.nbodies)
      D.ring[static_cast<size_t>(D.entry % D.force_cap) * D.nbodies * 3 + threadIdx.x] = 0.0;
    return;
  }
  rows3_run<T>(D, D.entry, blockIdx.x, gridDim.x);
}

}  // namespace d3
}  // namespace lbm

// ======================================================================================
// Runtime and C ABI

using namespace lbm;
using namespace lbm::d3;

namespace {

lbm_status fail3(lbm_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return s;
}

#define LBM3_CUDA(call)                                                               \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail3(LBM_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),  \
                   __FILE__, __LINE__);                                               \
  } while (0)

size_t esize(int storage) {
  return storage == LBM_F64 ? 8 : storage == LBM_F32 ? 4 : (storage == LBM_F16S || storage == LBM_BF16S) ? 2 : 0;
}
size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }
// directions of the lattice a parameter set selects (0 or 19: D3Q19, 15: D3Q15)
int nq_of(const lbm3_params &p) { return p.lattice == 15 ? 15 : 19; }
int e_of(int q, int a, int axis) {
  if (q == 15) return axis == 0 ? ex3<15>(a) : axis == 1 ? ey3<15>(a) : ez3<15>(a);
  return axis == 0 ? ex3<19>(a) : axis == 1 ? ey3<19>(a) : ez3<19>(a);
}
double w_of(int q, int a) {
  const int cls = a == 0 ? 0 : (a < 7 ? 1 : 2);
  return q == 15 ? w3<15>(cls) : w3<19>(cls);
}

struct Layout3 {
  size_t lat, mask_off, fvp_off, bodies_off, bodiesf_off, ring_off, status_off, moving_off, total;
};

// moving domains: shape table, reference centres, partial force sums, block counters,
// coupled-body state by parity and parameters
size_t moving_bytes3() {
  return up(sizeof(Shape3Dev) * kMaxShapes3, 256) + up(sizeof(double) * 3 * kMaxMoving3, 256) +
         up(sizeof(double) * 3 * kMaxMoving3 * kMaxMoveBlocks3, 256) + up(sizeof(uint32_t) * kMaxMoving3, 256) +
         up(sizeof(double) * 9 * 2 * kMaxMoving3, 256) + up(sizeof(double) * 12 * kMaxMoving3, 256) +
         up(sizeof(double) * 3 * kMaxMoving3 + sizeof(float) * kMaxMoving3, 256);
}

// Half extents of the box body b's shapes reach about its centre c (null: no body), two
// nodes wide beyond the shapes, the offsets and radii grown by `grow` (1 + |a| for a
// pulsating body); a z-cylinder spans the whole z axis (< 0)
void set_mbox3(Dom3 &D, const std::vector<Shape3Dev> &shapes, int b, const double *c, double grow) {
  for (int e = 0; e < 3; ++e) D.mbox[b][e] = 0.f;
  if (!c) return;
  for (const Shape3Dev &s : shapes) {
    if (s.body - 1 != b) continue;
    for (int e = 0; e < 3; ++e) {
      if (e == 2 && s.kind == LBM3_SHAPE_CYLINDER_Z) {
        D.mbox[b][2] = -1.f;
        continue;
      }
      if (D.mbox[b][e] < 0.f) continue;
      const double h = grow * (std::fabs(s.c[e] - c[e]) + s.radius) + 2.0;
      D.mbox[b][e] = std::max(D.mbox[b][e], static_cast<float>(h));
    }
  }
}

Layout3 layout3(const lbm3_params &p, int nb) {
  Layout3 L;
  const size_t pitch = up(static_cast<size_t>(p.nx), kPitchAlign);
  const size_t cells = pitch * p.ny * p.nz;
  const int cap = p.force_capacity > 0 ? p.force_capacity : 8192;
  L.lat = up(nq_of(p) * cells * esize(p.storage), 256);
  size_t o = 2 * L.lat;
  L.mask_off = o;
  o += up(cells, 256);
  L.fvp_off = o;
  o += up(cells * 3 * (p.storage == LBM_F64 ? 8 : 4), 256);
  L.bodies_off = o;
  o += up(sizeof(double) * 9 * std::max(1, nb), 256);
  L.bodiesf_off = o;
  o += up(sizeof(float) * 9 * std::max(1, nb), 256);
  L.ring_off = o;
  o += up(p.force_every > 0 ? sizeof(double) * 3 * std::max(1, nb) * cap : 16, 256);
  L.status_off = o;
  o += 256;
  L.moving_off = o;
  if (p.moving) o += moving_bytes3();
  L.total = o;
  return L;
}

template <typename T> void fill3(Const3<T> &c, int q, double omp, double omm, double eta, double rho0, double scale) {
  const double w0 = w_of(q, 0), w1 = w_of(q, 1), w2 = w_of(q, 7);
  c.one_m_omp = T(1.0 - omp);
  c.hp = T(0.5 * omp);
  c.hm = T(0.5 * omm);
  c.inv_2eta1 = T(1.0 / (2.0 * eta + 1.0));
  c.rho0 = T(rho0 * scale);
  c.pw0 = T(omp * w0);
  c.pw1 = T(omp * w1);
  c.pw2 = T(omp * w2);
  c.mw1 = T(3.0 * omm * w1);
  c.mw2 = T(3.0 * omm * w2);
  c.kw0 = T((1.0 - 0.5 * omp) * w0);
  c.kw1 = T((1.0 - 0.5 * omp) * w1);
  c.kw2 = T((1.0 - 0.5 * omp) * w2);
  c.qw1 = T(3.0 * (1.0 - 0.5 * omm) * w1);
  c.qw2 = T(3.0 * (1.0 - 0.5 * omm) * w2);
  c.wr0 = T(w0 * rho0);
  c.wr1 = T(w1 * rho0);
  c.wr2 = T(w2 * rho0);
}

}  // namespace

struct lbm3_domain {
  lbm3_params p{};
  int nbodies = 0, pitch = 0;
  cudaStream_t st = nullptr;
  lbm_alloc_fn afn = nullptr;
  lbm_free_fn ffn = nullptr;
  void *actx = nullptr;
  void *block = nullptr, *frows = nullptr, *rowsum = nullptr;
  std::vector<Shape3Dev> hshapes;  // moving domains: the reference shapes (body boxes)
  Dom3 h{};
  Dom3 hpar[2]{};  // sweep parameters reading lattice 0 resp. 1
  Dom3 *d_dom = nullptr;
  long long done = 0, drained = 0;
  int parity = 0;
  int grid = 0;      // sweep blocks: a persistent grid, every resident block of every SM
  int pipe = 0;      // sweep register budget (pipeline 0, 3 or 4)
  int sms = 0;       // multiprocessors of the device
  int aux_grid = 0;  // force-row reduction blocks
  int move_blocks = 0;  // blocks per body of the moving-domain kernels
  void *get(size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (afn) return afn(bytes, actx);
    void *q = nullptr;
    if (cudaMallocAsync(&q, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return q;
  }
  void put(void *q) {
    if (!q) return;
    if (ffn) ffn(q, actx);
    else cudaFreeAsync(q, st);
  }
};

namespace {

cudaError_t launch_sweep3_pipe(lbm3_domain *d, int pipe, long long n, int par) {
  const int q = nq_of(d->p);
  const bool def = d->h.deform != 0u;
  switch (d->p.storage) {
    case LBM_F64: return launch_sweep3_f64(q, pipe, def, d->grid, d->st, d->hpar[par], n, par);
    case LBM_F32: return launch_sweep3_f32(q, pipe, def, d->grid, d->st, d->hpar[par], n, par);
    case LBM_F16S: return launch_sweep3_f16s(q, pipe, def, d->grid, d->st, d->hpar[par], n, par);
    case LBM_BF16S: return launch_sweep3_bf16s(q, pipe, def, d->grid, d->st, d->hpar[par], n, par);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sweep3(lbm3_domain *d, long long n, int par) { return launch_sweep3_pipe(d, d->pipe, n, par); }

cudaError_t launch_forces3(lbm3_domain *d, long long n) {
  if (d->p.force_every <= 0 || (n + 1) % d->p.force_every != 0 || d->nbodies == 0) return cudaSuccess;
  const long long entry = (n + 1) / d->p.force_every - 1;
  if (d->p.moving) {
    const dim3 g(d->move_blocks, d->nbodies);
    if (d->p.storage == LBM_F64) mforce3_kernel<double><<<g, kMoveThreads3, 0, d->st>>>(d->h, n, entry);
    else mforce3_kernel<float><<<g, kMoveThreads3, 0, d->st>>>(d->h, n, entry);
    return cudaGetLastError();
  }
  if (d->h.nfrows == 0)
    return cudaMemsetAsync(d->h.ring + (entry % d->h.force_cap) * d->nbodies * 3, 0,
                           sizeof(double) * 3 * d->nbodies, d->st);
  if (d->p.storage == LBM_F64) rows3_kernel<double><<<d->aux_grid, kRowsThreads, 0, d->st>>>(d->h, entry);
  else rows3_kernel<float><<<d->aux_grid, kRowsThreads, 0, d->st>>>(d->h, entry);
  return cudaGetLastError();
}

// a moving domain's geometry for the next step (after the forces of step n)
cudaError_t launch_move3(lbm3_domain *d, long long n) {
  if (!d->p.moving || d->nbodies == 0) return cudaSuccess;
  mmove3_kernel<<<dim3(d->move_blocks, d->nbodies), kMoveThreads3, 0, d->st>>>(d->h, n);
  return cudaGetLastError();
}

lbm_status validate3(const lbm3_params *p, int nb, int ns, const lbm3_shape *shapes) {
  if (!p) return fail3(LBM_EINVAL, "params is NULL");
  if (p->nx < 3 || p->ny < 3 || p->nz < 3) return fail3(LBM_EINVAL, "nx, ny, nz must be >= 3");
  if (p->ny > 65535 || p->nz > 65535) return fail3(LBM_EINVAL, "ny and nz must be <= 65535");
  if (static_cast<double>(up(p->nx, kPitchAlign)) * p->ny * p->nz > 1.0e9)
    return fail3(LBM_EINVAL, "grid too large (more than 1e9 padded nodes)");
  if (esize(p->storage) == 0) return fail3(LBM_EINVAL, "unknown storage %d", p->storage);
  if (p->lattice != 0 && p->lattice != 15 && p->lattice != 19)
    return fail3(LBM_EINVAL, "lattice must be 15 (D3Q15) or 19 (D3Q19; 0 selects it too)");
  const double tau = p->nu > 0 ? 3.0 * p->nu + 0.5 : p->tau_plus;
  if (!(tau > 0.5)) return fail3(LBM_EINVAL, "tau_plus must exceed 1/2");
  if (!(p->magic_lambda > 0) || !(p->eta > 0) || !(p->rho0 > 0)) return fail3(LBM_EINVAL, "Lambda, eta, rho0 must be > 0");
  if (p->west != LBM_PERIODIC && p->west != LBM_INLET_EQ) return fail3(LBM_EINVAL, "west edge must be PERIODIC or INLET_EQ");
  if (p->east != LBM_PERIODIC && p->east != LBM_OUTFLOW_ZG) return fail3(LBM_EINVAL, "east edge must be PERIODIC or OUTFLOW_ZG");
  if ((p->west == LBM_PERIODIC) != (p->east == LBM_PERIODIC)) return fail3(LBM_EINVAL, "x edges: both periodic or neither");
  const int32_t yz[4] = {p->south, p->north, p->bottom, p->top};
  for (int q = 0; q < 4; ++q)
    if (yz[q] != LBM_PERIODIC && yz[q] != LBM_FREE_SLIP) return fail3(LBM_EINVAL, "y and z edges must be PERIODIC or FREE_SLIP");
  if ((p->south == LBM_PERIODIC) != (p->north == LBM_PERIODIC) || (p->bottom == LBM_PERIODIC) != (p->top == LBM_PERIODIC))
    return fail3(LBM_EINVAL, "y and z edges: both periodic or neither");
  if (nb < 0 || nb > 255) return fail3(LBM_EINVAL, "nbodies must be in [0, 255]");
  if (ns < 0 || (ns > 0 && !shapes)) return fail3(LBM_EINVAL, "shapes");
  for (int q = 0; q < ns; ++q) {
    if (shapes[q].kind != LBM3_SHAPE_SPHERE && shapes[q].kind != LBM3_SHAPE_CYLINDER_Z)
      return fail3(LBM_EINVAL, "shape %d: unknown kind", q);
    if (shapes[q].body < 1 || shapes[q].body > nb) return fail3(LBM_EINVAL, "shape %d: body id not in [1, %d]", q, nb);
  }
  if (p->force_every < 0 || p->force_capacity < 0) return fail3(LBM_EINVAL, "force_every/capacity must be >= 0");
  if (p->moving != 0 && p->moving != 1) return fail3(LBM_EINVAL, "moving must be 0 or 1");
  if (p->moving && (nb > kMaxMoving3 || ns > kMaxShapes3))
    return fail3(LBM_EINVAL, "a moving 3D domain has at most %d bodies and %d shapes", kMaxMoving3, kMaxShapes3);
  return LBM_OK;
}

// resident blocks per SM of the sweep in one pipeline (0: not available)
int sweep3_fits(int q, int storage, int pipe) {
  switch (storage) {
    case LBM_F64: return sweep3_fits_f64(q, pipe);
    case LBM_F32: return sweep3_fits_f32(q, pipe);
    case LBM_F16S: return sweep3_fits_f16s(q, pipe);
    case LBM_BF16S: return sweep3_fits_bf16s(q, pipe);
  }
  return 0;
}

template <int Q, int S> void launch_init3_as(lbm3_domain *d, void *lat, const lbm3_params *p, int nrows) {
  dim3 g((d->pitch + 127) / 128, Q, std::min(nrows, 4096));
  init3_kernel<Q, S><<<g, 128, 0, d->st>>>(static_cast<typename Codec<S>::E *>(lat), p->nx, nrows, d->pitch,
                                            p->rho0, p->u0[0], p->u0[1], p->u0[2]);
}

template <int Q> void launch_init3_q(lbm3_domain *d, void *lat, const lbm3_params *p, int nrows) {
  switch (p->storage) {
    case LBM_F64: launch_init3_as<Q, LBM_F64>(d, lat, p, nrows); break;
    case LBM_F32: launch_init3_as<Q, LBM_F32>(d, lat, p, nrows); break;
    case LBM_F16S: launch_init3_as<Q, LBM_F16S>(d, lat, p, nrows); break;
    case LBM_BF16S: launch_init3_as<Q, LBM_BF16S>(d, lat, p, nrows); break;
  }
}

template <int Q, int S> void launch_moments3_as(lbm3_domain *d, double *t0, double *t1, double *t2, double *t3) {
  dim3 g((d->p.nx + 127) / 128, d->p.ny, d->p.nz);
  moments3_kernel<Q, S><<<g, 128, 0, d->st>>>(d->d_dom, d->parity, t0, t1, t2, t3);
}

template <int Q> void launch_moments3_q(lbm3_domain *d, double *t0, double *t1, double *t2, double *t3) {
  switch (d->p.storage) {
    case LBM_F64: launch_moments3_as<Q, LBM_F64>(d, t0, t1, t2, t3); break;
    case LBM_F32: launch_moments3_as<Q, LBM_F32>(d, t0, t1, t2, t3); break;
    case LBM_F16S: launch_moments3_as<Q, LBM_F16S>(d, t0, t1, t2, t3); break;
    case LBM_BF16S: launch_moments3_as<Q, LBM_BF16S>(d, t0, t1, t2, t3); break;
  }
}

lbm_status read_status3(lbm3_domain *d) {
  int32_t status = 0;
  LBM3_CUDA(cudaMemcpyAsync(&status, d->h.status, sizeof(int32_t), cudaMemcpyDeviceToHost, d->st));
  LBM3_CUDA(cudaStreamSynchronize(d->st));
  if (status & 1) return fail3(LBM_EUNSTABLE, "3D domain diverged (rho out of range or not finite)");
  return LBM_OK;
}

// A batch of fixed-geometry 3D domains of one storage and lattice (lbm3_batch_*): every
// slot is a domain of its own (lbm3_domain: memory, initial state, rasteriser, force
// ring). A step is one persistent sweep launch per group of up to kGroup3 domains that
// still have steps left, their parameters in the launch's, then one force-reduction
// launch per group.
struct Batch3 {
  int max_domains = 0, storage = 0, q = 19, pipe = 0, sms = 0, grid = 0;
  size_t budget = 0, bytes_in_use = 0;
  cudaStream_t st = nullptr;
  lbm_alloc_fn afn = nullptr;
  lbm_free_fn ffn = nullptr;
  void *actx = nullptr;
  std::vector<lbm3_domain *> slot;  // nullptr: free
  std::vector<long long> target;    // step target per slot
  std::vector<size_t> bytes;        // lbm3_domain_bytes per slot
  uint32_t *d_ctr = nullptr;        // [groups][2] work-item counters
  long long launches = 0;
  void *get(size_t n) {
    if (n == 0) n = 256;
    if (afn) return afn(n, actx);
    void *q = nullptr;
    if (cudaMallocAsync(&q, n, st) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return q;
  }
  void put(void *q) {
    if (!q) return;
    if (ffn) ffn(q, actx);
    else cudaFreeAsync(q, st);
  }
};

int groups3(int max_domains) { return (max_domains + kGroup3 - 1) / kGroup3; }

cudaError_t launch_sweep3b(Batch3 *b, const Batch3Args &a) {
  switch (b->storage) {
    case LBM_F64: return launch_sweep3b_f64(b->q, b->pipe, b->grid, b->st, a);
    case LBM_F32: return launch_sweep3b_f32(b->q, b->pipe, b->grid, b->st, a);
    case LBM_F16S: return launch_sweep3b_f16s(b->q, b->pipe, b->grid, b->st, a);
    case LBM_BF16S: return launch_sweep3b_bf16s(b->q, b->pipe, b->grid, b->st, a);
  }
  return cudaErrorInvalidValue;
}

int sweep3b_fits(int q, int storage, int pipe) {
  switch (storage) {
    case LBM_F64: return sweep3b_fits_f64(q, pipe);
    case LBM_F32: return sweep3b_fits_f32(q, pipe);
    case LBM_F16S: return sweep3b_fits_f16s(q, pipe);
    case LBM_BF16S: return sweep3b_fits_bf16s(q, pipe);
  }
  return 0;
}

// One step (index within the chunk s) of the domains listed in `ks`: the sweep, then the
// force entries that fall due.
lbm_status batch3_step(Batch3 &b, const std::vector<int> &ks, long long s, int group) {
  const int strip = 32 * (b.storage == LBM_F64 ? 2 : 4);
  Batch3Args a{};
  long long acc = 0;
  a.ndom = static_cast<int32_t>(ks.size());
  for (int i = 0; i < a.ndom; ++i) {
    const lbm3_domain *d = b.slot[ks[i]];
    const long long n = d->done + s;
    a.dom[i] = d->hpar[(d->parity + static_cast<int>(s & 1)) & 1];
    a.n[i] = n;
    a.base[i] = static_cast<int32_t>(acc);
    acc += static_cast<long long>(d->p.ny) * d->p.nz * ((d->p.nx + strip - 1) / strip);
  }
  if (acc >= (1ll << 31)) return fail3(LBM_EINVAL, "a group of the batch holds 2^31 strips or more");
  a.base[a.ndom] = static_cast<int32_t>(acc);
  a.ctr = b.d_ctr + 2 * group;
  LBM3_CUDA(launch_sweep3b(&b, a));
  ++b.launches;
  Rows3Args r{};
  int gx = 1;
  for (int i = 0; i < a.ndom; ++i) {
    const lbm3_domain *d = b.slot[ks[i]];
    const long long n = d->done + s;
    if (d->p.force_every <= 0 || (n + 1) % d->p.force_every != 0 || d->nbodies == 0) continue;
    Rows3Dom &x = r.dom[r.ndom++];
    x.frows = d->h.frows;
    x.mask = d->h.mask;
    x.fvp = d->h.fvp;
    x.rowsum = d->h.rowsum;
    x.ring = d->h.ring;
    x.rows_done = d->h.rows_done;
    x.entry = (n + 1) / d->p.force_every - 1;
    x.pitch = d->h.pitch;
    x.nfrows = d->h.nfrows;
    x.nbodies = d->nbodies;
    x.force_cap = d->h.force_cap;
    gx = std::max(gx, d->aux_grid);
  }
  if (r.ndom > 0) {
    const dim3 g(gx, r.ndom);
    if (b.storage == LBM_F64) rows3_batch_kernel<double><<<g, kRowsThreads, 0, b.st>>>(r);
    else rows3_batch_kernel<float><<<g, kRowsThreads, 0, b.st>>>(r);
    LBM3_CUDA(cudaGetLastError());
    ++b.launches;
  }
  return LBM_OK;
}

}  // namespace

struct lbm3_batch {
  Batch3 b;
};

extern "C" {

void lbm3_params_default(lbm3_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->nx = p->ny = p->nz = 32;
  p->nu = 0.1;
  p->tau_plus = 0.8;
  p->magic_lambda = 3.0 / 16.0;
  p->eta = 1e-4;
  p->rho0 = 1.0;
  p->storage = LBM_F32;
  p->force_every = 1;
  p->force_capacity = 8192;
  p->lattice = 19;
}

size_t lbm3_domain_bytes(const lbm3_params *p, int32_t nbodies) {
  if (!p || esize(p->storage) == 0 || p->nx < 1 || p->ny < 1 || p->nz < 1) return 0;
  return layout3(*p, std::max(0, nbodies)).total;
}

lbm_status lbm3_domain_create(const lbm3_params *p, const lbm3_shape *shapes, int32_t nshapes,
                              const lbm3_body *bodies, int32_t nbodies, void *cuda_stream,
                              lbm_alloc_fn alloc, lbm_free_fn free_fn, void *alloc_ctx,
                              lbm3_domain **out) {
  if (!out) return fail3(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  lbm_status rc = validate3(p, nbodies, nshapes, shapes);
  if (rc != LBM_OK) return rc;
  if (nbodies > 0 && !bodies) return fail3(LBM_EINVAL, "bodies is NULL");
  int dev = 0, sms = 0;
  LBM3_CUDA(cudaGetDevice(&dev));
  LBM3_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  lbm3_domain *d = new lbm3_domain();
  d->p = *p;
  if (d->p.force_capacity == 0) d->p.force_capacity = 8192;
  d->nbodies = nbodies;
  d->pitch = static_cast<int>(up(p->nx, kPitchAlign));
  d->st = static_cast<cudaStream_t>(cuda_stream);
  d->afn = alloc;
  d->ffn = free_fn;
  d->actx = alloc_ctx;
  const Layout3 L = layout3(d->p, nbodies);
  void *dsh = nullptr;  // shape table (admission only)
  auto bail = [&](lbm_status r) {
    cudaStreamSynchronize(d->st);
    d->put(dsh);
    d->put(d->block);
    d->put(d->frows);
    d->put(d->rowsum);
    d->put(d->d_dom);
    delete d;
    return r;
  };
#define ADM3(call)                                                                           \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return bail(fail3(LBM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_))); \
  } while (0)
  d->block = d->get(L.total);
  d->d_dom = static_cast<Dom3 *>(d->get(sizeof(Dom3)));
  if (!d->block || !d->d_dom) return bail(fail3(LBM_ENOMEM, "device allocation of %zu bytes failed", L.total));
  char *base = static_cast<char *>(d->block);
  Dom3 &D = d->h;
  D.lat[0] = base;
  D.lat[1] = base + L.lat;
  D.mask = reinterpret_cast<uint8_t *>(base + L.mask_off);
  D.fvp = base + L.fvp_off;
  D.bodies = reinterpret_cast<double *>(base + L.bodies_off);
  D.bodies_f = reinterpret_cast<float *>(base + L.bodiesf_off);
  D.ring = reinterpret_cast<double *>(base + L.ring_off);
  D.status = reinterpret_cast<int32_t *>(base + L.status_off);
  D.rows_done = reinterpret_cast<uint32_t *>(base + L.status_off + 4);
  D.items = reinterpret_cast<uint32_t *>(base + L.status_off + 8);
  D.nx = p->nx;
  D.ny = p->ny;
  D.nz = p->nz;
  D.pitch = d->pitch;
  D.west = p->west;
  D.east = p->east;
  D.south = p->south;
  D.north = p->north;
  D.bottom = p->bottom;
  D.top = p->top;
  D.nbodies = nbodies;
  D.force_every = p->force_every;
  D.force_cap = d->p.force_capacity;
  const double tau_s = p->nu > 0 ? 3.0 * p->nu + 0.5 : p->tau_plus;
  const double tau_a = 0.5 + p->magic_lambda / (tau_s - 0.5);
  const double omp = 1.0 / tau_s, omm = 1.0 / tau_a;
  const bool shifted = p->storage == LBM_F16S || p->storage == LBM_BF16S;
  const double scale = p->storage == LBM_F16S ? double(kF16Scale) : 1.0;
  const int nq = nq_of(*p);
  fill3(D.cd, nq, omp, omm, p->eta, p->rho0, 1.0);
  fill3(D.cf, nq, omp, omm, p->eta, p->rho0, scale);
  {
    const Const3<float> &c = D.cf;
    auto two = [](float x) { return make_float2(x, x); };
    D.pc = Pair3{two(c.one_m_omp), two(c.hp), two(c.hm), two(c.rho0), two(c.pw0),
                 two(c.pw1), two(c.pw2), two(c.mw1), two(c.mw2)};
  }
  {
    // inlet ghost f^eq(rho0, u_in) in compute space, held as the storage would hold it
    const double *u = p->u_in;
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int a = 0; a < nq; ++a) {
      const double wa = w_of(nq, a);
      const double eu = e_of(nq, a, 0) * u[0] + e_of(nq, a, 1) * u[1] + e_of(nq, a, 2) * u[2];
      const double dev = p->rho0 * wa * (3.0 * eu + 4.5 * eu * eu - 1.5 * usq);
      D.cd.ghost[a] = p->rho0 * wa + dev;
      float gf;
      if (p->storage == LBM_F32) gf = float(p->rho0 * wa + dev) - float(wa * p->rho0);
      else if (p->storage == LBM_F16S) gf = __half2float(__float2half_rn(float(dev * scale)));
      else if (p->storage == LBM_BF16S) gf = __bfloat162float(__float2bfloat16_rn(float(dev)));
      else gf = float(dev);
      D.cf.ghost[a] = gf;
      (void)shifted;
    }
  }
  cudaStream_t st = d->st;
  // body tables (before the mask: a moving domain's shapes are placed from them)
  std::vector<double> hb(9 * std::max(1, nbodies), 0.0);
  for (int q = 0; q < nbodies; ++q)
    for (int e = 0; e < 3; ++e) {
      hb[9 * q + e] = bodies[q].c[e];
      hb[9 * q + 3 + e] = bodies[q].v[e];
      hb[9 * q + 6 + e] = bodies[q].w[e];
    }
  if (p->moving)
    for (int q = 0; q < nbodies; ++q)
      for (int e = 0; e < 3; ++e)
        if (!(std::fabs(bodies[q].v[e]) <= 1.0))
          return bail(fail3(LBM_EINVAL, "a moving body moves at most one node per step along each axis"));
  std::vector<float> hbf(hb.begin(), hb.end());
  ADM3(cudaMemcpyAsync(D.bodies, hb.data(), sizeof(double) * hb.size(), cudaMemcpyHostToDevice, st));
  ADM3(cudaMemcpyAsync(D.bodies_f, hbf.data(), sizeof(float) * hbf.size(), cudaMemcpyHostToDevice, st));
  // shapes -> mask
  std::vector<Shape3Dev> hs(std::max(1, nshapes));
  for (int q = 0; q < nshapes; ++q)
    hs[q] = Shape3Dev{shapes[q].kind, shapes[q].body, {shapes[q].c[0], shapes[q].c[1], shapes[q].c[2]}, shapes[q].radius};
  D.moving = p->moving;
  D.nshapes = p->moving ? nshapes : 0;
  if (p->moving) {
    // kept for the per-step geometry: shapes, reference centres, force partials, counters
    char *mb = base + L.moving_off;
    D.shapes = reinterpret_cast<const Shape3Dev *>(mb);
    mb += up(sizeof(Shape3Dev) * kMaxShapes3, 256);
    D.centre0 = reinterpret_cast<const double *>(mb);
    mb += up(sizeof(double) * 3 * kMaxMoving3, 256);
    D.mpart = reinterpret_cast<double *>(mb);
    mb += up(sizeof(double) * 3 * kMaxMoving3 * kMaxMoveBlocks3, 256);
    D.mcount = reinterpret_cast<uint32_t *>(mb);
    mb += up(sizeof(uint32_t) * kMaxMoving3, 256);
    D.fsi = reinterpret_cast<double *>(mb);
    mb += up(sizeof(double) * 9 * 2 * kMaxMoving3, 256);
    D.fsi_par = reinterpret_cast<const double *>(mb);
    D.coupled = 0u;
    mb += up(sizeof(double) * 12 * kMaxMoving3, 256);
    D.dpar = reinterpret_cast<const double *>(mb);
    D.kappa = reinterpret_cast<double *>(mb) + 2 * kMaxMoving3;
    D.kappa_f = reinterpret_cast<float *>(D.kappa + kMaxMoving3);
    D.deform = 0u;
    ADM3(cudaMemsetAsync(base + L.moving_off, 0, moving_bytes3(), st));
    ADM3(cudaMemcpyAsync(const_cast<Shape3Dev *>(D.shapes), hs.data(), sizeof(Shape3Dev) * nshapes,
                         cudaMemcpyHostToDevice, st));
    std::vector<double> c0(3 * kMaxMoving3, 0.0);
    for (int q = 0; q < nbodies; ++q)
      for (int e = 0; e < 3; ++e) c0[3 * q + e] = bodies[q].c[e];
    ADM3(cudaMemcpyAsync(const_cast<double *>(D.centre0), c0.data(), sizeof(double) * c0.size(),
                         cudaMemcpyHostToDevice, st));
    d->hshapes.assign(hs.begin(), hs.begin() + nshapes);
    for (int b = 0; b < kMaxMoving3; ++b) set_mbox3(D, d->hshapes, b, b < nbodies ? bodies[b].c : nullptr, 1.0);
  }
  dsh = d->get(sizeof(Shape3Dev) * hs.size());
  if (!dsh) return bail(fail3(LBM_ENOMEM, "shape buffer allocation failed"));
  ADM3(cudaMemcpyAsync(dsh, hs.data(), sizeof(Shape3Dev) * hs.size(), cudaMemcpyHostToDevice, st));
  rasterize3_kernel<<<dim3((d->pitch + 127) / 128, p->ny, p->nz), 128, 0, st>>>(
      D.mask, p->nx, p->ny, p->nz, d->pitch, static_cast<const Shape3Dev *>(dsh), nshapes,
      Place3{D.bodies, nbodies, 0u, nullptr, nullptr, 0u, nullptr}, 0);
  ADM3(cudaGetLastError());
  // rows that hold solid nodes (the force reduction visits only those)
  const size_t cells = static_cast<size_t>(d->pitch) * p->ny * p->nz;
  std::vector<uint8_t> hm(cells);
  ADM3(cudaMemcpyAsync(hm.data(), D.mask, cells, cudaMemcpyDeviceToHost, st));
  ADM3(cudaStreamSynchronize(st));
  d->put(dsh);
  dsh = nullptr;
  std::vector<int4> rows;  // (row, first solid column, last solid column + 1, 0)
  for (int r = 0; r < p->ny * p->nz; ++r) {
    const uint8_t *m = hm.data() + static_cast<size_t>(r) * d->pitch;
    int lo = -1, hi = -1;
    for (int i = 0; i < p->nx; ++i)
      if (m[i]) {
        if (m[i] > nbodies) return bail(fail3(LBM_EINVAL, "mask holds body id %d > %d", m[i], nbodies));
        if (lo < 0) lo = i;
        hi = i + 1;
      }
    if (lo >= 0) rows.push_back(make_int4(r, lo, hi, 0));
  }
  D.nfrows = static_cast<int32_t>(rows.size());
  d->frows = d->get(sizeof(int4) * std::max<size_t>(1, rows.size()));
  d->rowsum = d->get(sizeof(double) * 3 * std::max<size_t>(1, rows.size()) * std::max(1, nbodies));
  if (!d->frows || !d->rowsum) return bail(fail3(LBM_ENOMEM, "force row lists allocation failed"));
  D.frows = static_cast<const int4 *>(d->frows);
  D.rowsum = static_cast<double *>(d->rowsum);
  if (!rows.empty())
    ADM3(cudaMemcpyAsync(d->frows, rows.data(), sizeof(int4) * rows.size(), cudaMemcpyHostToDevice, st));
  // initial state: lattice A = f^eq(rho0, u0); lattice B, F_VP, ring, status zero
  {
    const int nrows = p->ny * p->nz;
    if (nq == 15) launch_init3_q<15>(d, D.lat[0], p, nrows);
    else launch_init3_q<19>(d, D.lat[0], p, nrows);
    ADM3(cudaGetLastError());
  }
  ADM3(cudaMemsetAsync(D.lat[1], 0, L.lat, st));
  ADM3(cudaMemsetAsync(D.fvp, 0, L.bodies_off - L.fvp_off, st));
  ADM3(cudaMemsetAsync(D.ring, 0, L.status_off - L.ring_off, st));
  // status, the reduction's block counter and the sweep's work-item counters
  ADM3(cudaMemsetAsync(D.status, 0, 16, st));
  ADM3(cudaMemcpyAsync(d->d_dom, &D, sizeof(Dom3), cudaMemcpyHostToDevice, st));
  ADM3(cudaStreamSynchronize(st));
#undef ADM3
  {
    const size_t dir_bytes = esize(p->storage) * static_cast<size_t>(d->pitch) * p->ny * p->nz;
    for (int par = 0; par < 2; ++par) {
      d->hpar[par] = D;
      for (int a = 0; a < nq; ++a) {
        d->hpar[par].src[a] = static_cast<const char *>(D.lat[par]) + a * dir_bytes;
        d->hpar[par].dst[a] = static_cast<char *>(D.lat[par ^ 1]) + a * dir_bytes;
      }
    }
  }
  // default register budget, measured on a 384 x 128 x 128 sphere channel: 20 resident
  // warps for the 16-bit D3Q15 sweep (80.5 against 86.1 us), 16 for the 16-bit D3Q19
  // sweep (its 20- and 24-warp budgets spill: 135 and 156 against 100 us)
  const bool k16 = p->storage == LBM_F16S || p->storage == LBM_BF16S;
  d->pipe = (k16 && nq == 15 && sweep3_fits(nq, p->storage, 3) > 0) ? 3 : 0;
  d->sms = sms;
  d->grid = std::max(1, sweep3_fits(nq, p->storage, d->pipe)) * sms;
  // force reduction: one warp per listed row, at most one block per SM
  d->aux_grid = std::max(1, std::min(sms, (D.nfrows + kRowsThreads / 32 - 1) / (kRowsThreads / 32)));
  // moving domains: 64 blocks per body (one row per warp for boxes of up to 512 rows; 211
  // blocks for the 41 x 41 rows of a D = 32 sphere measured slower)
  d->move_blocks = 64;
  static_assert(kMaxMoveBlocks3 <= kMoveThreads3, "the last block loads one partial per thread");
  *out = d;
  return LBM_OK;
}

lbm_status lbm3_step(lbm3_domain *d, int64_t nsteps) {
  if (!d) return fail3(LBM_EINVAL, "domain is NULL");
  if (nsteps < 0) return fail3(LBM_EINVAL, "nsteps must be >= 0");
  if (d->p.force_every > 0) {
    const long long produced = (d->done + nsteps) / d->p.force_every;
    if (produced - d->drained > d->p.force_capacity)
      return fail3(LBM_EBUSY, "force ring would overflow");
  }
  for (long long s = 0; s < nsteps; ++s) {
    const long long n = d->done + s;
    LBM3_CUDA(launch_sweep3(d, n, (d->parity + static_cast<int>(s & 1)) & 1));
    LBM3_CUDA(launch_forces3(d, n));
    LBM3_CUDA(launch_move3(d, n));
  }
  d->done += nsteps;
  d->parity = static_cast<int>((d->parity + nsteps) & 1);
  return LBM_OK;
}

lbm_status lbm3_profile(lbm3_domain *d, int32_t steps, double *sweep_us, double *force_us) {
  if (!d) return fail3(LBM_EINVAL, "domain is NULL");
  if (steps < 1) return fail3(LBM_EINVAL, "steps must be >= 1");
  if (d->p.force_every > 0 && (d->done + steps) / d->p.force_every - d->drained > d->p.force_capacity)
    return fail3(LBM_EBUSY, "force ring would overflow");
  std::vector<cudaEvent_t> ev(3 * steps);
  for (auto &e : ev) LBM3_CUDA(cudaEventCreate(&e));
  for (int s = 0; s < steps; ++s) {
    const long long n = d->done + s;
    cudaEventRecord(ev[3 * s], d->st);
    LBM3_CUDA(launch_sweep3(d, n, (d->parity + (s & 1)) & 1));
    cudaEventRecord(ev[3 * s + 1], d->st);
    LBM3_CUDA(launch_forces3(d, n));
    LBM3_CUDA(launch_move3(d, n));
    cudaEventRecord(ev[3 * s + 2], d->st);
  }
  LBM3_CUDA(cudaStreamSynchronize(d->st));
  double a = 0.0, c = 0.0;
  for (int s = 0; s < steps; ++s) {
    float x = 0.f, y = 0.f;
    cudaEventElapsedTime(&x, ev[3 * s], ev[3 * s + 1]);
    cudaEventElapsedTime(&y, ev[3 * s + 1], ev[3 * s + 2]);
    a += x;
    c += y;
  }
  for (auto &e : ev) cudaEventDestroy(e);
  d->done += steps;
  d->parity = (d->parity + steps) & 1;
  if (sweep_us) *sweep_us = 1000.0 * a / steps;
  if (force_us) *force_us = 1000.0 * c / steps;
  return LBM_OK;
}

lbm_status lbm3_set_tile(lbm3_domain *d, int32_t pipeline) {
  if (!d) return fail3(LBM_EINVAL, "domain is NULL");
  if (pipeline != 0 && pipeline != 3 && pipeline != 4) return fail3(LBM_EINVAL, "pipeline must be 0, 3 or 4");
  const int fits = sweep3_fits(nq_of(d->p), d->p.storage, pipeline);
  if (fits <= 0) return fail3(LBM_EINVAL, "pipeline %d is not available for storage %d", pipeline, d->p.storage);
  d->pipe = pipeline;
  d->grid = fits * d->sms;
  return LBM_OK;
}

lbm_status lbm3_get_tile(lbm3_domain *d, int32_t *pipeline) {
  if (!d || !pipeline) return fail3(LBM_EINVAL, "domain or pipeline is NULL");
  *pipeline = d->pipe;
  return LBM_OK;
}

lbm_status lbm3_autotune(lbm3_domain *d, int32_t reps, double *best_us) {
  if (!d) return fail3(LBM_EINVAL, "domain is NULL");
  if (reps < 1) return fail3(LBM_EINVAL, "reps must be >= 1");
  const int q = nq_of(d->p);
  cudaEvent_t e0, e1;
  LBM3_CUDA(cudaEventCreate(&e0));
  LBM3_CUDA(cudaEventCreate(&e1));
  double best = 1e300;
  int best_pipe = d->pipe;
  lbm_status rc = LBM_OK;
  const int keep_pipe = d->pipe, keep_grid = d->grid;
  for (int pipe : {0, 3, 4}) {
    const int fits = sweep3_fits(q, d->p.storage, pipe);
    if (fits <= 0) continue;
    d->pipe = pipe;
    d->grid = fits * d->sms;
    // the timing launches read the current lattice and write only the spare one
    for (int r = 0; r < 2 && rc == LBM_OK; ++r)
      if (launch_sweep3(d, d->done, d->parity) != cudaSuccess) rc = fail3(LBM_ECUDA, "autotune launch failed");
    cudaEventRecord(e0, d->st);
    for (int r = 0; r < reps && rc == LBM_OK; ++r)
      if (launch_sweep3(d, d->done, d->parity) != cudaSuccess) rc = fail3(LBM_ECUDA, "autotune launch failed");
    cudaEventRecord(e1, d->st);
    if (rc != LBM_OK) break;
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double us = 1000.0 * ms / reps;
    if (us < best) {
      best = us;
      best_pipe = pipe;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  d->pipe = keep_pipe;
  d->grid = keep_grid;
  if (rc != LBM_OK) return rc;
  rc = lbm3_set_tile(d, best_pipe);
  if (best_us) *best_us = best;
  return rc;
}

lbm_status lbm3_forces(lbm3_domain *d, double *out, int64_t max_entries, int64_t *written) {
  if (written) *written = 0;
  if (!d) return fail3(LBM_EINVAL, "domain is NULL");
  lbm_status rc = read_status3(d);
  const long long produced = d->p.force_every > 0 ? d->done / d->p.force_every : 0;
  const long long n = std::min(produced - d->drained, std::max<long long>(0, max_entries));
  if (n > 0 && !out) return fail3(LBM_EINVAL, "out is NULL");
  const size_t per = 3 * static_cast<size_t>(d->nbodies);
  long long copied = 0;
  while (copied < n && per > 0) {
    const long long e = d->drained + copied;
    const long long pos = e % d->p.force_capacity;
    const long long chunk = std::min(n - copied, static_cast<long long>(d->p.force_capacity) - pos);
    LBM3_CUDA(cudaMemcpyAsync(out + copied * per, d->h.ring + pos * per, sizeof(double) * per * chunk,
                              cudaMemcpyDeviceToHost, d->st));
    copied += chunk;
  }
  LBM3_CUDA(cudaStreamSynchronize(d->st));
  d->drained += n;
  if (written) *written = n;
  return rc;
}

lbm_status lbm3_moments(lbm3_domain *d, double *rho, double *ux, double *uy, double *uz) {
  if (!d) return fail3(LBM_EINVAL, "domain is NULL");
  const size_t cells = static_cast<size_t>(d->p.nx) * d->p.ny * d->p.nz;
  double *tmp = static_cast<double *>(d->get(sizeof(double) * 4 * cells));
  if (!tmp) return fail3(LBM_ENOMEM, "moments buffer allocation failed");
  double *t0 = tmp, *t1 = tmp + cells, *t2 = tmp + 2 * cells, *t3 = tmp + 3 * cells;
  if (nq_of(d->p) == 15) launch_moments3_q<15>(d, t0, t1, t2, t3);
  else launch_moments3_q<19>(d, t0, t1, t2, t3);
  cudaError_t e = cudaGetLastError();
  double *outs[4] = {rho, ux, uy, uz};
  for (int q = 0; q < 4 && e == cudaSuccess; ++q)
    if (outs[q]) e = cudaMemcpyAsync(outs[q], tmp + q * cells, sizeof(double) * cells, cudaMemcpyDefault, d->st);
  cudaStreamSynchronize(d->st);
  d->put(tmp);
  if (e != cudaSuccess) return fail3(LBM_ECUDA, "moments failed: %s", cudaGetErrorString(e));
  return read_status3(d);
}

static lbm_status pops3(lbm3_domain *d, void *out, const void *in, size_t bytes) {
  if (!d) return fail3(LBM_EINVAL, "domain is NULL");
  const size_t es = esize(d->p.storage);
  const size_t want = es * nq_of(d->p) * static_cast<size_t>(d->p.nx) * d->p.ny * d->p.nz;
  if (bytes != want) return fail3(LBM_EINVAL, "population buffer must be %zu bytes (got %zu)", want, bytes);
  char *lat = static_cast<char *>(d->h.lat[d->parity]);
  const size_t rowb = es * d->p.nx, pitchb = es * d->pitch;
  const size_t rows = static_cast<size_t>(nq_of(d->p)) * d->p.ny * d->p.nz;
  if (out) LBM3_CUDA(cudaMemcpy2DAsync(out, rowb, lat, pitchb, rowb, rows, cudaMemcpyDefault, d->st));
  else if (in) LBM3_CUDA(cudaMemcpy2DAsync(lat, pitchb, in, rowb, rowb, rows, cudaMemcpyDefault, d->st));
  else return fail3(LBM_EINVAL, "buffer is NULL");
  LBM3_CUDA(cudaStreamSynchronize(d->st));
  return LBM_OK;
}

lbm_status lbm3_get_populations(lbm3_domain *d, void *out, size_t bytes) {
  if (!out) return fail3(LBM_EINVAL, "out is NULL");
  return pops3(d, out, nullptr, bytes);
}

lbm_status lbm3_set_populations(lbm3_domain *d, const void *in, size_t bytes) {
  if (!in) return fail3(LBM_EINVAL, "in is NULL");
  return pops3(d, nullptr, in, bytes);
}

lbm_status lbm3_get_mask(lbm3_domain *d, uint8_t *out) {
  if (!d || !out) return fail3(LBM_EINVAL, "domain or out is NULL");
  LBM3_CUDA(cudaMemcpy2DAsync(out, d->p.nx, d->h.mask, d->pitch, d->p.nx,
                              static_cast<size_t>(d->p.ny) * d->p.nz, cudaMemcpyDefault, d->st));
  LBM3_CUDA(cudaStreamSynchronize(d->st));
  return LBM_OK;
}

lbm_status lbm3_steps_done(lbm3_domain *d, int64_t *steps) {
  if (!d) return fail3(LBM_EINVAL, "domain is NULL");
  if (steps) *steps = d->done;
  return LBM_OK;
}

static lbm_status place_at3(lbm3_domain *d, int64_t steps) {
  if (d->p.moving) {  // the mask and body table of that step index
    const Dom3 &D = d->h;
    const Place3 pl{D.bodies, d->nbodies, D.coupled,
                    D.fsi ? D.fsi + static_cast<size_t>(steps & 1) * kMaxMoving3 * 9 : nullptr, D.centre0, D.deform,
                    D.dpar};
    rasterize3_kernel<<<dim3((d->pitch + 127) / 128, d->p.ny, d->p.nz), 128, 0, d->st>>>(
        D.mask, d->p.nx, d->p.ny, d->p.nz, d->pitch, D.shapes, D.nshapes, pl, steps);
    LBM3_CUDA(cudaGetLastError());
    centres3_kernel<<<1, 32, 0, d->st>>>(d->d_dom, steps);
    LBM3_CUDA(cudaGetLastError());
  }
  LBM3_CUDA(cudaStreamSynchronize(d->st));
  d->done = steps;
  // entries before the index are gone; the ring slot of entry e stays e % capacity
  d->drained = d->p.force_every > 0 ? steps / d->p.force_every : 0;
  return LBM_OK;
}

lbm_status lbm3_set_steps_done(lbm3_domain *d, int64_t steps) {
  if (!d) return fail3(LBM_EINVAL, "domain is NULL");
  if (steps < 0) return fail3(LBM_EINVAL, "step index must be >= 0");
  if (d->h.coupled && steps != d->done)
    return fail3(LBM_EINVAL, "a domain with coupled bodies changes its step index through lbm3_restore_coupled");
  return place_at3(d, steps);
}

lbm_status lbm3_set_dynamics(lbm3_domain *d, int32_t body, const lbm3_body_dynamics *dyn) {
  if (!d || !dyn) return fail3(LBM_EINVAL, "domain or dynamics is NULL");
  if (!d->p.moving) return fail3(LBM_EINVAL, "coupled bodies need a moving domain");
  if (d->p.force_every != 1) return fail3(LBM_EINVAL, "coupled bodies need the force of every step (force_every = 1)");
  if (d->done != 0) return fail3(LBM_EINVAL, "dynamics are set before the first step");
  if (d->h.deform) return fail3(LBM_EINVAL, "a domain with pulsating bodies cannot have coupled bodies");
  if (body < 1 || body > d->nbodies) return fail3(LBM_EINVAL, "body %d outside 1..%d", body, d->nbodies);
  if (!(dyn->mass > 0.0) || !std::isfinite(dyn->mass)) return fail3(LBM_EINVAL, "mass must be finite and > 0");
  for (int e = 0; e < 3; ++e) {
    if (!(dyn->stiffness[e] >= 0.0) || !std::isfinite(dyn->stiffness[e]) || !(dyn->damping[e] >= 0.0) ||
        !std::isfinite(dyn->damping[e]))
      return fail3(LBM_EINVAL, "stiffness and damping must be finite and >= 0");
    if (dyn->free_axis[e] != 0 && dyn->free_axis[e] != 1) return fail3(LBM_EINVAL, "free_axis must be 0 or 1");
  }
  const int b = body - 1;
  double bt[9];
  LBM3_CUDA(cudaMemcpyAsync(bt, d->h.bodies + 9 * b, sizeof(bt), cudaMemcpyDeviceToHost, d->st));
  LBM3_CUDA(cudaStreamSynchronize(d->st));
  // state of index 0: the reference centre, the given velocity, no previous force
  const double st0[9] = {bt[0], bt[1], bt[2], bt[3], bt[4], bt[5], 0.0, 0.0, 0.0};
  const double par[12] = {dyn->mass, dyn->stiffness[0], dyn->stiffness[1], dyn->stiffness[2],
                          dyn->damping[0], dyn->damping[1], dyn->damping[2],
                          double(dyn->free_axis[0]), double(dyn->free_axis[1]), double(dyn->free_axis[2]), 0.0, 0.0};
  LBM3_CUDA(cudaMemcpyAsync(d->h.fsi + 9 * b, st0, sizeof(st0), cudaMemcpyHostToDevice, d->st));
  LBM3_CUDA(cudaMemcpyAsync(const_cast<double *>(d->h.fsi_par) + 12 * b, par, sizeof(par), cudaMemcpyHostToDevice,
                            d->st));
  d->h.coupled |= 1u << b;
  for (int q = 0; q < 2; ++q) d->hpar[q].coupled = d->h.coupled;
  LBM3_CUDA(cudaMemcpyAsync(d->d_dom, &d->h, sizeof(Dom3), cudaMemcpyHostToDevice, d->st));
  LBM3_CUDA(cudaStreamSynchronize(d->st));
  return LBM_OK;
}

lbm_status lbm3_set_deformation(lbm3_domain *d, int32_t body, double amplitude, double rate) {
  if (!d) return fail3(LBM_EINVAL, "domain is NULL");
  if (!d->p.moving) return fail3(LBM_EINVAL, "pulsating bodies need a moving domain");
  if (d->done != 0) return fail3(LBM_EINVAL, "a deformation is set before the first step");
  if (d->h.coupled) return fail3(LBM_EINVAL, "coupled bodies do not deform");
  if (body < 1 || body > d->nbodies) return fail3(LBM_EINVAL, "body %d outside 1..%d", body, d->nbodies);
  if (!(std::fabs(amplitude) < 1.0) || !std::isfinite(rate))
    return fail3(LBM_EINVAL, "the amplitude must satisfy |a| < 1 and the rate be finite");
  const int b = body - 1;
  for (const Shape3Dev &s : d->hshapes)
    if (s.body == body && s.kind != LBM3_SHAPE_SPHERE)
      return fail3(LBM_EINVAL, "a pulsating body is made of spheres (its dilation is isotropic)");
  double c0[3];
  LBM3_CUDA(cudaMemcpyAsync(c0, d->h.centre0 + 3 * b, sizeof(c0), cudaMemcpyDeviceToHost, d->st));
  LBM3_CUDA(cudaStreamSynchronize(d->st));
  const double par[2] = {amplitude, rate};
  LBM3_CUDA(cudaMemcpyAsync(const_cast<double *>(d->h.dpar) + 2 * b, par, sizeof(par), cudaMemcpyHostToDevice,
                            d->st));
  d->h.deform |= 1u << b;
  set_mbox3(d->h, d->hshapes, b, c0, 1.0 + std::fabs(amplitude));
  for (int q = 0; q < 2; ++q) {
    d->hpar[q].deform = d->h.deform;
    for (int e = 0; e < 3; ++e) d->hpar[q].mbox[b][e] = d->h.mbox[b][e];
  }
  LBM3_CUDA(cudaMemcpyAsync(d->d_dom, &d->h, sizeof(Dom3), cudaMemcpyHostToDevice, d->st));
  return place_at3(d, 0);  // the mask, centres and dilation rates of index 0
}

lbm_status lbm3_body_state(lbm3_domain *d, double *out) {
  if (!d || !out) return fail3(LBM_EINVAL, "domain or out is NULL");
  if (d->nbodies == 0) return LBM_OK;
  LBM3_CUDA(cudaMemcpyAsync(out, d->h.bodies, sizeof(double) * 9 * d->nbodies, cudaMemcpyDeviceToHost, d->st));
  LBM3_CUDA(cudaStreamSynchronize(d->st));
  return LBM_OK;
}

lbm_status lbm3_coupled_state(lbm3_domain *d, double *out) {
  if (!d || !out) return fail3(LBM_EINVAL, "domain or out is NULL");
  if (!d->h.coupled) return fail3(LBM_EINVAL, "the domain has no coupled body");
  std::vector<double> st(9 * kMaxMoving3);
  LBM3_CUDA(cudaMemcpyAsync(st.data(), d->h.fsi + static_cast<size_t>(d->done & 1) * kMaxMoving3 * 9,
                            sizeof(double) * st.size(), cudaMemcpyDeviceToHost, d->st));
  LBM3_CUDA(cudaStreamSynchronize(d->st));
  for (int b = 0; b < d->nbodies; ++b)
    for (int e = 0; e < 9; ++e) out[9 * b + e] = (d->h.coupled >> b & 1u) ? st[9 * b + e] : 0.0;
  return LBM_OK;
}

lbm_status lbm3_restore_coupled(lbm3_domain *d, int64_t steps, const double *in) {
  if (!d || !in) return fail3(LBM_EINVAL, "domain or state is NULL");
  if (!d->h.coupled) return fail3(LBM_EINVAL, "the domain has no coupled body");
  if (steps < 0) return fail3(LBM_EINVAL, "step index must be >= 0");
  for (int b = 0; b < d->nbodies; ++b)
    if (d->h.coupled >> b & 1u)
      for (int e = 0; e < 9; ++e)
        if (!std::isfinite(in[9 * b + e])) return fail3(LBM_EINVAL, "state of body %d is not finite", b + 1);
  double *cur = d->h.fsi + static_cast<size_t>(steps & 1) * kMaxMoving3 * 9;
  for (int b = 0; b < d->nbodies; ++b)
    if (d->h.coupled >> b & 1u)
      LBM3_CUDA(cudaMemcpyAsync(cur + 9 * b, in + 9 * b, sizeof(double) * 9, cudaMemcpyHostToDevice, d->st));
  return place_at3(d, steps);
}

lbm_status lbm3_domain_destroy(lbm3_domain *d) {
  if (!d) return LBM_OK;
  cudaStreamSynchronize(d->st);
  d->put(d->block);
  d->put(d->frows);
  d->put(d->rowsum);
  d->put(d->d_dom);
  cudaStreamSynchronize(d->st);
  delete d;
  return LBM_OK;
}

// ---- batches of fixed-geometry 3D domains -----------------------------------------------

lbm_status lbm3_batch_create(int32_t max_domains, size_t hbm_budget_bytes, int32_t storage, int32_t lattice,
                             void *cuda_stream, lbm_alloc_fn alloc, lbm_free_fn free_fn, void *alloc_ctx,
                             lbm3_batch **out) {
  if (!out) return fail3(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_domains < 1 || max_domains > 4096) return fail3(LBM_EINVAL, "max_domains must be in [1, 4096]");
  if (esize(storage) == 0) return fail3(LBM_EINVAL, "unknown storage %d", storage);
  if (lattice != 19 && lattice != 15) return fail3(LBM_EINVAL, "lattice must be 19 or 15");
  if ((alloc == nullptr) != (free_fn == nullptr)) return fail3(LBM_EINVAL, "alloc and free callbacks go together");
  lbm3_batch *h = new (std::nothrow) lbm3_batch();
  if (!h) return fail3(LBM_ENOMEM, "host allocation failed");
  Batch3 &b = h->b;
  b.max_domains = max_domains;
  b.storage = storage;
  b.q = lattice;
  b.budget = hbm_budget_bytes;
  b.st = static_cast<cudaStream_t>(cuda_stream);
  b.afn = alloc;
  b.ffn = free_fn;
  b.actx = alloc_ctx;
  b.slot.assign(max_domains, nullptr);
  b.target.assign(max_domains, 0);
  b.bytes.assign(max_domains, 0);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&b.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail3(LBM_ECUDA, "no CUDA device");
  }
  const bool k16 = storage == LBM_F16S || storage == LBM_BF16S;
  b.pipe = (k16 && lattice == 15 && sweep3b_fits(lattice, storage, 3) > 0) ? 3 : 0;
  b.grid = std::max(1, sweep3b_fits(lattice, storage, b.pipe)) * b.sms;
  b.d_ctr = static_cast<uint32_t *>(b.get(sizeof(uint32_t) * 2 * groups3(max_domains)));
  if (!b.d_ctr) {
    lbm3_batch_destroy(h);
    return fail3(LBM_ENOMEM, "batch allocation failed");
  }
  if (cudaMemsetAsync(b.d_ctr, 0, sizeof(uint32_t) * 2 * groups3(max_domains), b.st) != cudaSuccess) {
    cudaGetLastError();
    lbm3_batch_destroy(h);
    return fail3(LBM_ECUDA, "batch initialisation failed");
  }
  *out = h;
  return LBM_OK;
}

lbm_status lbm3_batch_admit(lbm3_batch *h, const lbm3_params *p, const lbm3_shape *shapes, int32_t nshapes,
                            const lbm3_body *bodies, int32_t nbodies, int64_t nsteps, int32_t *slot_out) {
  if (!h || !p || !slot_out) return fail3(LBM_EINVAL, "batch, params or slot is NULL");
  Batch3 &b = h->b;
  if (p->storage != b.storage) return fail3(LBM_EINVAL, "storage %d differs from the batch's %d", p->storage, b.storage);
  if (nq_of(*p) != b.q) return fail3(LBM_EINVAL, "lattice D3Q%d differs from the batch's D3Q%d", nq_of(*p), b.q);
  if (p->moving) return fail3(LBM_EINVAL, "a batch holds fixed-geometry domains only");
  if (nsteps < 0) return fail3(LBM_EINVAL, "nsteps must be >= 0");
  int k = -1;
  for (int q = 0; q < b.max_domains && k < 0; ++q)
    if (!b.slot[q]) k = q;
  if (k < 0) return fail3(LBM_EBUSY, "all %d slots are taken", b.max_domains);
  const size_t need = lbm3_domain_bytes(p, nbodies);
  if (need == 0) return fail3(LBM_EINVAL, "invalid domain parameters");
  if (b.budget > 0 && b.bytes_in_use + need > b.budget)
    return fail3(LBM_EBUSY, "memory budget exceeded (%zu + %zu > %zu)", b.bytes_in_use, need, b.budget);
  lbm3_domain *d = nullptr;
  lbm_status rc = lbm3_domain_create(p, shapes, nshapes, bodies, nbodies, b.st, b.afn, b.ffn, b.actx, &d);
  if (rc != LBM_OK) return rc;
  b.slot[k] = d;
  b.target[k] = nsteps;
  b.bytes[k] = need;
  b.bytes_in_use += need;
  *slot_out = k;
  return LBM_OK;
}

static lbm_status batch3_slot(lbm3_batch *h, int32_t k, lbm3_domain **d) {
  if (!h) return fail3(LBM_EINVAL, "batch is NULL");
  if (k < 0 || k >= h->b.max_domains || !h->b.slot[k]) return fail3(LBM_ENOTFOUND, "slot %d is not resident", k);
  *d = h->b.slot[k];
  return LBM_OK;
}

lbm_status lbm3_batch_run(lbm3_batch *h, int64_t max_steps, int64_t *steps_run) {
  if (steps_run) *steps_run = 0;
  if (!h) return fail3(LBM_EINVAL, "batch is NULL");
  if (max_steps < 0) return fail3(LBM_EINVAL, "max_steps must be >= 0");
  Batch3 &b = h->b;
  long long steps = 0;
  for (int k = 0; k < b.max_domains; ++k)
    if (b.slot[k]) steps = std::max(steps, std::min<long long>(max_steps, b.target[k] - b.slot[k]->done));
  if (steps <= 0) return LBM_OK;
  // every domain's force ring must hold the entries of its steps of this chunk
  for (int k = 0; k < b.max_domains; ++k) {
    const lbm3_domain *d = b.slot[k];
    if (!d || d->p.force_every <= 0) continue;
    const long long adv = std::max(0ll, std::min(steps, b.target[k] - d->done));
    if ((d->done + adv) / d->p.force_every - d->drained > d->p.force_capacity)
      return fail3(LBM_EBUSY, "slot %d: force ring would overflow (poll it first)", k);
  }
  // per step: the domains with steps left, in slot order, in groups of kGroup3
  std::vector<int> ks;
  ks.reserve(kGroup3);
  for (long long s = 0; s < steps; ++s) {
    int group = 0;
    ks.clear();
    for (int k = 0; k <= b.max_domains; ++k) {
      if (k < b.max_domains) {
        const lbm3_domain *d = b.slot[k];
        if (!d || d->done + s >= b.target[k]) continue;
        ks.push_back(k);
      }
      if (!ks.empty() && (static_cast<int>(ks.size()) == kGroup3 || k == b.max_domains)) {
        lbm_status rc = batch3_step(b, ks, s, group++);
        if (rc != LBM_OK) return rc;
        ks.clear();
      }
    }
  }
  for (int k = 0; k < b.max_domains; ++k) {
    lbm3_domain *d = b.slot[k];
    if (!d) continue;
    const long long adv = std::max(0ll, std::min(steps, b.target[k] - d->done));
    d->done += adv;
    d->parity = static_cast<int>((d->parity + adv) & 1);
  }
  if (steps_run) *steps_run = steps;
  return LBM_OK;
}

lbm_status lbm3_batch_poll(lbm3_batch *h, int32_t slot, double *out, int64_t max_entries, int64_t *written,
                           int32_t *done) {
  if (written) *written = 0;
  if (done) *done = 0;
  lbm3_domain *d = nullptr;
  lbm_status rc = batch3_slot(h, slot, &d);
  if (rc != LBM_OK) return rc;
  rc = lbm3_forces(d, out, max_entries, written);
  if (done) *done = d->done >= h->b.target[slot] ? 1 : 0;
  return rc;
}

lbm_status lbm3_batch_domain(lbm3_batch *h, int32_t slot, lbm3_domain **out) {
  if (!out) return fail3(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  return batch3_slot(h, slot, out);
}

lbm_status lbm3_batch_evict(lbm3_batch *h, int32_t slot) {
  lbm3_domain *d = nullptr;
  lbm_status rc = batch3_slot(h, slot, &d);
  if (rc != LBM_OK) return rc;
  Batch3 &b = h->b;
  lbm3_domain_destroy(d);  // synchronises the stream: no launch still reads the domain
  b.slot[slot] = nullptr;
  b.bytes_in_use -= b.bytes[slot];
  b.bytes[slot] = 0;
  b.target[slot] = 0;
  return LBM_OK;
}

lbm_status lbm3_batch_set_tile(lbm3_batch *h, int32_t pipeline) {
  if (!h) return fail3(LBM_EINVAL, "batch is NULL");
  if (pipeline != 0 && pipeline != 3 && pipeline != 4) return fail3(LBM_EINVAL, "pipeline must be 0, 3 or 4");
  const int fits = sweep3b_fits(h->b.q, h->b.storage, pipeline);
  if (fits <= 0) return fail3(LBM_EINVAL, "pipeline %d is not available for storage %d", pipeline, h->b.storage);
  h->b.pipe = pipeline;
  h->b.grid = fits * h->b.sms;
  return LBM_OK;
}

lbm_status lbm3_batch_info(lbm3_batch *h, int32_t *resident, int64_t *cells, int64_t *launches, size_t *bytes,
                           int32_t *pipeline) {
  if (!h) return fail3(LBM_EINVAL, "batch is NULL");
  int r = 0;
  long long c = 0;
  for (const lbm3_domain *d : h->b.slot)
    if (d) {
      ++r;
      c += static_cast<long long>(d->p.nx) * d->p.ny * d->p.nz;
    }
  if (resident) *resident = r;
  if (cells) *cells = c;
  if (launches) *launches = h->b.launches;
  if (bytes) *bytes = h->b.bytes_in_use;
  if (pipeline) *pipeline = h->b.pipe;
  return LBM_OK;
}

lbm_status lbm3_batch_destroy(lbm3_batch *h) {
  if (!h) return LBM_OK;
  Batch3 &b = h->b;
  cudaStreamSynchronize(b.st);
  for (lbm3_domain *&d : b.slot)
    if (d) {
      lbm3_domain_destroy(d);
      d = nullptr;
    }
  b.put(b.d_ctr);
  cudaStreamSynchronize(b.st);
  delete h;
  return LBM_OK;
}

}  // extern "C"
