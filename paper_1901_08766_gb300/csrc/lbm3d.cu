// 3D TRT-LBM-VP with the D3Q19 or the D3Q15 lattice: kernels and the single-domain
// runtime (the C ABI lbm3_* of include/lbm.h). The step is the algorithm of Sec. 2.2 with
// nineteen or fifteen directions (the paper's closing remark: D2Q9 is replaced by D3Q15
// or D3Q19); storage codecs, stochastic rounding with the node mass kept, and the
// strip/shuffle pull are those of the 2D sweep. Compiled with --fmad=false: every FMA is
// written out.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "lbm_sweep.cuh"
#include "lbm_turn.cuh"

namespace lbm {
namespace d3 {

constexpr int kQ3 = 19;  // the larger lattice: array bounds shared by both

// D3Q19: 0 rest; 1..6 +x -x +y -y +z -z; 7..18 +x+y -x-y +x-y -x+y +x+z -x-z +x-z -x+z
// +y+z -y-z +y-z -y+z. D3Q15: 0 rest; 1..6 as D3Q19; 7..14 +x+y+z -x-y-z +x+y-z -x-y+z
// +x-y+z -x+y-z -x+y+z +x-y-z. In both, directions 2m-1 and 2m are opposite; classes by
// index: 0 rest, 1..6 axis, 7.. diagonal (face diagonals of D3Q19, corners of D3Q15).
template <int Q> __host__ __device__ constexpr int ex3(int a) {
  if (Q == 15)
    return (a == 1 || a == 7 || a == 9 || a == 11 || a == 14) ? 1
         : (a == 2 || a == 8 || a == 10 || a == 12 || a == 13) ? -1 : 0;
  return (a == 1 || a == 7 || a == 9 || a == 11 || a == 13) ? 1
       : (a == 2 || a == 8 || a == 10 || a == 12 || a == 14) ? -1 : 0;
}
template <int Q> __host__ __device__ constexpr int ey3(int a) {
  if (Q == 15)
    return (a == 3 || a == 7 || a == 9 || a == 12 || a == 13) ? 1
         : (a == 4 || a == 8 || a == 10 || a == 11 || a == 14) ? -1 : 0;
  return (a == 3 || a == 7 || a == 10 || a == 15 || a == 17) ? 1
       : (a == 4 || a == 8 || a == 9 || a == 16 || a == 18) ? -1 : 0;
}
template <int Q> __host__ __device__ constexpr int ez3(int a) {
  if (Q == 15)
    return (a == 5 || a == 7 || a == 10 || a == 11 || a == 13) ? 1
         : (a == 6 || a == 8 || a == 9 || a == 12 || a == 14) ? -1 : 0;
  return (a == 5 || a == 11 || a == 14 || a == 15 || a == 18) ? 1
       : (a == 6 || a == 12 || a == 13 || a == 16 || a == 17) ? -1 : 0;
}
// specular reflection across a wall normal to y (e_y reversed) or z (e_z reversed)
template <int Q> __host__ __device__ constexpr int reflect_y3(int a) {
  for (int b = 0; b < Q; ++b)
    if (ex3<Q>(b) == ex3<Q>(a) && ey3<Q>(b) == -ey3<Q>(a) && ez3<Q>(b) == ez3<Q>(a)) return b;
  return a;
}
template <int Q> __host__ __device__ constexpr int reflect_z3(int a) {
  for (int b = 0; b < Q; ++b)
    if (ex3<Q>(b) == ex3<Q>(a) && ey3<Q>(b) == ey3<Q>(a) && ez3<Q>(b) == -ez3<Q>(a)) return b;
  return a;
}
// lattice weights per class: rest, axis, diagonal
template <int Q> constexpr double w3(int cls) {
  return Q == 15 ? (cls == 0 ? 2.0 / 9.0 : cls == 1 ? 1.0 / 9.0 : 1.0 / 72.0)
                 : (cls == 0 ? 1.0 / 3.0 : cls == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Per-domain constants in compute precision (per class: rest, axis, diagonal).
template <typename T> struct Const3 {
  T one_m_omp, hp, hm, inv_2eta1, rho0;
  T pw0, pw1, pw2, mw1, mw2, kw0, kw1, kw2, qw1, qw2, wr0, wr1, wr2;
  T ghost[kQ3];  // inlet populations in compute space, as a stored node holds them
};

// force-free constants duplicated for paired FP32 (both halves of a node pair)
struct Pair3 {
  float2 one_m_omp, hp, hm, rho0, pw0, pw1, pw2, mw1, mw2;
};

constexpr int kMaxMoving3 = 8;  // bodies of a moving 3D domain

struct Dom3 {
  void *lat[2];
  uint8_t *mask;
  void *fvp;              // [cells][3] F_VP of solid nodes (compute precision)
  double *bodies;         // [nbodies][9]: c, v, w
  float *bodies_f;
  double *ring;           // [cap][nbodies][3]
  double *rowsum;         // [nfrows][nbodies][3]
  const int4 *frows;      // rows holding solid nodes, ascending: (k * ny + j, first, last + 1, 0)
  int32_t *status;
  uint32_t *rows_done;    // blocks of the force reduction that finished (reset by the last)
  int32_t nx, ny, nz, pitch, nfrows;
  int32_t west, east, south, north, bottom, top;
  int32_t nbodies, force_every, force_cap;
  Const3<float> cf;
  Const3<double> cd;
  Pair3 pc;
  // moving domains (prescribed translation; zero / null otherwise)
  int32_t moving, nshapes;
  const struct Shape3Dev *shapes;  // reference geometry (step index 0)
  const double *centre0;           // [nbodies][3] reference centres
  float mbox[8][3];                // per body: half extents of the box its shapes reach
                                   // about its centre (< 0: the whole axis)
  double *mpart;                   // [8][kMaxMoveBlocks3][3] partial force sums
  uint32_t *mcount;                // [8] blocks of the moving force reduction finished
  // coupled bodies (null / zero otherwise): state [2][8][9] by step parity (x, v and the
  // previous step's force), parameters [8][12] (M, k[3], c[3], free[3]); bit b of
  // `coupled`: body b + 1 has dynamics
  double *fsi;
  const double *fsi_par;
  uint32_t coupled;
  // pulsating bodies (null / zero otherwise): [8][2] amplitude a and rate nu of
  // s(n) = 1 + a sin(nu n); the dilation rate kappa = s'/s of the current step [8] in FP64
  // and FP32 (zero for rigid bodies); bit b of `deform`: body b + 1 pulsates
  const double *dpar;
  double *kappa;
  float *kappa_f;
  uint32_t deform;
  // per-launch: base of each direction's array in the lattice read (src) and written (dst)
  const void *src[kQ3];
  void *dst[kQ3];
};

template <typename T> __device__ __forceinline__ const Const3<T> &const3(const Dom3 &d);
template <> __device__ __forceinline__ const Const3<float> &const3<float>(const Dom3 &d) { return d.cf; }
template <> __device__ __forceinline__ const Const3<double> &const3<double>(const Dom3 &d) { return d.cd; }

template <typename T> __device__ __forceinline__ T shift3(const Const3<T> &c, int a) {
  return a == 0 ? c.wr0 : (a < 7 ? c.wr1 : c.wr2);
}

// U_O = V + omega x (x - c) of body b at node (i, j, k), explicitly rounded in FP64; with
// DEF (some body pulsates) plus kappa (x - c), kappa zero for rigid bodies (the sweep is
// instantiated without the term unless a body of the domain pulsates)
template <bool DEF>
__device__ __forceinline__ void body_velocity3(const Dom3 &D, int b, int i, int j, int k, double (&uo)[3]) {
  const double *q = D.bodies + 9 * (b - 1);
  const double r0 = __dsub_rn(double(i), q[0]), r1 = __dsub_rn(double(j), q[1]), r2 = __dsub_rn(double(k), q[2]);
  uo[0] = __dadd_rn(q[3], __dsub_rn(__dmul_rn(q[7], r2), __dmul_rn(q[8], r1)));
  uo[1] = __dadd_rn(q[4], __dsub_rn(__dmul_rn(q[8], r0), __dmul_rn(q[6], r2)));
  uo[2] = __dadd_rn(q[5], __dsub_rn(__dmul_rn(q[6], r1), __dmul_rn(q[7], r0)));
  if constexpr (DEF) {
    const double kp = D.kappa[b - 1];
    uo[0] = __dadd_rn(uo[0], __dmul_rn(kp, r0));
    uo[1] = __dadd_rn(uo[1], __dmul_rn(kp, r1));
    uo[2] = __dadd_rn(uo[2], __dmul_rn(kp, r2));
  }
}
template <bool DEF>
__device__ __forceinline__ void body_velocity3(const Dom3 &D, int b, int i, int j, int k, float (&uo)[3]) {
  const float *q = D.bodies_f + 9 * (b - 1);
  const float r0 = float(i) - q[0], r1 = float(j) - q[1], r2 = float(k) - q[2];
  uo[0] = q[3] + (q[7] * r2 - q[8] * r1);
  uo[1] = q[4] + (q[8] * r0 - q[6] * r2);
  uo[2] = q[5] + (q[6] * r1 - q[7] * r0);
  if constexpr (DEF) {
    const float kp = D.kappa_f[b - 1];
    uo[0] += kp * r0;
    uo[1] += kp * r1;
    uo[2] += kp * r2;
  }
}

template <typename T> struct Macro3 {
  T d, rho, u[3], f[3];
};

// steps (3)-(5) at one node: Eq. (rho), Eq. (rho*velocity-star), penalization (Eq. d-V,
// Eq. force-density) and Eq. (velocity-r), in a fixed order of operations
template <int Q, typename T, bool SHIFT, bool FORCE>
__device__ __forceinline__ Macro3<T> macro3(const T (&x)[Q], const Const3<T> &c, bool solid,
                                            const T (&uo)[3]) {
  Macro3<T> m;
  T dm[10], sp[10];
#pragma unroll
  for (int p = 1; p <= (Q - 1) / 2; ++p) {
    dm[p] = x[2 * p - 1] - x[2 * p];
    sp[p] = x[2 * p - 1] + x[2 * p];
  }
  T jx, jy, jz;
  if constexpr (Q == 19) {
    m.d = (x[0] + ((sp[1] + sp[2]) + sp[3])) + (((sp[4] + sp[5]) + (sp[6] + sp[7])) + (sp[8] + sp[9]));
    jx = (dm[1] + dm[4]) + (dm[5] + (dm[6] + dm[7]));
    jy = (dm[2] + dm[4]) + ((dm[8] + dm[9]) - dm[5]);
    jz = (dm[3] + dm[6]) + ((dm[8] - dm[9]) - dm[7]);
  } else {
    m.d = (x[0] + ((sp[1] + sp[2]) + sp[3])) + ((sp[4] + sp[5]) + (sp[6] + sp[7]));
    jx = (dm[1] + dm[4]) + ((dm[5] + dm[6]) - dm[7]);
    jy = (dm[2] + dm[4]) + ((dm[5] - dm[6]) + dm[7]);
    jz = (dm[3] + dm[4]) + ((dm[6] - dm[5]) + dm[7]);
  }
  m.rho = SHIFT ? c.rho0 + m.d : m.d;
  const T inv = rcp_(m.rho);
  m.u[0] = jx * inv;
  m.u[1] = jy * inv;
  m.u[2] = jz * inv;
  m.f[0] = m.f[1] = m.f[2] = T(0);
  if (FORCE && solid) {
    const T two_rho = m.rho + m.rho;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const T du = (uo[e] - m.u[e]) * c.inv_2eta1;
      m.f[e] = two_rho * du;
      m.u[e] = m.u[e] + du;
    }
  }
  return m;
}

// TRT collision with the split Guo term per opposite pair (the 2D form; nine pairs for
// D3Q19, seven for D3Q15)
template <int Q, typename T, bool SHIFT, bool FORCE>
__device__ __forceinline__ void collide3(T (&x)[Q], const Macro3<T> &m, const Const3<T> &c) {
  const T base = SHIFT ? m.d : m.rho;
  const T ux = m.u[0], uy = m.u[1], uz = m.u[2];
  const T q = T(1.5) * fma_(uz, uz, fma_(uy, uy, ux * ux));
  const T a0 = c.pw0 * m.rho, b0 = c.pw0 * base;
  const T a1 = c.pw1 * m.rho, b1 = c.pw1 * base;
  const T a2 = c.pw2 * m.rho, b2 = c.pw2 * base;
  const T m1 = c.mw1 * m.rho, m2 = c.mw2 * m.rho;
  T uf = T(0);
  if (FORCE) uf = fma_(uz, m.f[2], fma_(uy, m.f[1], ux * m.f[0]));
  {
    T g0 = fma_(c.one_m_omp, x[0], fma_(-a0, q, b0));
    if (FORCE) g0 = fma_(T(-3) * c.kw0, uf, g0);
    x[0] = g0;
  }
  auto pair = [&](int ia, int ib, T eu, T ef, T a, T b, T mm, T kw, T qw) {
    const T xs = x[ia] + x[ib];
    const T xd = x[ia] - x[ib];
    const T c1 = fma_(T(4.5) * eu, eu, -q);
    const T eqs = fma_(a, c1, b);
    T S = fma_(-c.hp, xs, eqs);
    T A = fma_(-c.hm, xd, mm * eu);
    if (FORCE) {
      S = fma_(kw, fma_(T(9) * eu, ef, T(-3) * uf), S);
      A = fma_(qw, ef, A);
    }
    x[ia] = (x[ia] + S) + A;
    x[ib] = (x[ib] + S) - A;
  };
  const T fx = m.f[0], fy = m.f[1], fz = m.f[2];
  pair(1, 2, ux, fx, a1, b1, m1, c.kw1, c.qw1);
  pair(3, 4, uy, fy, a1, b1, m1, c.kw1, c.qw1);
  pair(5, 6, uz, fz, a1, b1, m1, c.kw1, c.qw1);
  if constexpr (Q == 19) {
    pair(7, 8, ux + uy, fx + fy, a2, b2, m2, c.kw2, c.qw2);
    pair(9, 10, ux - uy, fx - fy, a2, b2, m2, c.kw2, c.qw2);
    pair(11, 12, ux + uz, fx + fz, a2, b2, m2, c.kw2, c.qw2);
    pair(13, 14, ux - uz, fx - fz, a2, b2, m2, c.kw2, c.qw2);
    pair(15, 16, uy + uz, fy + fz, a2, b2, m2, c.kw2, c.qw2);
    pair(17, 18, uy - uz, fy - fz, a2, b2, m2, c.kw2, c.qw2);
  } else {
    pair(7, 8, (ux + uy) + uz, (fx + fy) + fz, a2, b2, m2, c.kw2, c.qw2);
    pair(9, 10, (ux + uy) - uz, (fx + fy) - fz, a2, b2, m2, c.kw2, c.qw2);
    pair(11, 12, (ux - uy) + uz, (fx - fy) + fz, a2, b2, m2, c.kw2, c.qw2);
    pair(13, 14, (uy + uz) - ux, (fy + fz) - fx, a2, b2, m2, c.kw2, c.qw2);
  }
}

// 16-bit words of two nodes' values with stochastic rounding and the node mass kept
// (the 2D rule: moving values rounded first, the rest value stored as the pulled mass
// minus their rounded sum, pairs summed in a fixed order)
template <int Q, int S>
__device__ __forceinline__ void encode3_pair(const F2 (&x)[Q], F2 d, uint32_t bits, uint32_t (&w)[Q]) {
  F2 sp[10];
#pragma unroll
  for (int p = 1; p <= (Q - 1) / 2; ++p) {
    w[2 * p - 1] = Codec<S>::enc2_sr(x[2 * p - 1].v.x, x[2 * p - 1].v.y, bits);
    w[2 * p] = Codec<S>::enc2_sr(x[2 * p].v.x, x[2 * p].v.y, bits);
    sp[p] = F2(Codec<S>::dec2(w[2 * p - 1])) + F2(Codec<S>::dec2(w[2 * p]));
  }
  F2 diag = (sp[4] + sp[5]) + (sp[6] + sp[7]);
  if constexpr (Q == 19) diag = diag + (sp[8] + sp[9]);
  const F2 moved = ((sp[1] + sp[2]) + sp[3]) + diag;
  const F2 rest = d - moved;
  w[0] = Codec<S>::enc2_sr(rest.v.x, rest.v.y, bits);
}

// constants of the force-free update broadcast to both halves of a node pair
__device__ __forceinline__ Const3<F2> pair_const3(const Pair3 &c) {
  Const3<F2> p;
  p.one_m_omp = F2(c.one_m_omp);
  p.hp = F2(c.hp);
  p.hm = F2(c.hm);
  p.rho0 = F2(c.rho0);
  p.pw0 = F2(c.pw0);
  p.pw1 = F2(c.pw1);
  p.pw2 = F2(c.pw2);
  p.mw1 = F2(c.mw1);
  p.mw2 = F2(c.mw2);
  return p;
}

// source row of direction a for row (j, k): y rule, then z rule
template <int Q>
__device__ __forceinline__ void src_row3(const Dom3 &D, int a, int j, int k, int &sa, int &sy, int &sz) {
  sa = a;
  sy = j - ey3<Q>(a);
  sz = k - ez3<Q>(a);
  if (sy < 0) {
    if (D.south == LBM_FREE_SLIP) { sy = 0; sa = reflect_y3<Q>(sa); }
    else sy += D.ny;
  } else if (sy > D.ny - 1) {
    if (D.north == LBM_FREE_SLIP) { sy = D.ny - 1; sa = reflect_y3<Q>(sa); }
    else sy -= D.ny;
  }
  if (sz < 0) {
    if (D.bottom == LBM_FREE_SLIP) { sz = 0; sa = reflect_z3<Q>(sa); }
    else sz += D.nz;
  } else if (sz > D.nz - 1) {
    if (D.top == LBM_FREE_SLIP) { sz = D.nz - 1; sa = reflect_z3<Q>(sa); }
    else sz -= D.nz;
  }
}

#ifndef LBM3_THREADS16
#define LBM3_THREADS16 256
#endif
#ifndef LBM3_MINB16
#define LBM3_MINB16 2
#endif
#ifndef LBM3_THREADS32
#define LBM3_THREADS32 128
#endif
#ifndef LBM3_MINB32
#define LBM3_MINB32 3
#endif

// Launch shape per storage (measured on the 384 x 128 x 128 sphere channel): the 16-bit
// sweeps run 256-thread blocks, two per SM (128 registers), force-free warps in paired
// FP32; FP32/FP64 128-thread blocks, three per SM (168 registers).
template <int S> struct Sweep3Shape {
  static constexpr bool k16 = S == LBM_F16S || S == LBM_BF16S;
  static constexpr int kThreads = k16 ? LBM3_THREADS16 : LBM3_THREADS32;
  static constexpr int kMinBlocks = k16 ? LBM3_MINB16 : LBM3_MINB32;
  static constexpr bool kPaired = k16;
  static constexpr int kV = S == LBM_F64 ? 2 : 4;
};

// Source rows of the pull for row (j, k): element offsets within one direction's array of
// the rows j - e_y (index e_y + 1) and planes k - e_z (index e_z + 1), with the free-slip
// flags (the source direction is then mirrored). Fits 32 bits: a direction holds < 2^31
// elements.
struct RowOff3 {
  uint32_t y[3], z[3];
  bool my[3], mz[3];
};

__device__ __forceinline__ RowOff3 row_off3(const Dom3 &D, int j, int k) {
  RowOff3 r;
  const uint32_t pitch = static_cast<uint32_t>(D.pitch), plane = pitch * static_cast<uint32_t>(D.ny);
  r.my[0] = r.my[1] = r.my[2] = false;
  r.mz[0] = r.mz[1] = r.mz[2] = false;
  int sy = j - 1;  // e_y = +1
  if (sy < 0) {
    r.my[2] = D.south == LBM_FREE_SLIP;
    sy = r.my[2] ? 0 : D.ny - 1;
  }
  r.y[2] = static_cast<uint32_t>(sy) * pitch;
  r.y[1] = static_cast<uint32_t>(j) * pitch;
  sy = j + 1;  // e_y = -1
  if (sy > D.ny - 1) {
    r.my[0] = D.north == LBM_FREE_SLIP;
    sy = r.my[0] ? D.ny - 1 : 0;
  }
  r.y[0] = static_cast<uint32_t>(sy) * pitch;
  int sz = k - 1;  // e_z = +1
  if (sz < 0) {
    r.mz[2] = D.bottom == LBM_FREE_SLIP;
    sz = r.mz[2] ? 0 : D.nz - 1;
  }
  r.z[2] = static_cast<uint32_t>(sz) * plane;
  r.z[1] = static_cast<uint32_t>(k) * plane;
  sz = k + 1;  // e_z = -1
  if (sz > D.nz - 1) {
    r.mz[0] = D.top == LBM_FREE_SLIP;
    sz = r.mz[0] ? D.nz - 1 : 0;
  }
  r.z[0] = static_cast<uint32_t>(sz) * plane;
  return r;
}

// source row of direction a (A a compile-time constant after unrolling)
template <int Q, typename E, int A>
__device__ __forceinline__ const E *src_row_ptr(const Dom3 &D, const RowOff3 &r) {
  constexpr int iy = ey3<Q>(A) + 1, iz = ez3<Q>(A) + 1;
  constexpr int ay = reflect_y3<Q>(A), az = reflect_z3<Q>(A), ayz = reflect_z3<Q>(reflect_y3<Q>(A));
  const bool my = r.my[iy], mz = r.mz[iz];
  const void *base = my ? (mz ? D.src[ayz] : D.src[ay]) : (mz ? D.src[az] : D.src[A]);
  return static_cast<const E *>(base) + (r.z[iz] + r.y[iy]);
}

template <int Q, int A, typename F> __device__ __forceinline__ void for_dirs(F &&f) {
  if constexpr (A < Q) {
    f(std::integral_constant<int, A>{});
    for_dirs<Q, A + 1>(f);
  }
}

// The fused 3D sweep: one warp per strip of 32 V cells of one row (j, k) at a time
// (persistent grid), Q vector loads per lane, the +-1 x-shift by shuffles, strip ends by
// broadcast loads, update, Q vector stores into the other lattice. With 16-bit storage,
// warps without solid nodes update two nodes at once in paired FP32 (the same operations
// in the same order on each half).
template <int Q, int S, int V, bool DEF>
__global__ void __launch_bounds__(Sweep3Shape<S>::kThreads, Sweep3Shape<S>::kMinBlocks)
    sweep3_kernel(const __grid_constant__ Dom3 dom, long long n, int par) {
  using Cd = Codec<S>;
  using E = typename Cd::E;
  using T = typename Cd::T;
  constexpr bool SHIFT = Cd::kShiftCompute;
  constexpr bool kAddShift = Cd::kShiftCompute && !Cd::kStoreShifted;
  constexpr int kStrip = 32 * V;
  constexpr T kRhoMid = T(50.005) * T(Cd::kScale), kRhoHalf = T(49.995) * T(Cd::kScale);
  constexpr T kUnscale = T(1) / T(Cd::kScale);
  const Dom3 &D = dom;  // kernel parameter: constants are read from the parameter bank
  const Const3<T> &C = const3<T>(D);
  const int lane = threadIdx.x & 31;
  const int nx = D.nx, ny = D.ny, nz = D.nz, pitch = D.pitch;
  const int strips = (nx + kStrip - 1) / kStrip;
  const long long items = static_cast<long long>(ny) * nz * strips;
  const long long wg = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const long long nw = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
  const bool west_inlet = D.west == LBM_INLET_EQ, east_out = D.east == LBM_OUTFLOW_ZG;
  int unstable = 0;
  for (long long it = wg; it < items; it += nw) {
    const int row = static_cast<int>(it / strips);
    const int x0 = static_cast<int>(it % strips) * kStrip;
    const int j = row % ny, k = row / ny;
    const int xl = x0 + lane * V;
    const bool lane_on = xl < nx;
    const bool west_edge = x0 == 0, east_edge = x0 + kStrip >= nx;
    const int col_l = west_edge ? (west_inlet ? 0 : nx - 1) : x0 - 1;
    const int col_r = east_edge ? 0 : x0 + kStrip;
    const int k_last = nx - 1 - xl;
    const int xl_ld = min(xl, pitch - V);
    Strip<S, V> v[Q];
    E end_in[Q];
    {
      const RowOff3 R = row_off3(D, j, k);
      for_dirs<Q, 0>([&](auto ac) {
        constexpr int a = decltype(ac)::value;
        const E *rp = src_row_ptr<Q, E, a>(D, R);
        v[a].load(rp + xl_ld);
        end_in[a] = E(0);
        if constexpr (ex3<Q>(a) == 1) end_in[a] = __ldg(rp + col_l);
        else if constexpr (ex3<Q>(a) == -1) end_in[a] = __ldg(rp + col_r);
      });
    }
    uint8_t b[V];
    {
      const uint8_t *mrow = D.mask + (static_cast<size_t>(k) * ny + j) * pitch + xl_ld;
#pragma unroll
      for (int q = 0; q < V; ++q) b[q] = lane_on ? __ldg(mrow + q) : uint8_t(0);
    }
    // the +-1 x-shift of the pull
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      const int ex = ex3<Q>(a);
      if (ex == 1) {
        E in = shfl_up1<E>(v[a].last());
        in = lane == 0 ? end_in[a] : in;
        v[a].shift_up(in);
      } else if (ex == -1) {
        E keep = E(0);
        if (east_edge) {
#pragma unroll
          for (int q = 0; q < V; ++q) keep = (q == k_last) ? v[a].get(q) : keep;
        }
        E in = shfl_down1<E>(v[a].first());
        in = (lane == 31 && !east_edge) ? end_in[a] : in;
        v[a].shift_down(in);
        if (east_edge) {
          const E fix = east_out ? keep : end_in[a];
#pragma unroll
          for (int q = 0; q < V; ++q)
            if (q == k_last) v[a].set(q, fix);
        }
      }
    }
    bool any_lane = false;
#pragma unroll
    for (int q = 0; q < V; ++q) any_lane |= b[q] != 0;
    const bool any_solid = __any_sync(0xffffffffu, any_lane);
    const unsigned valid_bits =
        east_edge ? (nx - xl >= V ? (1u << V) - 1u : (nx > xl ? (1u << (nx - xl)) - 1u : 0u)) : (1u << V) - 1u;
    unsigned bad_bits = 0u;
    auto update = [&](T (&x)[Q], int q) -> T {
      if (q == 0 && west_edge && west_inlet && lane == 0) {
#pragma unroll
        for (int a = 1; a < Q; ++a)
          if (ex3<Q>(a) == 1) x[a] = C.ghost[a];
      }
      Macro3<T> m;
      if (any_solid) {
        T uo[3] = {T(0), T(0), T(0)};
        const bool solid = b[q] != 0;
        if (solid) body_velocity3<DEF>(D, b[q], xl + q, j, k, uo);
        m = macro3<Q, T, SHIFT, true>(x, C, solid, uo);
        collide3<Q, T, SHIFT, true>(x, m, C);
        if (solid) {
          T *fv = static_cast<T *>(D.fvp) + 3 * ((static_cast<size_t>(k) * ny + j) * pitch + xl + q);
          fv[0] = m.f[0] * kUnscale;
          fv[1] = m.f[1] * kUnscale;
          fv[2] = m.f[2] * kUnscale;
        }
      } else {
        const T uo[3] = {T(0), T(0), T(0)};
        m = macro3<Q, T, SHIFT, false>(x, C, false, uo);
        collide3<Q, T, SHIFT, false>(x, m, C);
      }
      bad_bits |= (fabs(m.rho - kRhoMid) < kRhoHalf ? 0u : 1u) << q;
      return m.d;
    };
    if constexpr (sizeof(E) == 2) {
      const uint32_t sr_g = sr_group_bits(sr_row_key(n, row), xl);
      if (Sweep3Shape<S>::kPaired && !any_solid) {
        const Const3<F2> CP = pair_const3(D.pc);
#pragma unroll
        for (int q = 0; q < V; q += 2) {
          F2 x[Q];
#pragma unroll
          for (int a = 0; a < Q; ++a) x[a] = F2(Cd::dec2(v[a].w[q >> 1]));
          if (q == 0 && west_edge && west_inlet) {
            const bool g = lane == 0;
#pragma unroll
            for (int a = 1; a < Q; ++a)
              if (ex3<Q>(a) == 1) x[a].v.x = g ? C.ghost[a] : x[a].v.x;
          }
          const F2 uo[3] = {F2(0.f), F2(0.f), F2(0.f)};
          const Macro3<F2> m = macro3<Q, F2, SHIFT, false>(x, CP, false, uo);
          collide3<Q, F2, SHIFT, false>(x, m, CP);
          bad_bits |= (fabsf(m.rho.v.x - kRhoMid) < kRhoHalf ? 0u : 1u) << q;
          bad_bits |= (fabsf(m.rho.v.y - kRhoMid) < kRhoHalf ? 0u : 1u) << (q + 1);
          uint32_t w[Q];
          encode3_pair<Q, S>(x, m.d, sr_pair_bits(sr_g, xl + q), w);
#pragma unroll
          for (int a = 0; a < Q; ++a) v[a].w[q >> 1] = w[a];
        }
      } else {
#pragma unroll
        for (int q = 0; q < V; q += 2) {
          T x0v[Q], x1v[Q];
#pragma unroll
          for (int a = 0; a < Q; ++a) {
            const float2 p = Cd::dec2(v[a].w[q >> 1]);
            x0v[a] = p.x;
            x1v[a] = p.y;
          }
          const float d0 = update(x0v, q);
          const float d1 = update(x1v, q + 1);
          F2 x[Q];
#pragma unroll
          for (int a = 0; a < Q; ++a) x[a] = F2(make_float2(x0v[a], x1v[a]));
          uint32_t w[Q];
          encode3_pair<Q, S>(x, F2(make_float2(d0, d1)), sr_pair_bits(sr_g, xl + q), w);
#pragma unroll
          for (int a = 0; a < Q; ++a) v[a].w[q >> 1] = w[a];
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < V; ++q) {
        T x[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) x[a] = Cd::dec(v[a].get(q));
        if constexpr (kAddShift) {
#pragma unroll
          for (int a = 0; a < Q; ++a) x[a] -= shift3(C, a);  // exact (Sterbenz)
        }
        update(x, q);
        if constexpr (kAddShift) {
#pragma unroll
          for (int a = 0; a < Q; ++a) x[a] += shift3(C, a);
        }
#pragma unroll
        for (int a = 0; a < Q; ++a) v[a].set(q, Cd::enc(x[a]));
      }
    }
    if (bad_bits & valid_bits) unstable = 1;
    if (east_edge) {
#pragma unroll
      for (int q = 0; q < V; ++q)
        if (!((valid_bits >> q) & 1u)) {
#pragma unroll
          for (int a = 0; a < Q; ++a) v[a].set(q, E(0));
        }
    }
    if (lane_on) {
      const uint32_t off = (static_cast<uint32_t>(k) * ny + j) * static_cast<uint32_t>(pitch) + xl;
#pragma unroll
      for (int a = 0; a < Q; ++a) v[a].store(static_cast<E *>(D.dst[a]) + off);
    }
  }
  if (__any_sync(0xffffffffu, unstable) && lane == 0) atomicOr(D.status, 1);
}

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

template <typename T>
__global__ void __launch_bounds__(kRowsThreads) rows3_kernel(const __grid_constant__ Dom3 dom, long long entry) {
  const Dom3 &D = dom;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
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
  if (threadIdx.x == 0) last = atomicAdd(D.rows_done, 1u) == gridDim.x - 1;
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
  int grid = 0;      // sweep blocks
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

template <int Q, int S> cudaError_t launch_sweep3_as(lbm3_domain *d, long long n, int par) {
  using Sh = Sweep3Shape<S>;
  if (d->h.deform) sweep3_kernel<Q, S, Sh::kV, true><<<d->grid, Sh::kThreads, 0, d->st>>>(d->hpar[par], n, par);
  else sweep3_kernel<Q, S, Sh::kV, false><<<d->grid, Sh::kThreads, 0, d->st>>>(d->hpar[par], n, par);
  return cudaGetLastError();
}

template <int Q> cudaError_t launch_sweep3_q(lbm3_domain *d, long long n, int par) {
  switch (d->p.storage) {
    case LBM_F64: return launch_sweep3_as<Q, LBM_F64>(d, n, par);
    case LBM_F32: return launch_sweep3_as<Q, LBM_F32>(d, n, par);
    case LBM_F16S: return launch_sweep3_as<Q, LBM_F16S>(d, n, par);
    case LBM_BF16S: return launch_sweep3_as<Q, LBM_BF16S>(d, n, par);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sweep3(lbm3_domain *d, long long n, int par) {
  return nq_of(d->p) == 15 ? launch_sweep3_q<15>(d, n, par) : launch_sweep3_q<19>(d, n, par);
}

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

template <int Q, int S> int sweep3_blocks_as(int sms) {
  using Sh = Sweep3Shape<S>;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep3_kernel<Q, S, Sh::kV, false>, Sh::kThreads, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    n = 1;
  }
  return sms * std::max(1, n);
}

template <int Q> int sweep3_blocks_q(int storage, int sms) {
  switch (storage) {
    case LBM_F64: return sweep3_blocks_as<Q, LBM_F64>(sms);
    case LBM_F32: return sweep3_blocks_as<Q, LBM_F32>(sms);
    case LBM_F16S: return sweep3_blocks_as<Q, LBM_F16S>(sms);
    case LBM_BF16S: return sweep3_blocks_as<Q, LBM_BF16S>(sms);
  }
  return sms;
}

// persistent grid of the sweep: every resident block slot of every SM
int sweep3_blocks(int q, int storage, int sms) {
  return q == 15 ? sweep3_blocks_q<15>(storage, sms) : sweep3_blocks_q<19>(storage, sms);
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

}  // namespace

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
  ADM3(cudaMemsetAsync(D.status, 0, 8, st));  // status and the reduction's block counter
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
  d->grid = sweep3_blocks(nq, p->storage, sms);
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

}  // extern "C"
