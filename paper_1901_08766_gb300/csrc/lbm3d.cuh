// 3D TRT-LBM-VP with the D3Q19 or the D3Q15 lattice: lattice tables, domain parameters,
// the node update and the fused sweep kernel, shared by the runtime (lbm3d.cu) and the
// translation units that instantiate the sweep per storage (lbm3d_sweep_*.cu). The step
// is the algorithm of Sec. 2.2 with nineteen or fifteen directions (the paper's closing
// remark: D2Q9 is replaced by D3Q15 or D3Q19); storage codecs, stochastic rounding with
// the node mass kept, and the strip/shuffle pull are those of the 2D sweep. Compiled with
// --fmad=false: every FMA is written out.
#pragma once
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
  uint32_t *items;        // [2] the sweep's next strip and finished warps (reset by the last)
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

// Launch shape per storage and register budget (measured on the 384 x 128 x 128 sphere
// channel). Pipeline 0: the 16-bit sweeps run 256-thread blocks, two per SM (16 warps,
// 128 registers), force-free warps in paired FP32; FP32/FP64 128-thread blocks, three per
// SM (12 warps, 168 registers). Pipelines 3 and 4 (16-bit storage only): 320- and
// 384-thread blocks, two per SM (20 or 24 resident warps, at most 102 or 85 registers):
// more warps in flight for fewer registers, as the 2D sweep's budgets. Work distribution:
// the 16-bit sweeps' warps take strips from a device counter (strips with solid nodes
// cost more; 86 against 90 us for D3Q15, 100 against 104 us for D3Q19); the FP32/FP64
// warps take every (grid warps)-th strip, which measured faster for them (157 against
// 164 us for D3Q19 FP32).
template <int S, int P = 0> struct Sweep3Shape {
  static constexpr bool k16 = S == LBM_F16S || S == LBM_BF16S;
  static constexpr bool kDynamic = k16;
  static constexpr int kThreads = P == 3 ? 320 : (P == 4 ? 384 : (k16 ? 256 : 128));
  static constexpr int kMinBlocks = P == 3 || P == 4 ? 2 : (k16 ? 2 : 3);
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

// One strip of 32 V cells of row `row` (= k ny + j) of domain D starting at column x0, at
// step index n: Q vector loads per lane from the lattice D.src, the +-1 x-shift by
// shuffles, strip ends by broadcast loads, the node update, Q vector stores into D.dst.
// With 16-bit storage, warps without solid nodes update two nodes at once in paired FP32
// (the same operations in the same order on each half). `unstable` is set when a node's
// density leaves (0.01, 100) or is not finite.
template <int Q, int S, int V, bool DEF>
__device__ __forceinline__ void sweep3_strip(const Dom3 &D, const int row, const int x0, const long long n,
                                             const int lane, int &unstable) {
  using Cd = Codec<S>;
  using E = typename Cd::E;
  using T = typename Cd::T;
  constexpr bool SHIFT = Cd::kShiftCompute;
  constexpr bool kAddShift = Cd::kShiftCompute && !Cd::kStoreShifted;
  constexpr int kStrip = 32 * V;
  constexpr T kRhoMid = T(50.005) * T(Cd::kScale), kRhoHalf = T(49.995) * T(Cd::kScale);
  constexpr T kUnscale = T(1) / T(Cd::kScale);
  const Const3<T> &C = const3<T>(D);
  const int nx = D.nx, ny = D.ny, pitch = D.pitch;
  const bool west_inlet = D.west == LBM_INLET_EQ, east_out = D.east == LBM_OUTFLOW_ZG;
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

// The fused 3D sweep of one domain: a persistent grid whose warps each update one strip
// (sweep3_strip) at a time.
template <int Q, int S, int V, bool DEF, int P>
__global__ void __launch_bounds__(Sweep3Shape<S, P>::kThreads, Sweep3Shape<S, P>::kMinBlocks)
    sweep3_kernel(const __grid_constant__ Dom3 dom, long long n, int par) {
  constexpr int kStrip = 32 * V;
  const Dom3 &D = dom;  // kernel parameter: constants are read from the parameter bank
  const int lane = threadIdx.x & 31;
  const int strips = (D.nx + kStrip - 1) / kStrip;
  const int items = D.ny * D.nz * strips;  // < 2^31: a direction holds < 2^31 elements
  int unstable = 0;
  // strips from the device counter (the last warp to finish resets it for the next
  // launch), or every (grid warps)-th strip
  constexpr bool kDyn = Sweep3Shape<S, P>::kDynamic;
  const int nw = static_cast<int>((gridDim.x * blockDim.x) >> 5);
  int item = static_cast<int>((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if constexpr (kDyn) {
    if (lane == 0) item = static_cast<int>(atomicAdd(&D.items[0], 1u));
    item = __shfl_sync(0xffffffffu, item, 0);
  }
  while (item < items) {
    int next = item + nw;
    if constexpr (kDyn) {
      if (lane == 0) next = static_cast<int>(atomicAdd(&D.items[0], 1u));
    }
    const int row = item / strips;
    sweep3_strip<Q, S, V, DEF>(D, row, (item - row * strips) * kStrip, n, lane, unstable);
    item = kDyn ? __shfl_sync(0xffffffffu, next, 0) : next;
  }
  if (__any_sync(0xffffffffu, unstable) && lane == 0) atomicOr(D.status, 1);
  if (kDyn && lane == 0) {
    __threadfence();  // this warp's last fetch is ordered before its count
    if (atomicAdd(&D.items[1], 1u) == gridDim.x * (blockDim.x >> 5) - 1u) {
      D.items[0] = 0u;
      D.items[1] = 0u;
    }
  }
}

// ---- batches of 3D domains (lbm3_batch_*) ----------------------------------------------

constexpr int kGroup3 = 16;  // domains per batched launch (their parameters in the kernel's)

// One step of up to kGroup3 domains in one launch. Each domain's parameters (for the
// lattice it reads at this step) and step index travel in the kernel parameter bank, as
// the single-domain sweep's do; domain d owns items base[d] .. base[d + 1] - 1, one strip
// each, rows in order.
struct Batch3Args {
  Dom3 dom[kGroup3];
  long long n[kGroup3];
  int32_t base[kGroup3 + 1];
  uint32_t *ctr;  // [2]: next item, finished warps (reset by the last)
  int32_t ndom;
};

// The batched sweep: warps take strips of every listed domain from one device counter.
// Fixed geometry only (no moving, coupled or pulsating bodies).
template <int Q, int S, int V, int P>
__global__ void __launch_bounds__(Sweep3Shape<S, P>::kThreads, Sweep3Shape<S, P>::kMinBlocks)
    sweep3_batch_kernel(const __grid_constant__ Batch3Args args) {
  constexpr int kStrip = 32 * V;
  const int lane = threadIdx.x & 31;
  const int total = args.base[args.ndom];
  int item = 0;
  if (lane == 0) item = static_cast<int>(atomicAdd(&args.ctr[0], 1u));
  item = __shfl_sync(0xffffffffu, item, 0);
  while (item < total) {
    int next = 0;
    if (lane == 0) next = static_cast<int>(atomicAdd(&args.ctr[0], 1u));
    int d = 0;  // the listed domain owning the item (uniform over the warp)
    while (d + 1 < args.ndom && args.base[d + 1] <= item) ++d;
    const Dom3 &D = args.dom[d];
    const int strips = (D.nx + kStrip - 1) / kStrip;
    const int local = item - args.base[d];
    const int row = local / strips;
    int unstable = 0;
    sweep3_strip<Q, S, V, false>(D, row, (local - row * strips) * kStrip, args.n[d], lane, unstable);
    if (__any_sync(0xffffffffu, unstable) && lane == 0) atomicOr(D.status, 1);
    item = __shfl_sync(0xffffffffu, next, 0);
  }
  if (lane == 0) {
    __threadfence();  // this warp's last fetch is ordered before its count
    if (atomicAdd(&args.ctr[1], 1u) == gridDim.x * (blockDim.x >> 5) - 1u) {
      args.ctr[0] = 0u;
      args.ctr[1] = 0u;
    }
  }
}

// Launch the sweep of one storage (lbm3d_sweep_<storage>.cu): pipeline 0, 3 or 4 (3 and 4
// for 16-bit storage only), grid blocks of Sweep3Shape<S, P>::kThreads threads.
// sweep3_fits gives the resident blocks per SM of that shape (0: not compiled or cannot
// run).
#define LBM3_SWEEP_DECL(NAME)                                                                   \
  cudaError_t launch_sweep3_##NAME(int q, int pipe, bool deform, int grid, cudaStream_t st,     \
                                   const Dom3 &dom, long long n, int par);                      \
  int sweep3_fits_##NAME(int q, int pipe);                                                      \
  cudaError_t launch_sweep3b_##NAME(int q, int pipe, int grid, cudaStream_t st,                 \
                                    const Batch3Args &args);                                    \
  int sweep3b_fits_##NAME(int q, int pipe);
LBM3_SWEEP_DECL(f64)
LBM3_SWEEP_DECL(f32)
LBM3_SWEEP_DECL(f16s)
LBM3_SWEEP_DECL(bf16s)
#undef LBM3_SWEEP_DECL

// The launcher and occupancy query of storage S (instantiated by its translation unit).
template <int S, int P>
cudaError_t launch_sweep3_sp(int q, bool deform, int grid, cudaStream_t st, const Dom3 &dom, long long n, int par) {
  using Sh = Sweep3Shape<S, P>;
  if (q == 15) {
    if (deform) sweep3_kernel<15, S, Sh::kV, true, P><<<grid, Sh::kThreads, 0, st>>>(dom, n, par);
    else sweep3_kernel<15, S, Sh::kV, false, P><<<grid, Sh::kThreads, 0, st>>>(dom, n, par);
  } else {
    if (deform) sweep3_kernel<19, S, Sh::kV, true, P><<<grid, Sh::kThreads, 0, st>>>(dom, n, par);
    else sweep3_kernel<19, S, Sh::kV, false, P><<<grid, Sh::kThreads, 0, st>>>(dom, n, par);
  }
  return cudaGetLastError();
}

template <int S, int P> int sweep3_fits_sp(int q) {
  using Sh = Sweep3Shape<S, P>;
  int nb = 0;
  const cudaError_t e = q == 15
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep3_kernel<15, S, Sh::kV, false, P>, Sh::kThreads, 0)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep3_kernel<19, S, Sh::kV, false, P>, Sh::kThreads, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

// The batched launcher and its occupancy query (blocks per SM) for storage S, pipeline P.
template <int S, int P>
cudaError_t launch_sweep3b_sp(int q, int grid, cudaStream_t st, const Batch3Args &args) {
  using Sh = Sweep3Shape<S, P>;
  if (q == 15) sweep3_batch_kernel<15, S, Sh::kV, P><<<grid, Sh::kThreads, 0, st>>>(args);
  else sweep3_batch_kernel<19, S, Sh::kV, P><<<grid, Sh::kThreads, 0, st>>>(args);
  return cudaGetLastError();
}

template <int S, int P> int sweep3b_fits_sp(int q) {
  using Sh = Sweep3Shape<S, P>;
  int nb = 0;
  const cudaError_t e = q == 15
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep3_batch_kernel<15, S, Sh::kV, P>, Sh::kThreads, 0)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep3_batch_kernel<19, S, Sh::kV, P>, Sh::kThreads, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

}  // namespace d3
}  // namespace lbm

