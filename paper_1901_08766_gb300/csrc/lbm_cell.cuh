// Device-side building blocks of the TRT-LBM-VP step: storage codecs, the per-node
// update (moments, penalization, TRT collision with split Guo forcing) and the scalar
// pull with the domain-edge rules. The translation units are compiled with
// --fmad=false: every fused multiply-add below is written out with fma(), so each
// instantiation of the update performs the same roundings and results do not depend
// on the tile shape or on which kernel evaluates a node.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_internal.h"

namespace lbm {

// D2Q9 velocity set, Eq. (D2Q9): alpha = 0 rest, 1..4 axes at (alpha-1) pi/2, 5..8
// diagonals at (2 alpha-9) pi/4; ex_of/ey_of give the components.

// Reflection of a direction across a horizontal wall (e_y -> -e_y): free-slip edges.
__host__ __device__ constexpr int reflect_y(int a) {
  return a == 2 ? 4 : a == 4 ? 2 : a == 5 ? 8 : a == 8 ? 5 : a == 6 ? 7 : a == 7 ? 6 : a;
}
__host__ __device__ constexpr int ex_of(int a) {
  return (a == 1 || a == 5 || a == 8) ? 1 : (a == 3 || a == 6 || a == 7) ? -1 : 0;
}
__host__ __device__ constexpr int ey_of(int a) {
  return (a == 2 || a == 5 || a == 6) ? 1 : (a == 4 || a == 7 || a == 8) ? -1 : 0;
}

// ---- storage codecs --------------------------------------------------------------------
// F64 / F32 store f (F32 rounded to nearest even); F16S stores kF16Scale (f - w_alpha
// rho0), BF16S f - w_alpha rho0, both rounded stochastically (see PairEncoder).
// kStoreShifted: the stored value is the shifted f - w_alpha rho0. kShiftCompute: the
// node update works on f - w_alpha rho0 (for F32 storage the shift is subtracted after
// loading, exactly, and added back before storing), so that no O(1) population meets a
// rounded relaxation constant: that would bias mass by about one FP32 unit per node and
// step. kScale: the power of two the compute space carries (the update works on the
// stored values as they are; the domain's rho0 in compute precision carries the scale, so
// rho, the equilibrium amplitudes and the Guo terms come out scaled and u = j / rho does
// not). FP16's normal range then starts at 2^-14 / kF16Scale = 6e-8 instead of 6e-5:
// the small deviations of slow flows keep full relative precision and round exactly.

template <int S> struct Codec;

template <> struct Codec<LBM_F64> {
  using E = double;
  using T = double;
  static constexpr bool kStoreShifted = false;
  static constexpr bool kShiftCompute = false;
  static constexpr float kScale = 1.0f;
  __device__ static T dec(E e) { return e; }
  __device__ static E enc(T t) { return t; }
};
template <> struct Codec<LBM_F32> {
  using E = float;
  using T = float;
  static constexpr bool kStoreShifted = false;
  static constexpr bool kShiftCompute = true;
  static constexpr float kScale = 1.0f;
  __device__ static T dec(E e) { return e; }
  __device__ static E enc(T t) { return t; }
};
template <> struct Codec<LBM_F16S> {
  using E = uint16_t;
  using T = float;
  static constexpr bool kStoreShifted = true;
  static constexpr bool kShiftCompute = true;
  static constexpr float kScale = kF16Scale;
  __device__ static T dec(E e) { return __half2float(__ushort_as_half(e)); }
  __device__ static E enc(T t) { return __half_as_ushort(__float2half_rn(t)); }
  // two packed elements (low = first)
  __device__ static float2 dec2(uint32_t w) {
    return __half22float2(*reinterpret_cast<const __half2 *>(&w));
  }
  __device__ static uint32_t enc2(float lo, float hi) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
  }
  // Stochastic rounding: each element rounds away from zero with probability equal to
  // its distance from the truncated value in units of the last place. 13 random bits are
  // added below the FP16 mantissa of the FP32 magnitude (lower element bits 12..0, upper
  // element bits 31..19), then the value is truncated. Exact wherever the FP16 result is
  // normal (exactly 13 bits are dropped), i.e. for stored values of magnitude >= 2^-14,
  // shifted populations >= 6e-8 with the storage scale; below that fewer than the dropped
  // bits are randomized, a bias toward zero of less than one FP16 subnormal unit
  // (2^-24 / 1024 = 6e-11 in population units). (The sm_100 family's cvt.rs conversion
  // is exact everywhere but needs more registers in this kernel.)
  __device__ static uint32_t enc2_sr(float lo, float hi, uint32_t rbits) {
    const float l = __uint_as_float(__float_as_uint(lo) + (rbits & 0x1fffu));
    const float h = __uint_as_float(__float_as_uint(hi) + (rbits >> 19));
    uint32_t d;
    asm("cvt.rz.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(h), "f"(l));
    return d;
  }
};
template <> struct Codec<LBM_BF16S> {
  using E = uint16_t;
  using T = float;
  static constexpr bool kStoreShifted = true;
  static constexpr bool kShiftCompute = true;
  static constexpr float kScale = 1.0f;
  __device__ static T dec(E e) { return __uint_as_float(static_cast<uint32_t>(e) << 16); }
  __device__ static E enc(T t) { return __bfloat16_as_ushort(__float2bfloat16_rn(t)); }
  __device__ static float2 dec2(uint32_t w) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
  }
  __device__ static uint32_t enc2(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
  }
  // BF16 keeps the FP32 exponent range, so the same form is exact for every normal FP32
  // value: 16 random bits below the BF16 mantissa (lower element bits 15..0, upper element
  // bits 31..16), then truncation.
  __device__ static uint32_t enc2_sr(float lo, float hi, uint32_t rbits) {
    const float l = __uint_as_float(__float_as_uint(lo) + (rbits & 0xffffu));
    const float h = __uint_as_float(__float_as_uint(hi) + (rbits >> 16));
    uint32_t d;
    asm("cvt.rz.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(h), "f"(l));
    return d;
  }
};

// ---- per-domain constants in compute precision -----------------------------------------

// w_alpha rho0 of direction a in compute precision (the shift of the shifted variables)
template <typename T> __device__ __forceinline__ T shift_of(const CellConst<T> &c, int a) {
  return a == 0 ? c.wr0 : (a < 5 ? c.wr1 : c.wr2);
}

template <typename T> __device__ __forceinline__ const CellConst<T> &cell_const(const DomDev &d);
template <> __device__ __forceinline__ const CellConst<float> &cell_const<float>(const DomDev &d) {
  return d.cf;
}
template <> __device__ __forceinline__ const CellConst<double> &cell_const<double>(const DomDev &d) {
  return d.cd;
}

__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
// FP32 reciprocal of rho: the hardware approximation (max error about 1 ulp), one
// instruction instead of the correctly rounded sequence; FP64 keeps the IEEE division.
__device__ __forceinline__ float rcp_(float a) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ double rcp_(double a) { return 1.0 / a; }

// Two nodes' values in the two lanes of a packed FP32 pair. Every operation is the
// lane-wise IEEE operation rounded to nearest (the paired FP32 instructions of sm_100 and
// later), so a node updated as half of a pair gets the same bits as when updated alone;
// the pair halves the instruction count of the FP32 update.
struct F2 {
  float2 v;
  F2() = default;
  __device__ __forceinline__ explicit F2(float s) : v(make_float2(s, s)) {}
  __device__ __forceinline__ F2(float2 p) : v(p) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(make_float2(-a.v.x, -a.v.y)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__fadd2_rn(a.v, (-b).v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 fma_(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ F2 rcp_(F2 a) { return F2(make_float2(rcp_(a.v.x), rcp_(a.v.y))); }

// Constants of the force-free update broadcast to both lanes of a pair.
__device__ __forceinline__ CellConst<F2> pair_const(const CellConst<float> &c) {
  CellConst<F2> p;
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

// Rounding of two nodes' post-collision values (compute space, packed in pairs) to the
// 16-bit storage words.
//
// Stochastic rounding. A 16-bit unit of a moving population (about 1.5e-5 at the
// magnitudes of flows at U = 0.05) is far above the per-step change of slow modes: the
// relaxation of the mean-density level of an open channel, a viscous spin-up, the decay
// of a weak shear wave. Rounded to nearest, such increments are lost every step and
// those modes freeze. Each value is therefore rounded up or down with probabilities that
// make the stored value exact in expectation, using counter-based random bits: a hash of
// (step index, row, aligned group of eight columns), multiplied by an odd constant per
// column pair of the group (a bijection of the 32-bit words, so both 16-bit halves stay
// uniformly distributed; the pair's first node takes the low half, the second the high
// half). The nine values of a node share their bits: each is still exact in
// expectation. The bits depend on nothing else, so results are the same for every tile
// shape, kernel variant and batch composition.
//
// Mass kept. The collision conserves each node's mass (Eq. (rho) of the post-collision
// populations equals that of the pulled ones, d), but rounding the nine values
// separately does not. The eight moving populations are rounded first and the rest
// population is stored as d minus their rounded values, rounded once: the stored node
// mass is d within one unit of the rest population (whose shifted value is small, so
// that unit is the finest of the nine), and exact in expectation. `d` is the pulled
// mass (the sum of the nine pulled values in compute space).

// 32-bit integer finalizer of the xorshift-multiply family (shift/multiply constants
// from C. Wellons' published hash-prospector search, "lowbias32").
__device__ __forceinline__ uint32_t sr_hash(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// hash input of a row: step index and row. The odd multipliers here and below are the
// five 32-bit primes of Y. Collet's published xxHash32 (PRIME32_1, _2, _3, _5, and _4 less
// one, doubled per column pair), used only as well-mixed odd constants.
__device__ __forceinline__ uint32_t sr_row_key(long long n, int j) {
  return static_cast<uint32_t>(n) * 0x9e3779b1u + static_cast<uint32_t>(j) * 0x85ebca77u;
}
// bits of the aligned group of eight columns holding column i
__device__ __forceinline__ uint32_t sr_group_bits(uint32_t row_key, int i) {
  return sr_hash(row_key + static_cast<uint32_t>(i >> 3) * 0xc2b2ae3du);
}
// bits of the column pair (i, i + 1), i even, from its group's bits: odd multiplier per
// pair of the group
__device__ __forceinline__ uint32_t sr_pair_bits(uint32_t group_bits, int i) {
  return group_bits * (0x165667b1u + (static_cast<uint32_t>((i >> 1) & 3) << 1) * 0x27d4eb2eu);
}

// Encoder of one node pair, fed opposite direction pairs (a, -a) in the order (1,3),
// (2,4), (5,7), (6,8) as the collision finishes them (so their FP32 values need not stay
// live), then finished with the pulled mass.
template <int S> struct PairEncoder {
  uint32_t bits;
  uint32_t w[kQ];
  F2 s[4];  // rounded r_a + r_-a per opposite pair
  __device__ __forceinline__ explicit PairEncoder(uint32_t b) : bits(b) {}
  __device__ __forceinline__ void operator()(int ia, int ib, F2 xa, F2 xb) {
    w[ia] = Codec<S>::enc2_sr(xa.v.x, xa.v.y, bits);
    w[ib] = Codec<S>::enc2_sr(xb.v.x, xb.v.y, bits);
    const int q = ia == 1 ? 0 : ia == 2 ? 1 : ia == 5 ? 2 : 3;
    s[q] = F2(Codec<S>::dec2(w[ia])) + F2(Codec<S>::dec2(w[ib]));
  }
  __device__ __forceinline__ void finish(F2 d) {
    const F2 moved = (s[0] + s[1]) + (s[2] + s[3]);
    const F2 rest = d - moved;
    w[0] = Codec<S>::enc2_sr(rest.v.x, rest.v.y, bits);
  }
};

template <int S>
__device__ __forceinline__ void encode_pair_mass_kept(const F2 (&x)[kQ], F2 d, uint32_t bits,
                                                      uint32_t (&w)[kQ]) {
  PairEncoder<S> e(bits);
  e(1, 3, x[1], x[3]);
  e(2, 4, x[2], x[4]);
  e(5, 7, x[5], x[7]);
  e(6, 8, x[6], x[8]);
  e.finish(d);
#pragma unroll
  for (int a = 0; a < kQ; ++a) w[a] = e.w[a];
}

// Macroscopic quantities of one node (steps (4)-(5) of the algorithm, Sec. 2.2).
template <typename T> struct NodeMacro {
  T d;       // sum of the stored values (rho - rho0 for shifted storage, rho otherwise)
  T rho;     // Eq. (rho)
  T ux, uy;  // corrected velocity u = u* + du, Eq. (velocity-r)
  T fx, fy;  // F_VP, Eq. (force-density); zero in fluid nodes
};

// x[]: the nine pulled values in compute space. solid: chi = 1 at this node, with
// obstacle velocity (uox, uoy).
template <typename T, bool SHIFT, bool FORCE>
__device__ __forceinline__ NodeMacro<T> node_macro(const T (&x)[kQ], const CellConst<T> &c,
                                                   bool solid, T uox, T uoy) {
  NodeMacro<T> m;
  // Eq. (rho) and Eq. (rho*velocity-star), in a fixed pairwise order
  m.d = (x[0] + (x[1] + x[3])) + ((x[2] + x[4]) + ((x[5] + x[7]) + (x[6] + x[8])));
  m.rho = SHIFT ? c.rho0 + m.d : m.d;
  const T jx = (x[1] - x[3]) + ((x[5] - x[7]) + (x[8] - x[6]));
  const T jy = (x[2] - x[4]) + ((x[5] - x[7]) + (x[6] - x[8]));
  const T inv = rcp_(m.rho);
  m.ux = jx * inv;  // u*
  m.uy = jy * inv;
  m.fx = T(0);
  m.fy = T(0);
  if (FORCE && solid) {
    // Eq. (d-V) with chi = 1, dt = 1: du = (U_O - u*) / (2 eta + 1);
    // Eq. (force-density): F_VP = 2 rho (U_O - u*) / (2 eta + 1) = 2 rho du
    const T dux = (uox - m.ux) * c.inv_2eta1;
    const T duy = (uoy - m.uy) * c.inv_2eta1;
    const T two_rho = m.rho + m.rho;
    m.fx = two_rho * dux;
    m.fy = two_rho * duy;
    m.ux = m.ux + dux;  // Eq. (velocity-r)
    m.uy = m.uy + duy;
  }
  return m;
}

// TRT collision with the split Guo term, Eq. (TRT-collision) and Eq. (collision-modified):
//   g_a = f_a - w+ (f^s_a - f^eq,s_a) - w- (f^a_a - f^eq,a_a) + (1 - w+/2) F^s_a + (1 - w-/2) F^a_a
// evaluated per opposite pair (a, -a), in place on x[]. For shifted storage every
// symmetric quantity is taken relative to w_a rho0, which cancels in f^s - f^eq,s.
struct NoPairHook {
  template <typename T> __device__ __forceinline__ void operator()(int, int, T, T) {}
};

// `done(ia, ib, x[ia], x[ib])` is called as each opposite pair is finished.
template <typename T, bool SHIFT, bool FORCE, typename Hook = NoPairHook>
__device__ __forceinline__ void collide(T (&x)[kQ], const NodeMacro<T> &m, const CellConst<T> &c,
                                        Hook &&done = Hook()) {
  const T base = SHIFT ? m.d : m.rho;
  const T q = T(1.5) * fma_(m.uy, m.uy, m.ux * m.ux);  // 1.5 |u|^2
  // per class: omega+ w rho, omega+ w base, 3 omega- w rho
  const T a0 = c.pw0 * m.rho, b0 = c.pw0 * base;
  const T a1 = c.pw1 * m.rho, b1 = c.pw1 * base;
  const T a2 = c.pw2 * m.rho, b2 = c.pw2 * base;
  const T m1 = c.mw1 * m.rho, m2 = c.mw2 * m.rho;
  T uf = T(0);
  if (FORCE) uf = fma_(m.uy, m.fy, m.ux * m.fx);
  // rest population: g0 = f0 - w+ (f0 - w0 rho (1 - 1.5 u^2)) + (1 - w+/2)(-3 w0 u.F)
  {
    T g0 = fma_(c.one_m_omp, x[0], fma_(-a0, q, b0));
    if (FORCE) g0 = fma_(T(-3) * c.kw0, uf, g0);
    x[0] = g0;
  }
  // one opposite pair with direction e (eu = e.u, ef = e.F)
  auto pair = [&](int ia, int ib, T eu, T ef, T a, T b, T mm, T kw, T qw) {
    const T xs = x[ia] + x[ib];
    const T xd = x[ia] - x[ib];
    const T c1 = fma_(T(4.5) * eu, eu, -q);      // 4.5 (e.u)^2 - 1.5 u^2
    const T eqs = fma_(a, c1, b);                // w+ * (f^eq,s - shift)
    T S = fma_(-c.hp, xs, eqs);                  // -w+ (f^s - f^eq,s)
    T A = fma_(-c.hm, xd, mm * eu);              // -w- (f^a - f^eq,a)
    if (FORCE) {
      S = fma_(kw, fma_(T(9) * eu, ef, T(-3) * uf), S);  // (1 - w+/2) F^s
      A = fma_(qw, ef, A);                               // (1 - w-/2) F^a
    }
    x[ia] = (x[ia] + S) + A;
    x[ib] = (x[ib] + S) - A;
    done(ia, ib, x[ia], x[ib]);
  };
  pair(1, 3, m.ux, m.fx, a1, b1, m1, c.kw1, c.qw1);
  pair(2, 4, m.uy, m.fy, a1, b1, m1, c.kw1, c.qw1);
  pair(5, 7, m.ux + m.uy, m.fx + m.fy, a2, b2, m2, c.kw2, c.qw2);
  pair(6, 8, m.uy - m.ux, m.fy - m.fx, a2, b2, m2, c.kw2, c.qw2);
}

// Obstacle velocity of body id b at node (i, j): V + omega z x (x - c), plus
// kappa (x - c) with DEF, in the compute precision (FP64 with explicit roundings for the
// FP64 storage, FP32 otherwise). kappa is a pulsating body's dilation rate and zero for
// rigid bodies: with DEF the term is added without a branch on the body; sweeps of
// batches without pulsating bodies are instantiated without it (it raised their spills).
template <bool DEF>
__device__ __forceinline__ void body_velocity(const DomDev &d, int b, int i, int j,
                                              double &uox, double &uoy) {
  const double *bd = d.bodies + 5 * (b - 1);
  const double cx = __ldg(bd + 0), cy = __ldg(bd + 1), vx = __ldg(bd + 2), vy = __ldg(bd + 3),
               om = __ldg(bd + 4);
  uox = __dsub_rn(vx, __dmul_rn(om, __dsub_rn(double(j), cy)));
  uoy = __dadd_rn(vy, __dmul_rn(om, __dsub_rn(double(i + d.x0), cx)));  // global column
  if constexpr (DEF) {
    const double kp = __ldg(d.kappa + (b - 1));
    uox = __dadd_rn(uox, __dmul_rn(kp, __dsub_rn(double(i + d.x0), cx)));
    uoy = __dadd_rn(uoy, __dmul_rn(kp, __dsub_rn(double(j), cy)));
  }
}

template <bool DEF>
__device__ __forceinline__ void body_velocity(const DomDev &d, int b, int i, int j,
                                              float &uox, float &uoy) {
  const float *bd = d.bodies_f + 5 * (b - 1);
  const float cx = __ldg(bd + 0), cy = __ldg(bd + 1), vx = __ldg(bd + 2), vy = __ldg(bd + 3),
              om = __ldg(bd + 4);
  uox = vx - om * (float(j) - cy);
  uoy = vy + om * (float(i + d.x0) - cx);
  if constexpr (DEF) {
    const float kp = __ldg(d.kappa_f + (b - 1));
    uox += kp * (float(i + d.x0) - cx);
    uoy += kp * (float(j) - cy);
  }
}

// Scalar pull of direction a at node (i, j) with the edge rules (Eq. streaming):
// source (i - e_x, j - e_y); west inlet -> ghost, east outflow -> last column, x first;
// then free-slip -> reflected direction in the clamped row; periodic edges wrap.
template <int S>
__device__ __forceinline__ typename Codec<S>::T pull_scalar(const DomDev &d, const void *lat,
                                                           int a, int i, int j) {
  using Cd = Codec<S>;
  using E = typename Cd::E;
  int sx = i - ex_of(a), sy = j - ey_of(a), src = a;
  // a NEIGHBOR edge reads the adjacent column of the linked domain's lattice (the same
  // lattice index: linked domains step together)
  const void *from = lat;
  int pitch = d.pitch;
  const int par = lat == d.lat[1] ? 1 : 0;
  if (sx < 0) {
    if (d.west == LBM_INLET_EQ) return cell_const<typename Cd::T>(d).ghost[a];
    if (d.west == LBM_NEIGHBOR) {
      from = d.nb_lat[0][par];
      pitch = d.nb_pitch[0];
      sx = d.nb_nx[0] - 1;
    } else {
      sx += d.nx;
    }
  } else if (sx > d.nx - 1) {
    if (d.east == LBM_NEIGHBOR) {
      from = d.nb_lat[1][par];
      pitch = d.nb_pitch[1];
      sx = 0;
    } else {
      sx = (d.east == LBM_OUTFLOW_ZG) ? d.nx - 1 : sx - d.nx;
    }
  }
  if (sy < 0) {
    if (d.south == LBM_FREE_SLIP) { sy = 0; src = reflect_y(a); }
    else sy += d.ny;
  } else if (sy > d.ny - 1) {
    if (d.north == LBM_FREE_SLIP) { sy = d.ny - 1; src = reflect_y(a); }
    else sy -= d.ny;
  }
  const E *p = static_cast<const E *>(from);
  typename Cd::T x = Cd::dec(p[(static_cast<size_t>(src) * d.ny + sy) * pitch + sx]);
  if (Cd::kShiftCompute && !Cd::kStoreShifted) x -= shift_of(cell_const<typename Cd::T>(d), a);
  return x;
}

}  // namespace lbm
