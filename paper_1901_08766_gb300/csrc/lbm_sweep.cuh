// The fused TRT-LBM-VP sweep: one launch advances every active domain of a batch by
// one time step (steps (3), (4), (5), (6), (2) of the algorithm of Sec. 2.2, fused per
// node since volume penalization needs only the node's own variables).
//
// Work decomposition. A persistent grid walks a tile list. A tile is a strip of
// 32 * V cells of one row range: lane l of each warp owns V consecutive cells
// x0 + l*V .. x0 + l*V + V-1 and a warp walks `rows` rows of it; the warps take these
// (tile, rows) items in turn from a device counter. Each of the nine
// populations of a row is read with one aligned vector load per lane from the
// structure-of-arrays lattice [9][ny][pitch]; the +-1 x-shift of the pull (Eq.
// streaming) is done in registers with one warp shuffle per direction, the two
// strip-end cells come from a scalar load by the end lanes, and the domain-edge
// rules are applied to the row pointers (y) and to the end cells (x). The update is
// written back with aligned vector stores to the other lattice (double buffering).
#pragma once

#include "lbm_cell.cuh"

namespace lbm {

// V consecutive storage elements held by one lane.
template <int S, int V> struct Strip;

// 16-bit storage: V/2 packed 32-bit words, element 2k in the low half of word k.
template <int S, int V> struct Strip16 {
  static_assert(V % 2 == 0, "16-bit strips hold an even number of cells");
  static constexpr int kW = V / 2;
  uint32_t w[kW];
  // Row loads are read-only for the whole launch; the L2 256-byte prefetch hint makes the
  // DRAM requests of a warp's 512-byte row segment arrive as whole 256-byte blocks
  // (measured 3 % faster than plain 16-byte loads on the batched workload).
  __device__ void load(const uint16_t *p) {
    if constexpr (kW == 4) {
      asm volatile("ld.global.nc.L2::256B.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
                   : "l"(p));
    } else if constexpr (kW == 2) {
      asm volatile("ld.global.nc.L2::256B.v2.u32 {%0, %1}, [%2];" : "=r"(w[0]), "=r"(w[1]) : "l"(p));
    } else {
      w[0] = __ldg(reinterpret_cast<const unsigned int *>(p));
    }
  }
  // aligned vector read from shared memory
  __device__ void load_shared(const uint16_t *p) {
    if constexpr (kW == 4) {
      const uint4 v = *reinterpret_cast<const uint4 *>(p);
      w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else if constexpr (kW == 2) {
      const uint2 v = *reinterpret_cast<const uint2 *>(p);
      w[0] = v.x; w[1] = v.y;
    } else {
      w[0] = *reinterpret_cast<const uint32_t *>(p);
    }
  }
  __device__ void store(uint16_t *p) const {
    if constexpr (kW == 4) {
      *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    } else if constexpr (kW == 2) {
      *reinterpret_cast<uint2 *>(p) = make_uint2(w[0], w[1]);
    } else {
      *reinterpret_cast<uint32_t *>(p) = w[0];
    }
  }
  __device__ void zero() {
#pragma unroll
    for (int k = 0; k < kW; ++k) w[k] = 0u;
  }
  __device__ uint16_t get(int k) const {
    return static_cast<uint16_t>((k & 1) ? (w[k >> 1] >> 16) : (w[k >> 1] & 0xffffu));
  }
  __device__ void set(int k, uint16_t e) {
    uint32_t &x = w[k >> 1];
    x = (k & 1) ? ((x & 0x0000ffffu) | (static_cast<uint32_t>(e) << 16))
                : ((x & 0xffff0000u) | e);
  }
  // element k <- element k-1; element 0 <- `in` (the previous cell)
  __device__ void shift_up(uint16_t in) {
#pragma unroll
    for (int k = kW - 1; k > 0; --k) w[k] = __byte_perm(w[k - 1], w[k], 0x5432);
    w[0] = __byte_perm(static_cast<uint32_t>(in) << 16, w[0], 0x5432);
  }
  // element k <- element k+1; element V-1 <- `in` (the next cell)
  __device__ void shift_down(uint16_t in) {
#pragma unroll
    for (int k = 0; k < kW - 1; ++k) w[k] = __byte_perm(w[k], w[k + 1], 0x5432);
    w[kW - 1] = __byte_perm(w[kW - 1], static_cast<uint32_t>(in), 0x5432);
  }
  __device__ uint16_t last() const { return static_cast<uint16_t>(w[kW - 1] >> 16); }
  __device__ uint16_t first() const { return static_cast<uint16_t>(w[0] & 0xffffu); }
};

template <int V> struct Strip<LBM_F16S, V> : Strip16<LBM_F16S, V> {};
template <int V> struct Strip<LBM_BF16S, V> : Strip16<LBM_BF16S, V> {};

// 32/64-bit storage: one register (pair) per element.
template <typename E, int V> struct StripW {
  E w[V];
  __device__ void load(const E *p) {
    constexpr int kBytes = V * int(sizeof(E));
    if constexpr (kBytes == 16) {
      if constexpr (sizeof(E) == 4) {
        asm volatile("ld.global.nc.L2::256B.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(w[0]), "=f"(w[1]), "=f"(w[2]), "=f"(w[3])
                     : "l"(p));
      } else {
        asm volatile("ld.global.nc.L2::256B.v2.f64 {%0, %1}, [%2];" : "=d"(w[0]), "=d"(w[1]) : "l"(p));
      }
    } else if constexpr (kBytes == 8) {
      if constexpr (sizeof(E) == 4) {
        asm volatile("ld.global.nc.L2::256B.v2.f32 {%0, %1}, [%2];" : "=f"(w[0]), "=f"(w[1]) : "l"(p));
      } else {
        w[0] = __ldg(p);
      }
    } else {
#pragma unroll
      for (int k = 0; k < V; ++k) w[k] = __ldg(p + k);
    }
  }
  __device__ void load_shared(const E *p) {
    constexpr int kBytes = V * int(sizeof(E));
    if constexpr (kBytes == 16) {
      if constexpr (sizeof(E) == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
      } else {
        const double2 v = *reinterpret_cast<const double2 *>(p);
        w[0] = v.x; w[1] = v.y;
      }
    } else if constexpr (kBytes == 8 && sizeof(E) == 4) {
      const float2 v = *reinterpret_cast<const float2 *>(p);
      w[0] = v.x; w[1] = v.y;
    } else {
#pragma unroll
      for (int k = 0; k < V; ++k) w[k] = p[k];
    }
  }
  __device__ void store(E *p) const {
    constexpr int kBytes = V * int(sizeof(E));
    if constexpr (kBytes == 16) {
      if constexpr (sizeof(E) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(w[0], w[1], w[2], w[3]);
      } else {
        *reinterpret_cast<double2 *>(p) = make_double2(w[0], w[1]);
      }
    } else if constexpr (kBytes == 8 && sizeof(E) == 4) {
      *reinterpret_cast<float2 *>(p) = make_float2(w[0], w[1]);
    } else {
#pragma unroll
      for (int k = 0; k < V; ++k) p[k] = w[k];
    }
  }
  __device__ void zero() {
#pragma unroll
    for (int k = 0; k < V; ++k) w[k] = E(0);
  }
  __device__ E get(int k) const { return w[k]; }
  __device__ void set(int k, E e) { w[k] = e; }
  __device__ void shift_up(E in) {
#pragma unroll
    for (int k = V - 1; k > 0; --k) w[k] = w[k - 1];
    w[0] = in;
  }
  __device__ void shift_down(E in) {
#pragma unroll
    for (int k = 0; k < V - 1; ++k) w[k] = w[k + 1];
    w[V - 1] = in;
  }
  __device__ E last() const { return w[V - 1]; }
  __device__ E first() const { return w[0]; }
};

template <int V> struct Strip<LBM_F32, V> : StripW<float, V> {};
template <int V> struct Strip<LBM_F64, V> : StripW<double, V> {};

template <typename E> __device__ __forceinline__ E shfl_up1(E v) {
  if constexpr (sizeof(E) == 2) {
    return static_cast<E>(__shfl_up_sync(0xffffffffu, static_cast<uint32_t>(v), 1));
  } else {
    return __shfl_up_sync(0xffffffffu, v, 1);
  }
}
template <typename E> __device__ __forceinline__ E shfl_down1(E v) {
  if constexpr (sizeof(E) == 2) {
    return static_cast<E>(__shfl_down_sync(0xffffffffu, static_cast<uint32_t>(v), 1));
  } else {
    return __shfl_down_sync(0xffffffffu, v, 1);
  }
}

// Decode element k of every direction into compute space.
template <int S, int V>
__device__ __forceinline__ void decode_cell(const Strip<S, V> (&v)[kQ], int k,
                                            typename Codec<S>::T (&x)[kQ]) {
#pragma unroll
  for (int a = 0; a < kQ; ++a) x[a] = Codec<S>::dec(v[a].get(k));
}

// One strip row of the nine source populations, its strip-end values and body ids.
template <int S, int V> struct RowData {
  Strip<S, V> v[kQ];
  typename Codec<S>::E end_in[kQ];
  uint32_t mb[(V + 3) / 4];  // body ids of the V cells, four per word (low byte first)
  __device__ int body(int k) const { return (mb[k >> 2] >> (8 * (k & 3))) & 0xff; }
};

// Phase 3 of a strip row, shared by the row pipelines: update the V pulled nodes of a
// lane in place (inlet ghost, moments, penalization, collision, F_VP of solid nodes,
// stability check, rounding to the storage type) and zero the padding beyond nx. mb: the
// nodes' body ids, four per word; fvp: the F_VP field of this step's parity. The caller
// stores v[].
// The update of a 16-bit strip that holds solid nodes, node by node in FP32 (moments,
// penalization, collision, F_VP, stability bits as in update_strip), out of line: the
// strips of the force-free path, nearly all of them, then run with the registers this
// path would otherwise claim (the direct sweep at 24 resident warps: 168 B of spills
// before, 72 B after; 376 -> 358 us on the 64-domain batch). w: the strip's words
// [kQ][V / 2], updated in place; mb0, mb1: its mask bytes; fvp: the F_VP field of this
// step's parity. Returns the nodes whose density left (0.01, 100) as bits.
template <int S, int V, bool DEF>
__device__ __noinline__ unsigned solid_strip16(uint32_t *w, uint32_t mb0, uint32_t mb1, const DomDev &D,
                                             void *fvp, const CellConst<float> &C, int lane, int xl, int j,
                                             bool west_first, uint32_t sr_g) {
  using Cd = Codec<S>;
  constexpr bool SHIFT = Cd::kShiftCompute;
  constexpr float kRhoMid = 50.005f * float(Cd::kScale), kRhoHalf = 49.995f * float(Cd::kScale);
  constexpr float kUnscale = 1.0f / float(Cd::kScale);
  float *__restrict__ dfvp = static_cast<float *>(fvp);
  unsigned bb = 0u;
#pragma unroll
  for (int k = 0; k < V; k += 2) {
    float x0[kQ], x1[kQ];
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
      const float2 p = Cd::dec2(w[a * (V / 2) + (k >> 1)]);
      x0[a] = p.x;
      x1[a] = p.y;
    }
    float d[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float (&x)[kQ] = h ? x1 : x0;
      const int kk = k + h;
      if (kk == 0 && west_first) {
        const bool g = lane == 0;
        x[1] = g ? C.ghost[1] : x[1];
        x[5] = g ? C.ghost[5] : x[5];
        x[8] = g ? C.ghost[8] : x[8];
      }
      float uox = 0.f, uoy = 0.f;
      const uint32_t mw = kk < 4 ? mb0 : mb1;
      const int bk = (mw >> (8 * (kk & 3))) & 0xff;
      const bool solid = bk != 0;
      if (solid) body_velocity<DEF>(D, bk, xl + kk, j, uox, uoy);
      NodeMacro<float> m = node_macro<float, SHIFT, true>(x, C, solid, uox, uoy);
      collide<float, SHIFT, true>(x, m, C);
      if (solid) {
        float *__restrict__ fv = dfvp + 2 * (static_cast<size_t>(j) * D.pitch + xl + kk);
        fv[0] = m.fx * kUnscale;
        fv[1] = m.fy * kUnscale;
      }
      bb |= (fabs(m.rho - kRhoMid) < kRhoHalf ? 0u : 1u) << kk;
      d[h] = m.d;
    }
    F2 xp[kQ];
#pragma unroll
    for (int a = 0; a < kQ; ++a) xp[a] = F2(make_float2(x0[a], x1[a]));
    uint32_t ww[kQ];
    encode_pair_mass_kept<S>(xp, F2(make_float2(d[0], d[1])), sr_pair_bits(sr_g, xl + k + D.x0), ww);
#pragma unroll
    for (int a = 0; a < kQ; ++a) w[a * (V / 2) + (k >> 1)] = ww[a];
  }
  return bb;
}

template <int S, int V, bool DEF>
__device__ __forceinline__ void update_strip(Strip<S, V> (&v)[kQ], const uint32_t (&mb)[(V + 3) / 4],
                                             const DomDev &D,
                                             const CellConst<typename Codec<S>::T> &C,
                                             const CellConst<typename Codec<S>::T> &CF,
                                             const CellConst<F2> &CP, const int lane, const int xl,
                                             const int j, const long long n, const bool west_edge,
                                             const bool west_inlet, const bool east_edge,
                                             const int nx, void *fvp, int &unstable) {
  using Cd = Codec<S>;
  using E = typename Cd::E;
  using T = typename Cd::T;
  constexpr bool SHIFT = Cd::kShiftCompute;
  constexpr bool kAddShift = Cd::kShiftCompute && !Cd::kStoreShifted;
  constexpr T kRhoMid = T(50.005) * T(Cd::kScale), kRhoHalf = T(49.995) * T(Cd::kScale);
  constexpr T kUnscale = T(1) / T(Cd::kScale);
  const int pitch = D.pitch;
  T *__restrict__ dfvp = static_cast<T *>(fvp);
  bool any_solid_lane = false;
#pragma unroll
  for (int q = 0; q < (V + 3) / 4; ++q) any_solid_lane |= (mb[q] != 0u);
  const bool any_solid = __any_sync(0xffffffffu, any_solid_lane);

  // ---- phase 3: update the V nodes in place ----------------------------------------
  // bit k: node xl + k lies inside the domain (all V except at the east edge)
  const unsigned valid_bits =
      east_edge ? (nx - xl >= V ? (1u << V) - 1u : (nx > xl ? (1u << (nx - xl)) - 1u : 0u))
                : (1u << V) - 1u;
  unsigned bad_bits = 0u;
  // random bits of the 16-bit rounding (a strip of V <= 8 cells lies in one group)
  // (keyed by the global column: slabs of one grid round as the whole grid does)
  const uint32_t sr_g = sizeof(E) == 2 ? sr_group_bits(sr_row_key(n, j), xl + D.x0) : 0u;
  // one node: inlet ghost, moments, penalization, collision, F_VP, stability check
  auto update = [&](T (&x)[kQ], int k) {
    if (k == 0 && west_edge && west_inlet) {
      // inlet ghost populations entering node 0 from x = -1
      const bool g = lane == 0;
      x[1] = g ? C.ghost[1] : x[1];
      x[5] = g ? C.ghost[5] : x[5];
      x[8] = g ? C.ghost[8] : x[8];
    }
    NodeMacro<T> m;
    if (any_solid) {
      T uox = T(0), uoy = T(0);
      const int bk = ((mb[k >> 2] >> (8 * (k & 3))) & 0xff);
      const bool solid = bk != 0;
      if (solid) body_velocity<DEF>(D, bk, xl + k, j, uox, uoy);
      m = node_macro<T, SHIFT, true>(x, C, solid, uox, uoy);
      collide<T, SHIFT, true>(x, m, C);
      if (solid) {
        // F_VP of this node for the body-force reduction (unscaled: power of two)
        T *__restrict__ fv = dfvp + 2 * (static_cast<size_t>(j) * pitch + xl + k);
        fv[0] = m.fx * kUnscale;
        fv[1] = m.fy * kUnscale;
      }
    } else {
      m = node_macro<T, SHIFT, false>(x, CF, false, T(0), T(0));
      collide<T, SHIFT, false>(x, m, CF);
    }
    // rho outside (0.01, 100) or not finite; padding nodes are masked out per row
    bad_bits |= (fabs(m.rho - kRhoMid) < kRhoHalf ? 0u : 1u) << k;
    return m.d;
  };
#ifndef LBM_PAIRED
#define LBM_PAIRED 1
#endif
  if constexpr (sizeof(E) == 2) {
    // 16-bit storage: two nodes per packed word, converted pairwise
    if (LBM_PAIRED && !any_solid) {
      // force-free rows: both nodes of a word updated together in packed FP32 pairs
#pragma unroll
      for (int k = 0; k < V; k += 2) {
        F2 x[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) x[a] = F2(Cd::dec2(v[a].w[k >> 1]));
        if (k == 0 && west_edge && west_inlet) {
          const bool g = lane == 0;
          x[1].v.x = g ? C.ghost[1] : x[1].v.x;
          x[5].v.x = g ? C.ghost[5] : x[5].v.x;
          x[8].v.x = g ? C.ghost[8] : x[8].v.x;
        }
        const NodeMacro<F2> m = node_macro<F2, SHIFT, false>(x, CP, false, F2(0.f), F2(0.f));
        bad_bits |= (fabsf(m.rho.v.x - kRhoMid) < kRhoHalf ? 0u : 1u) << k;
        bad_bits |= (fabsf(m.rho.v.y - kRhoMid) < kRhoHalf ? 0u : 1u) << (k + 1);
        // each opposite pair is rounded as soon as the collision finishes it
        PairEncoder<S> enc(sr_pair_bits(sr_g, xl + k + D.x0));
        collide<F2, SHIFT, false>(x, m, CP, enc);
        enc.finish(m.d);
#pragma unroll
        for (int a = 0; a < kQ; ++a) v[a].w[k >> 1] = enc.w[a];
      }
    } else if constexpr (S == LBM_F16S) {
      // strips with solid nodes: out of line (solid_strip16)
      uint32_t wl[kQ * (V / 2)];
#pragma unroll
      for (int a = 0; a < kQ; ++a)
#pragma unroll
        for (int q = 0; q < V / 2; ++q) wl[a * (V / 2) + q] = v[a].w[q];
      bad_bits |= solid_strip16<S, V, DEF>(wl, mb[0], (V + 3) / 4 > 1 ? mb[(V + 3) / 4 - 1] : 0u, D, fvp, C, lane,
                                           xl, j, west_edge && west_inlet, sr_g);
#pragma unroll
      for (int a = 0; a < kQ; ++a)
#pragma unroll
        for (int q = 0; q < V / 2; ++q) v[a].w[q] = wl[a * (V / 2) + q];
    } else {
      // BF16-shifted: inline (its force-free path spilled more with the call: 377 -> 383 us)
#pragma unroll
      for (int k = 0; k < V; k += 2) {
        T x0[kQ], x1[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) {
          const float2 p = Cd::dec2(v[a].w[k >> 1]);
          x0[a] = p.x;
          x1[a] = p.y;
        }
        const float d0 = update(x0, k);
        const float d1 = update(x1, k + 1);
        F2 xp[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) xp[a] = F2(make_float2(x0[a], x1[a]));
        uint32_t w[kQ];
        encode_pair_mass_kept<S>(xp, F2(make_float2(d0, d1)), sr_pair_bits(sr_g, xl + k + D.x0), w);
#pragma unroll
        for (int a = 0; a < kQ; ++a) v[a].w[k >> 1] = w[a];
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k) {
      T x[kQ];
      decode_cell<S, V>(v, k, x);
      if constexpr (kAddShift) {
#pragma unroll
        for (int a = 0; a < kQ; ++a) x[a] -= shift_of(CF, a);  // exact (Sterbenz)
      }
      update(x, k);
      if constexpr (kAddShift) {
#pragma unroll
        for (int a = 0; a < kQ; ++a) x[a] += shift_of(CF, a);
      }
#pragma unroll
      for (int a = 0; a < kQ; ++a) v[a].set(k, Cd::enc(x[a]));
    }
  }
  if (bad_bits & valid_bits) unstable = 1;
  if (east_edge) {
    // keep the row padding beyond nx at zero
#pragma unroll
    for (int k = 0; k < V; ++k)
      if (!((valid_bits >> k) & 1u)) {
#pragma unroll
        for (int a = 0; a < kQ; ++a) v[a].set(k, E(0));
      }
  }
}

// The sweep body. PF = false: each warp loads a row, then updates it. PF = true: the
// loads of the warp's next row are issued into a second register set before the current
// row is updated, so that they overlap the update (more registers, fewer warps).
template <int S, int V, bool PF, bool DEF = true>
__device__ __forceinline__ void sweep_body(const SweepArgs &args, int s) {
  using Cd = Codec<S>;
  using E = typename Cd::E;
  using T = typename Cd::T;
  constexpr int kStrip = 32 * V;
  static_assert(sizeof(E) != 2 || (V <= 8 && 8 % V == 0),
                "a 16-bit strip must lie in one group of eight columns (rounding bits)");
  const int lane = threadIdx.x & 31;
  const int ntiles = args.ctr->ntiles;
  const long long run_base = args.ctr->run_base;
  int unstable = 0;

  // Work items are (tile, warp slot) pairs: the `rows` rows y0 + slot * rows ... of a tile.
  // Warps take them in turn from a counter (the next index is fetched while the current
  // item is processed), so the warps finish together however unevenly the items cost
  // (tiles holding bodies take the force path). The last warp to run out resets the
  // counters for the next launch; items are visited in tile order.
  Counters *const ctr = const_cast<Counters *>(args.ctr);
  const int slots = static_cast<int>(blockDim.x >> 5);
  const int nitems = ntiles * slots;
  int item = 0;
  if (lane == 0) item = atomicAdd(&ctr->item_next, 1);
  item = __shfl_sync(0xffffffffu, item, 0);
  while (item < nitems) {
    int next = 0;
    if (lane == 0) next = atomicAdd(&ctr->item_next, 1);
    const int t = item / slots;
    const int slot = item - t * slots;
    const TileDev tile = args.tiles[t];
    const DomDev &D = args.doms[tile.dom];
    const DomDyn dy = args.dyn[tile.dom];
    const long long n = dy.step0 + run_base + s;
    if (n >= dy.step_end) {
      item = __shfl_sync(0xffffffffu, next, 0);
      continue;
    }
    const int par = (dy.parity + static_cast<int>((run_base + s) & 1)) & 1;
    const E *__restrict__ src = static_cast<const E *>(D.lat[par]);
    E *__restrict__ dst = static_cast<E *>(D.lat[par ^ 1]);
    const int nx = D.nx, ny = D.ny, pitch = D.pitch;
    const int x0 = tile.x0;
    const int xl = x0 + lane * V;
    const bool lane_on = xl < nx;
    const bool west_edge = (x0 == 0);
    const bool east_edge = (x0 + kStrip >= nx);
    const bool west_inlet = D.west == LBM_INLET_EQ;
    const bool east_out = D.east == LBM_OUTFLOW_ZG;
    const bool south_slip = D.south == LBM_FREE_SLIP;
    const bool north_slip = D.north == LBM_FREE_SLIP;
    const CellConst<T> &C = cell_const<T>(D);
#ifndef LBM_CONST_REGS
#define LBM_CONST_REGS 1
#endif
#if LBM_CONST_REGS
    // The force-free update's constants, read once per tile into registers (the update
    // would otherwise re-read them from global memory on every row).
    CellConst<T> CF;
    CF.omp = C.omp;
    CF.omm = C.omm;
    CF.hp = C.hp;
    CF.hm = C.hm;
    CF.one_m_omp = C.one_m_omp;
    CF.rho0 = C.rho0;
    CF.pw0 = C.pw0;
    CF.pw1 = C.pw1;
    CF.pw2 = C.pw2;
    CF.mw1 = C.mw1;
    CF.mw2 = C.mw2;
    CF.wr0 = C.wr0;
    CF.wr1 = C.wr1;
    CF.wr2 = C.wr2;
#else
    const CellConst<T> &CF = C;
#endif
    // the same constants broadcast to packed pairs (16-bit storage, force-free rows)
    CellConst<F2> CP;
    if constexpr (sizeof(E) == 2) CP = pair_const(CF);
    const uint8_t *__restrict__ dmask = D.mask;
    // strip-end columns read by the end lanes (or -1: nothing to read); at a linked
    // (NEIGHBOR) edge the value comes from the neighbour's lattice instead (below)
    const bool west_link = west_edge && D.west == LBM_NEIGHBOR;
    const bool east_link = east_edge && D.east == LBM_NEIGHBOR;
    const int col_left = west_edge ? ((west_inlet || west_link) ? -1 : nx - 1) : x0 - 1;
    const int col_right = east_edge ? ((east_out || east_link) ? -1 : 0) : x0 + kStrip;
    // the lane holding column nx-1 (east edge tiles) and its element index
    const int k_last = nx - 1 - xl;
    const size_t plane = static_cast<size_t>(ny) * pitch;

    // ---- phase 1: every load of row j ------------------------------------------------
    auto load_row = [&](RowData<S, V> &R, const int j) {
      const E *row[kQ];
      const E *rj = src + static_cast<size_t>(j) * pitch;
      if (j > 0 && j < ny - 1) {
#pragma unroll
        for (int a = 0; a < kQ; ++a) row[a] = rj + (a * plane - static_cast<ptrdiff_t>(ey_of(a)) * pitch);
      } else {
#pragma unroll
        for (int a = 0; a < kQ; ++a) {
          // y rule for this direction (warp-uniform): periodic wrap or free-slip mirror
          const int ey = ey_of(a);
          int sy = j - ey, sa = a;
          if (sy < 0) {
            if (south_slip) { sy = 0; sa = reflect_y(a); }
            else sy += ny;
          } else if (sy > ny - 1) {
            if (north_slip) { sy = ny - 1; sa = reflect_y(a); }
            else sy -= ny;
          }
          row[a] = src + sa * plane + static_cast<size_t>(sy) * pitch;
        }
      }
      auto &v = R.v;
      auto &end_in = R.end_in;
      // Loads are issued by every lane without branches: a lane past the end of the row
      // reads a clamped (valid) strip whose results are neither stored nor used, and the
      // strip-end columns are read by all lanes at one common address (a broadcast) and
      // kept only by the end lanes.
      const int xl_ld = min(xl, pitch - V);
      const int col_l = col_left >= 0 ? col_left : 0;
      const int col_r = col_right >= 0 ? col_right : 0;
#pragma unroll
      for (int a = 0; a < kQ; ++a) {
        v[a].load(row[a] + xl_ld);
        const int ex = ex_of(a);
        end_in[a] = E(0);
        if (ex == 1) end_in[a] = __ldg(row[a] + col_l);
        else if (ex == -1) end_in[a] = __ldg(row[a] + col_r);
      }
      if (west_link || east_link) {
        // linked edge: the adjacent column of the neighbour (its last column to the west,
        // its first to the east), same direction and y rule, same lattice index
#pragma unroll
        for (int a = 0; a < kQ; ++a) {
          const int ex = ex_of(a);
          const int side = ex == 1 ? 0 : 1;
          if (ex == 0 || (ex == 1 && !west_link) || (ex == -1 && !east_link)) continue;
          int sy = j - ey_of(a), sa = a;
          if (sy < 0) {
            if (south_slip) { sy = 0; sa = reflect_y(a); }
            else sy += ny;
          } else if (sy > ny - 1) {
            if (north_slip) { sy = ny - 1; sa = reflect_y(a); }
            else sy -= ny;
          }
          const int npitch = D.nb_pitch[side];
          const E *nrow = static_cast<const E *>(D.nb_lat[side][par]) +
                          (static_cast<size_t>(sa) * ny + sy) * npitch;
          end_in[a] = __ldg(nrow + (side == 0 ? D.nb_nx[0] - 1 : 0));
        }
      }
      {
        // body ids, kept packed (zero for lanes past the end of the row)
        const uint8_t *mrow = dmask + static_cast<size_t>(j) * pitch + xl_ld;
        if constexpr (V == 8) {
          const uint2 mw = __ldg(reinterpret_cast<const uint2 *>(mrow));
          R.mb[0] = lane_on ? mw.x : 0u;
          R.mb[1] = lane_on ? mw.y : 0u;
        } else if constexpr (V == 4) {
          const uint32_t mw = __ldg(reinterpret_cast<const unsigned int *>(mrow));
          R.mb[0] = lane_on ? mw : 0u;
        } else if constexpr (V == 2) {
          const uint32_t mw = __ldg(reinterpret_cast<const unsigned short *>(mrow));
          R.mb[0] = lane_on ? mw : 0u;
        } else {
          const uint32_t mw = __ldg(mrow);
          R.mb[0] = lane_on ? mw : 0u;
        }
      }
    };
    // ---- phases 2 and 3: shift, update and store row j ---------------------------------
    auto process_row = [&](RowData<S, V> &R, const int j) {
      auto &v = R.v;
      const auto &end_in = R.end_in;
      // ---- phase 2: the +-1 x-shift of the pull, in registers -----------------------
#pragma unroll
      for (int a = 0; a < kQ; ++a) {
        const int ex = ex_of(a);
        if (ex == 1) {
          // source i - 1: previous lane's last element; lane 0 takes the strip-end load
          // (at the west edge of an inlet it is replaced by the ghost after decoding)
          E in = shfl_up1<E>(v[a].last());
          in = lane == 0 ? end_in[a] : in;
          v[a].shift_up(in);
        } else if (ex == -1) {
          // source i + 1: next lane's first element; lane 31 takes the strip-end load
          E keep = E(0);
          if (east_edge) {
#pragma unroll
            for (int k = 0; k < V; ++k) keep = (k == k_last) ? v[a].get(k) : keep;
          }
          E in = shfl_down1<E>(v[a].first());
          in = (lane == 31 && !east_edge) ? end_in[a] : in;
          v[a].shift_down(in);
          if (east_edge) {
            const E fix = east_out ? keep : end_in[a];  // zero gradient or periodic
#pragma unroll
            for (int k = 0; k < V; ++k)
              if (k == k_last) v[a].set(k, fix);
          }
        }
      }
      update_strip<S, V, DEF>(v, R.mb, D, C, CF, CP, lane, xl, j, n, west_edge, west_inlet,
                              east_edge, nx, D.fvp[par], unstable);
      if (lane_on) {
#pragma unroll
        for (int a = 0; a < kQ; ++a)
          v[a].store(dst + a * plane + static_cast<size_t>(j) * pitch + xl);
      }
    };
    const int j0 = tile.y0 + slot * args.rows;
    if constexpr (!PF) {
      for (int r = 0; r < args.rows; ++r) {
        const int j = j0 + r;
        if (j >= ny) break;
        RowData<S, V> R;
        load_row(R, j);
        process_row(R, j);
      }
    } else {
      const int jend = min(j0 + args.rows, ny);
      if (j0 < jend) {
        RowData<S, V> A, B;
        load_row(A, j0);
        for (int j = j0; j < jend; j += 2) {
          if (j + 1 < jend) load_row(B, j + 1);
          process_row(A, j);
          if (j + 1 >= jend) break;
          if (j + 2 < jend) load_row(A, j + 2);
          process_row(B, j + 1);
        }
      }
    }
    if (__any_sync(0xffffffffu, unstable)) {
      if (lane == 0) atomicOr(D.status, 1);
      unstable = 0;
    }
    item = __shfl_sync(0xffffffffu, next, 0);
  }
  if (lane == 0) {
    __threadfence();  // this warp's last fetch is ordered before its count
    if (atomicAdd(&ctr->item_done, 1) == static_cast<int>(gridDim.x) * slots - 1) {
      ctr->item_next = 0;
      ctr->item_done = 0;
    }
  }
}

// Register budgets of the direct sweep: the resident warps per SM it is compiled for.
// Row pipeline 0: 16 warps (blocks of up to 16 warps, 128 registers); 3: 20 warps (blocks
// of up to 10 warps, two or more per SM, at most 102 registers); 4: 24 warps (blocks of up
// to 12 warps, at most 85 registers). More resident warps cover more DRAM latency at the
// price of spilled registers; with warps taking work items from the counter (rows of
// unequal cost finish together) 24 warps measured fastest on the 64-domain batch.
template <int R> struct Budget;
template <> struct Budget<16> { static constexpr int kThreads = 512, kBlocks = 1; };
template <> struct Budget<20> { static constexpr int kThreads = 320, kBlocks = 2; };
template <> struct Budget<24> { static constexpr int kThreads = 384, kBlocks = 2; };

constexpr int budget_of_pipe(int pipe) { return pipe == 3 ? 20 : (pipe == 4 ? 24 : 16); }

// DEF: some domain of the batch has pulsating bodies (the kappa term of U_O)
template <int S, int V, bool DEF, int R>
__global__ void __launch_bounds__(Budget<R>::kThreads, Budget<R>::kBlocks) sweep_kernel(SweepArgs args, int s) {
  sweep_body<S, V, false, DEF>(args, s);
}

template <int S, int V>
__global__ void __launch_bounds__(256) sweep_pf_kernel(SweepArgs args, int s) {
  sweep_body<S, V, true>(args, s);
}

template <int S, int V, int R>
cudaError_t launch_sweep_r(int grid, int warps, cudaStream_t st, const SweepArgs &a, int s, bool def) {
  if (def) sweep_kernel<S, V, true, R><<<grid, warps * 32, 0, st>>>(a, s);
  else sweep_kernel<S, V, false, R><<<grid, warps * 32, 0, st>>>(a, s);
  return cudaGetLastError();
}

// The direct sweep (row pipelines 0, 3, 4: its register budgets)
template <int S, int V>
cudaError_t launch_sweep_t(int grid, int warps, cudaStream_t st, const SweepArgs &a, int s, bool def,
                           int pipe) {
  switch (budget_of_pipe(pipe)) {
    case 20: return launch_sweep_r<S, V, 20>(grid, warps, st, a, s, def);
    case 24: return launch_sweep_r<S, V, 24>(grid, warps, st, a, s, def);
    default: return launch_sweep_r<S, V, 16>(grid, warps, st, a, s, def);
  }
}

template <int S, int V>
cudaError_t launch_sweep_pf_t(int grid, int warps, cudaStream_t st, const SweepArgs &a, int s) {
  sweep_pf_kernel<S, V><<<grid, warps * 32, 0, st>>>(a, s);
  return cudaGetLastError();
}

template <int S, int V, int R> int max_blocks_r(int warps) {
  if (warps * 32 > Budget<R>::kThreads) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_kernel<S, V, false, R>, warps * 32, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <int S, int V> int max_blocks_t(int warps, int pipe) {
  switch (budget_of_pipe(pipe)) {
    case 20: return max_blocks_r<S, V, 20>(warps);
    case 24: return max_blocks_r<S, V, 24>(warps);
    default: return max_blocks_r<S, V, 16>(warps);
  }
}

template <int S, int V> int max_blocks_pf_t(int warps) {
  if (warps * 32 > 256) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_pf_kernel<S, V>, warps * 32, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace lbm
