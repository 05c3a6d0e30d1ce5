// TMA-staged variant of the fused TRT-LBM-VP sweep.
//
// Same per-node arithmetic and tile decomposition as sweep_kernel (lbm_sweep.cuh); only
// the way a row reaches the registers differs. Each warp owns a two-stage ring in shared
// memory. While the warp updates row k from stage k&1, one lane has already issued,
// for row k+1, ten 1D bulk copies (cp.async.bulk, the Tensor Memory Accelerator) into
// the other stage: the nine source row segments of the pull (the y rules applied to the
// row addresses, a 16-byte halo on each side for the +-1 x-shift) and the mask row. An
// mbarrier per stage counts the arriving bytes. DRAM latency thus overlaps the compute
// of the previous row instead of stalling it.
//
// Every wait is bounded: if a stage does not complete within the spin limit the warp
// sets bit 1 of the domain status word (reported as LBM_ETIMEOUT), waits a bounded time
// for its other stage and returns. A stage that never completed may still have copies in
// flight when the block exits; the host reports the domain as failed and does not use
// its state. Tests reach this path by host-side injection (bit 0 of SweepArgs::inject),
// which takes it only after the stage's wait has completed.
#pragma once

#include "lbm_sweep.cuh"

namespace lbm {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  constexpr int kSpinLimit = 1 << 22;
  for (int i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Shared-memory geometry of one stage for a given storage type and strip width.
template <int S, int V> struct TmaGeom {
  using E = typename Codec<S>::E;
  static constexpr int kEs = int(sizeof(E));
  static constexpr int kStrip = 32 * V;           // cells per strip
  static constexpr int kHalo = 16 / kEs;          // elements in a 16-byte halo
  static constexpr int kSegElems = kStrip + 2 * kHalo;
  static constexpr int kSegBytes = kSegElems * kEs;
  static constexpr int kMaskBytes = (kStrip + 15) / 16 * 16;
  static constexpr int kStageBytes = ((kQ * kSegBytes + kMaskBytes) + 127) / 128 * 128;
  static constexpr int kWarpBytes = 2 * kStageBytes;
};

template <int S, int V> constexpr int tma_smem_bytes(int warps) {
  return warps * TmaGeom<S, V>::kWarpBytes + warps * 2 * 8;
}

template <int S, int V>
__global__ void __launch_bounds__(512) sweep_tma_kernel(SweepArgs args, int s) {
  using Cd = Codec<S>;
  using E = typename Cd::E;
  using T = typename Cd::T;
  using G = TmaGeom<S, V>;
  constexpr bool SHIFT = Cd::kShiftCompute;
  constexpr bool kAddShift = Cd::kShiftCompute && !Cd::kStoreShifted;
  constexpr int kStrip = G::kStrip;
  constexpr int H = G::kHalo;
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  unsigned char *wbase = smem + warp * G::kWarpBytes;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + nwarps * G::kWarpBytes) + 2 * warp;
  const int ntiles = args.ctr->ntiles;
  const long long run_base = args.ctr->run_base;
  const int rows = args.rows;

  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();

  // Row items of this warp, in order: tiles blockIdx.x, +gridDim.x, ...; rows
  // y0 + warp*rows + r of each. `find` moves (t, r) to the first valid item at or after it.
  auto find = [&](int &t, int &r) -> bool {
    while (t < ntiles) {
      const TileDev tile = args.tiles[t];
      const DomDyn dy = args.dyn[tile.dom];
      const int ny = args.doms[tile.dom].ny;
      const bool active = dy.step0 + run_base + s < dy.step_end;
      if (active && r < rows && tile.y0 + warp * rows + r < ny) return true;
      t += gridDim.x;
      r = 0;
    }
    return false;
  };

  // Lane 0: issue the bulk copies of item (t, r) into stage st.
  auto issue = [&](int t, int r, int st) {
    const TileDev tile = args.tiles[t];
    const DomDev &D = args.doms[tile.dom];
    const DomDyn dy = args.dyn[tile.dom];
    const int par = (dy.parity + static_cast<int>((run_base + s) & 1)) & 1;
    const E *src = static_cast<const E *>(D.lat[par]);
    const int ny = D.ny, pitch = D.pitch;
    const int j = tile.y0 + warp * rows + r;
    const int x0 = tile.x0;
    const int lo = x0 == 0 ? 0 : x0 - H;
    const int hi = min(x0 + kStrip + H, pitch);
    const uint32_t bytes = static_cast<uint32_t>(hi - lo) * G::kEs;
    const int mhi = min(x0 + kStrip, pitch);
    const uint32_t mbytes = static_cast<uint32_t>(mhi - x0);
    unsigned char *sb = wbase + st * G::kStageBytes;
    mbar_expect_tx(&bar[st], kQ * bytes + mbytes);
    const size_t plane = static_cast<size_t>(ny) * pitch;
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
      const int ey = ey_of(a);
      int sy = j - ey, sa = a;
      if (sy < 0) {
        if (D.south == LBM_FREE_SLIP) { sy = 0; sa = reflect_y(a); }
        else sy += ny;
      } else if (sy > ny - 1) {
        if (D.north == LBM_FREE_SLIP) { sy = ny - 1; sa = reflect_y(a); }
        else sy -= ny;
      }
      const E *row = src + sa * plane + static_cast<size_t>(sy) * pitch;
      E *dst = reinterpret_cast<E *>(sb + a * G::kSegBytes) + (lo - (x0 - H));
      tma_load_1d(dst, row + lo, bytes, &bar[st]);
    }
    tma_load_1d(sb + kQ * G::kSegBytes, D.mask + static_cast<size_t>(j) * pitch + x0, mbytes,
                &bar[st]);
  };

  uint32_t phase = 0u;  // bit st: parity of the next phase of stage st
  int t = blockIdx.x, r = 0;
  bool have = find(t, r);
  if (have && lane == 0) issue(t, r, 0);
  int st = 0;
  int unstable = 0;

  while (have) {
    // prefetch the next item into the other stage
    int tn = t, rn = r + 1;
    const bool have_n = find(tn, rn);
    if (have_n && lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(tn, rn, st ^ 1);
    }
    const TileDev tile = args.tiles[t];
    const DomDev &D = args.doms[tile.dom];
    // bounded wait; the vote keeps the warp's decision uniform. Injected failure (bit 0
    // of args.inject): the wait has completed, then the warp takes the timeout path, so
    // the path runs with no copy of this stage in flight.
    const bool arrived = mbar_wait_bounded(&bar[st], (phase >> st) & 1u);
    if (!__all_sync(0xffffffffu, arrived && !(args.inject & 1))) {
      if (lane == 0) atomicOr(D.status, 2);
      // the other stage's copies (issued above) are awaited, again with a bound. After a
      // real timeout the copies of this stage may still be in flight when the block exits.
      if (have_n) mbar_wait_bounded(&bar[st ^ 1], (phase >> (st ^ 1)) & 1u);
      return;
    }
    phase ^= 1u << st;

    const DomDyn dy = args.dyn[tile.dom];
    const int par = (dy.parity + static_cast<int>((run_base + s) & 1)) & 1;
    const E *__restrict__ src = static_cast<const E *>(D.lat[par]);
    E *__restrict__ dstg = static_cast<E *>(D.lat[par ^ 1]);
    const int nx = D.nx, ny = D.ny, pitch = D.pitch;
    const int j = tile.y0 + warp * rows + r;
    const int x0 = tile.x0;
    const int xl = x0 + lane * V;
    const bool lane_on = xl < nx;
    const bool west_edge = (x0 == 0);
    const bool east_edge = (x0 + kStrip >= nx);
    const bool west_inlet = D.west == LBM_INLET_EQ;
    const bool east_out = D.east == LBM_OUTFLOW_ZG;
    const CellConst<T> &C = cell_const<T>(D);
    const int k_last = nx - 1 - xl;
    const bool has_last = east_edge && k_last >= 0 && k_last < V;
    const size_t plane = static_cast<size_t>(ny) * pitch;
    const unsigned char *sb = wbase + st * G::kStageBytes;

    // row pointers are needed only for the periodic strip ends at the domain edges
    // (side 0 / 1: the west / east linked neighbour's lattice, same lattice index)
    auto edge_row = [&](int a, int side = -1) -> const E * {
      const int ey = ey_of(a);
      int sy = j - ey, sa = a;
      if (sy < 0) {
        if (D.south == LBM_FREE_SLIP) { sy = 0; sa = reflect_y(a); }
        else sy += ny;
      } else if (sy > ny - 1) {
        if (D.north == LBM_FREE_SLIP) { sy = ny - 1; sa = reflect_y(a); }
        else sy -= ny;
      }
      if (side >= 0)
        return static_cast<const E *>(D.nb_lat[side][par]) +
               (static_cast<size_t>(sa) * ny + sy) * D.nb_pitch[side];
      return src + sa * plane + static_cast<size_t>(sy) * pitch;
    };

    Strip<S, V> v[kQ];
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
      const E *seg = reinterpret_cast<const E *>(sb + a * G::kSegBytes);
      if (lane_on) v[a].load_shared(seg + H + lane * V);
      else v[a].zero();
    }
    uint8_t b[V];
    {
      const uint8_t *mseg = sb + kQ * G::kSegBytes + lane * V;
      if constexpr (V == 8) {
        const uint2 mw = lane_on ? *reinterpret_cast<const uint2 *>(mseg) : make_uint2(0u, 0u);
#pragma unroll
        for (int k = 0; k < 4; ++k) b[k] = (mw.x >> (8 * k)) & 0xff;
#pragma unroll
        for (int k = 0; k < 4; ++k) b[4 + k] = (mw.y >> (8 * k)) & 0xff;
      } else if constexpr (V == 4) {
        const uint32_t mw = lane_on ? *reinterpret_cast<const uint32_t *>(mseg) : 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) b[k] = (mw >> (8 * k)) & 0xff;
      } else {
#pragma unroll
        for (int k = 0; k < V; ++k) b[k] = lane_on ? mseg[k] : 0;
      }
    }
#pragma unroll
    for (int a = 0; a < kQ; ++a) {
      const E *seg = reinterpret_cast<const E *>(sb + a * G::kSegBytes);
      const int ex = ex_of(a);
      if (ex == 1) {
        E in = shfl_up1<E>(v[a].last());
        if (lane == 0) {
          if (!west_edge) in = seg[H - 1];
          else if (D.west == LBM_NEIGHBOR) in = __ldg(edge_row(a, 0) + D.nb_nx[0] - 1);  // linked
          else if (!west_inlet) in = __ldg(edge_row(a) + nx - 1);  // periodic
          else in = E(0);  // inlet: replaced by the ghost after decoding
        }
        v[a].shift_up(in);
      } else if (ex == -1) {
        E keep = E(0);
        if (has_last) {
#pragma unroll
          for (int k = 0; k < V; ++k)
            if (k == k_last) keep = v[a].get(k);
        }
        E in = shfl_down1<E>(v[a].first());
        if (lane == 31 && !east_edge) in = seg[H + kStrip];
        v[a].shift_down(in);
        if (has_last) {
          // zero gradient, linked neighbour or periodic
          const E fix = east_out ? keep : __ldg(D.east == LBM_NEIGHBOR ? edge_row(a, 1) : edge_row(a));
#pragma unroll
          for (int k = 0; k < V; ++k)
            if (k == k_last) v[a].set(k, fix);
        }
      }
    }
    // the stage has been read: it may be refilled after the warp has converged
    __syncwarp();

    bool any_solid_lane = false;
#pragma unroll
    for (int k = 0; k < V; ++k) any_solid_lane |= (b[k] != 0);
    const bool any_solid = __any_sync(0xffffffffu, any_solid_lane);
    const unsigned valid_bits =
        east_edge ? (nx - xl >= V ? (1u << V) - 1u : (nx > xl ? (1u << (nx - xl)) - 1u : 0u))
                  : (1u << V) - 1u;
    unsigned bad_bits = 0u;

    auto update = [&](T (&x)[kQ], int k) {
      if (k == 0 && west_edge && west_inlet && lane == 0) {
        x[1] = C.ghost[1];
        x[5] = C.ghost[5];
        x[8] = C.ghost[8];
      }
      NodeMacro<T> m;
      if (any_solid) {
        T uox = T(0), uoy = T(0);
        const bool solid = b[k] != 0;
        if (solid) body_velocity<true>(D, b[k], xl + k, j, uox, uoy);
        m = node_macro<T, SHIFT, true>(x, C, solid, uox, uoy);
        collide<T, SHIFT, true>(x, m, C);
        if (solid) {
          T *fv = static_cast<T *>(D.fvp[par]) + 2 * (static_cast<size_t>(j) * pitch + xl + k);
          fv[0] = m.fx * (T(1) / T(Cd::kScale));  // unscaled (power of two: exact)
          fv[1] = m.fy * (T(1) / T(Cd::kScale));
        }
      } else {
        m = node_macro<T, SHIFT, false>(x, C, false, T(0), T(0));
        collide<T, SHIFT, false>(x, m, C);
      }
      bad_bits |= (fabs(m.rho - T(50.005) * T(Cd::kScale)) < T(49.995) * T(Cd::kScale) ? 0u : 1u) << k;
      return m.d;
    };
    if constexpr (sizeof(E) == 2) {
#pragma unroll
      for (int k = 0; k < V; k += 2) {
        T x0v[kQ], x1v[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) {
          const float2 p = Cd::dec2(v[a].w[k >> 1]);
          x0v[a] = p.x;
          x1v[a] = p.y;
        }
        const float d0 = update(x0v, k);
        const float d1 = update(x1v, k + 1);
        F2 xp[kQ];
#pragma unroll
        for (int a = 0; a < kQ; ++a) xp[a] = F2(make_float2(x0v[a], x1v[a]));
        uint32_t w[kQ];
        encode_pair_mass_kept<S>(xp, F2(make_float2(d0, d1)), sr_pair_bits(sr_group_bits(sr_row_key(dy.step0 + run_base + s, j), xl + D.x0), xl + k + D.x0), w);
#pragma unroll
        for (int a = 0; a < kQ; ++a) v[a].w[k >> 1] = w[a];
      }
    } else {
#pragma unroll
      for (int k = 0; k < V; ++k) {
        T x[kQ];
        decode_cell<S, V>(v, k, x);
        if constexpr (kAddShift) {
#pragma unroll
          for (int a = 0; a < kQ; ++a) x[a] -= shift_of(C, a);  // exact (Sterbenz)
        }
        update(x, k);
        if constexpr (kAddShift) {
#pragma unroll
          for (int a = 0; a < kQ; ++a) x[a] += shift_of(C, a);
        }
#pragma unroll
        for (int a = 0; a < kQ; ++a) v[a].set(k, Cd::enc(x[a]));
      }
    }
    if (bad_bits & valid_bits) unstable = 1;
    if (east_edge) {
#pragma unroll
      for (int k = 0; k < V; ++k)
        if (!((valid_bits >> k) & 1u)) {
#pragma unroll
          for (int a = 0; a < kQ; ++a) v[a].set(k, E(0));
        }
    }
    if (lane_on) {
#pragma unroll
      for (int a = 0; a < kQ; ++a)
        v[a].store(dstg + a * plane + static_cast<size_t>(j) * pitch + xl);
    }
    if (__any_sync(0xffffffffu, unstable)) {
      if (lane == 0) atomicOr(D.status, 1);
      unstable = 0;
    }
    t = tn;
    r = rn;
    have = have_n;
    st ^= 1;
  }
}

template <int S, int V>
cudaError_t launch_sweep_tma_t(int grid, int warps, cudaStream_t st, const SweepArgs &a, int s) {
  const int bytes = tma_smem_bytes<S, V>(warps);
  cudaError_t e = cudaFuncSetAttribute(sweep_tma_kernel<S, V>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  sweep_tma_kernel<S, V><<<grid, warps * 32, bytes, st>>>(a, s);
  return cudaGetLastError();
}

template <int S, int V> int max_blocks_tma_t(int warps) {
  const int bytes = tma_smem_bytes<S, V>(warps);
  if (cudaFuncSetAttribute(sweep_tma_kernel<S, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_tma_kernel<S, V>, warps * 32, bytes) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace lbm
