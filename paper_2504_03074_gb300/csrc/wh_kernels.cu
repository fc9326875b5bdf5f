// wh_kernels.cu -- CUDA kernels of one WaveHoltz iteration on an overset grid (sm_103a).
//
// Per time step (Algorithm 2, Sec. 3.2) the library launches
//   march_kernel      advance every discretization point of every grid (explicit
//                     scheme, Eq. WaveSchemeexplicit) and fold the new level into the
//                     time-filter accumulator (Eq. updateDiscreteExplicit);
//   bc_gather_kernel  ghost-point rules of every physical side, and the overset
//                     interpolation of every receiver (tensor-product Lagrange, Sec. 3.1)
//                     with its filter contribution.
// The two parts of bc_gather_kernel are independent: ghost rules read only
// discretization/Dirichlet points of the new level and donors are never ghosts.
//
// GB300 note: FP64 throughput is ~2 FMA/clk/SM, so these kernels are FP64-ALU bound;
// the weights fold dt^2, c(x)^2 and the "2 W^n" of the leapfrog into one per-point
// stencil so that an order-4 point costs 11 FP64 instructions (9 stencil FMAs, the
// forcing FMA and the filter FMA).
#include <cstdint>

#include "wh_internal.h"
#include "wh_widen.cuh"

namespace wh {

__device__ __forceinline__ int wrap(int i, int n, int per) {
  if (per) {
    i = i < 0 ? i + n : i;
    i = i >= n ? i - n : i;
  }
  return i;
}

// Row offset of row jj in a grid (wrapping on a periodic axis, clamped to the extended
// rows otherwise: clamped rows only feed points that are not stored).
__device__ __forceinline__ int64_t row_off(const DevGrid &G, int jj) {
  jj = wrap(jj, G.n1, G.per1);
  jj = jj < -G.g1 ? -G.g1 : (jj >= G.n1 + G.g1 ? G.n1 + G.g1 - 1 : jj);
  return G.base + (int64_t)(jj + G.g1) * G.pitch + G.g0;
}

// Programmatic dependent launch.  Kernels of the iteration graph start with pdl_wait: the
// previous kernel in the stream has completed and its writes are visible (a no-op when the
// launch did not ask for programmatic serialization).  The next kernel is released as this
// grid's blocks exit (no early trigger: triggering at kernel start, which lets the next
// grids' blocks sit in SM slots while they wait, measured 5-12% slower), which hides the
// launch gap between the graph's kernels (measured +2% FP64, +3% FP32 on the disk workload).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Constant cross weight k and forcing factor of step n in the march precision.  The FP32
// values are rounded once on the host: converting FP64 to FP32 in the kernel is an FP64-pipe
// instruction on this part, several times the cost of a DFMA, and was most of that pipe's
// load in the FP32 march.  Same values as converting here.
template <typename T>
__device__ __forceinline__ T grid_w(const DevGrid &G, int k);
template <>
__device__ __forceinline__ double grid_w<double>(const DevGrid &G, int k) {
  return G.cw[k];
}
template <>
__device__ __forceinline__ float grid_w<float>(const DevGrid &G, int k) {
  return G.cwf[k];
}
template <typename T>
__device__ __forceinline__ T step_fc(const InstDev &I, int n, double fs, bool first);
template <>
__device__ __forceinline__ double step_fc<double>(const InstDev &I, int n, double fs,
                                                  bool first) {
  return first ? 0.5 * fs * I.dt2 : fs * I.fc[n];
}
template <>
__device__ __forceinline__ float step_fc<float>(const InstDev &I, int n, double fs, bool first) {
  return fs == 0.0 ? 0.0f : (first ? I.dt2hf : I.fcf[n]);  // fs is 0 or 1
}

// ---------------------------------------------------------------------------------
// Per-point arithmetic shared by the graph path and the persistent kernel.
// ---------------------------------------------------------------------------------

// A Dirichlet point with boundary data at step n -> n + 1: the filter takes its level-n
// value (like an interpolation point's), and its level n + 1 is the data g cos(omega_e
// t^{n+1}) (fcos1 = that cosine times the forcing switch).
template <typename T>
__device__ __forceinline__ void dirichlet_step(const DevGrid &G, int64_t p, const T *Wn,
                                               T *Wout, double *V, double wf_cur,
                                               double fcos1) {
  V[p] = fma(wf_cur, to_f64(Wn[p]), V[p]);
  Wout[p] = (T)(fcos1 * G.gb[p]);
}

// One time step at point (i, j) of grid G (Eq. WaveSchemeexplicit), fused with the filter:
//   FIRST: W^1 = (sum_k w_k W^0_k)/2 - fc f            (fc = dt^2/2, or 0 without forcing)
//   else : W^{n+1} = sum_k w_k W^n_k - W^{n-1} - fc f   (fc = dt^2 cos(omega_e t^n))
// W^{n+1} is written over W^{n-1} (Wout).  Discretization points: V += wf_new W^{n+1}.
// Interpolation points: V += wf_cur W^n (their level-n values are final when the march
// runs).  The weights fold dt^2, c(x)^2 and the leapfrog "2 W^n" into one stencil, so an
// order-4 point costs 11 FP64 FMAs.
// The state arrays (Wn, Wout, V) are written inside the persistent kernel, so they are
// never declared __restrict__: their loads must not take the non-coherent read-only path.
template <typename T, int ORDER, bool FIRST, bool NOF = false>
__device__ __forceinline__ void march_point(const DevGrid &G, int i, int j,
                                            const int8_t *__restrict__ mask,
                                            const T *Wn, const T *Wprev, T *Wout,
                                            const T *__restrict__ F, const T *__restrict__ Wt,
                                            double *V, T fc, double wf_new, double wf_cur,
                                            double fcos1) {
  constexpr int R = ORDER / 2;
  const int64_t row = row_off(G, j);
  const int64_t p = row + i;
  const int8_t mk = mask[p];
  if (mk == 2) {
    V[p] = fma(wf_cur, to_f64(Wn[p]), V[p]);
    return;
  }
  if (mk == 3) {
    if (G.gb) dirichlet_step(G, p, Wn, Wout, V, wf_cur, fcos1);
    return;
  }
  if (mk != 1) return;
  T a;
  if (G.stencil == kConstCross) {
    const T c0 = grid_w<T>(G, 0), x1 = grid_w<T>(G, 1), y1 = grid_w<T>(G, 3);
    const int64_t up = row_off(G, j + 1) + i, dn = row_off(G, j - 1) + i;
    const int im = wrap(i - 1, G.n0, G.per0), ip = wrap(i + 1, G.n0, G.per0);
    a = FIRST ? c0 * Wn[p] : fma(c0, Wn[p], -Wprev[p]);
    a = fma(x1, Wn[row + im], a);
    a = fma(x1, Wn[row + ip], a);
    a = fma(y1, Wn[dn], a);
    a = fma(y1, Wn[up], a);
    if (ORDER == 4) {
      const T x2 = grid_w<T>(G, 2), y2 = grid_w<T>(G, 4);
      const int64_t up2 = row_off(G, j + 2) + i, dn2 = row_off(G, j - 2) + i;
      const int im2 = wrap(i - 2, G.n0, G.per0), ip2 = wrap(i + 2, G.n0, G.per0);
      a = fma(x2, Wn[row + im2], a);
      a = fma(x2, Wn[row + ip2], a);
      a = fma(y2, Wn[dn2], a);
      a = fma(y2, Wn[up2], a);
    }
  } else if (G.stencil == kPointCross) {
    // planes: centre, axis-0 offsets -R..-1, 1..R, axis-1 offsets -R..-1, 1..R
    const int64_t q = G.wbase + (p - G.base), E = G.ext;
    a = FIRST ? Wt[q] * Wn[p] : fma(Wt[q], Wn[p], -Wprev[p]);
    int pl = 1;
#pragma unroll
    for (int k = -R; k <= R; ++k) {
      if (k == 0) continue;
      a = fma(Wt[q + pl * E], Wn[row + wrap(i + k, G.n0, G.per0)], a);
      ++pl;
    }
#pragma unroll
    for (int k = -R; k <= R; ++k) {
      if (k == 0) continue;
      a = fma(Wt[q + pl * E], Wn[row_off(G, j + k) + i], a);
      ++pl;
    }
  } else {
    // box: plane (b + R) * (2R + 1) + (a + R) holds the weight of offset (a, b)
    const int64_t q = G.wbase + (p - G.base), E = G.ext;
    a = FIRST ? (T)0 : -Wprev[p];
#pragma unroll
    for (int b = -R; b <= R; ++b) {
      const int64_t rb = row_off(G, j + b);
#pragma unroll
      for (int aa = -R; aa <= R; ++aa)
        a = fma(Wt[q + ((b + R) * (2 * R + 1) + (aa + R)) * E], Wn[rb + wrap(i + aa, G.n0, G.per0)],
                a);
    }
  }
  if (FIRST) a *= (T)0.5;
  // NOF: a step with zero forcing (the map S of the Krylov and eigensolver products), where
  // fma(-0, F, a) is a (F is finite by construction): the load and the FMA are left out.
  // A compile-time choice: a run-time test in front of the load keeps it from being issued
  // with the stencil loads (measured 9% slower on the FP64 march with forcing)
  if (!NOF) a = fma(-fc, F[p], a);
  Wout[p] = a;
  V[p] = fma(wf_new, to_f64(a), V[p]);
}

// Ghost rule of one boundary point (ghost-point rules for g = 0; see the library notes):
//   type 0, Neumann order 2: D0 W = 0 -> G1 = U1;
//   type 1, Neumann order 4: 8(U1 - G1) - (U2 - G2) = 0 and D+^5 G2 = 0;
//   type 2, Dirichlet order 4: c^2 (a_nn D_nn + b_n D_n) W_b = f_b cos(omega_e t) and
//   D+^5 G2 = 0, solved as G1 = (F - A2(-30U0 + 16U1 - U2) - B1(8U1 - U2) + (A2 - B1) E) /
//   (11 A2 - 3 B1), G2 = 5 G1 + E with E = -10U0 + 10U1 - 5U2 + U3.
// Load of a state value: through L1, or (CG) from L2 only, for values another SM wrote
// during the same launch.
template <bool CG, typename T>
__device__ __forceinline__ T ld_state(const T *p) {
  if (CG) return __ldcg(p);
  return *p;
}

template <typename T, bool CG = false>
__device__ __forceinline__ void bc_item(const BcItem &it, T *W, const T *__restrict__ F,
                                        double fcos) {
  const double U0 = to_f64(ld_state<CG>(W + it.u[0])), U1 = to_f64(ld_state<CG>(W + it.u[1]));
  if (it.type == 0) {
    W[it.g[0]] = (T)U1;
    return;
  }
  const double U2 = to_f64(ld_state<CG>(W + it.u[2])), U3 = to_f64(ld_state<CG>(W + it.u[3]));
  const double E = -10.0 * U0 + 10.0 * U1 - 5.0 * U2 + U3;
  double G1;
  if (it.type == 1) {
    G1 = (18.0 * U1 - 10.0 * U0 - 6.0 * U2 + U3) * (1.0 / 3.0);
  } else {
    const double Fb = (to_f64(F[it.u[0]]) + it.fg) * fcos;
    G1 = (Fb - it.A2 * (-30.0 * U0 + 16.0 * U1 - U2) - it.B1 * (8.0 * U1 - U2) +
          (it.A2 - it.B1) * E) * it.inv;
  }
  W[it.g[0]] = (T)G1;
  W[it.g[1]] = (T)(5.0 * G1 + E);
}

// Warp-cooperative gather of receiver r: LANES lanes split its (p+1)^2 donors and combine
// their partial sums with xor shuffles.  Every lane of the warp must call this (live may be
// false); lane 0 of the group stores the value.
template <typename T, int ORDER, bool CG = false>
__device__ __forceinline__ void gather_group(int r, int lane, bool live,
                                             const int32_t *__restrict__ didx,
                                             const double *__restrict__ dw,
                                             const int64_t *__restrict__ ridx, T *W) {
  constexpr int ND = (ORDER + 1) * (ORDER + 1);
  constexpr int LANES = ORDER == 4 ? 8 : 4;
  double s = 0.0;
  if (live) {
    const int32_t *di = didx + (int64_t)r * ND;
    const double *wi = dw + (int64_t)r * ND;
#pragma unroll
    for (int d = lane; d < ND; d += LANES) s = fma(wi[d], to_f64(ld_state<CG>(W + di[d])), s);
  }
#pragma unroll
  for (int off = LANES / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off, LANES);
  if (live && lane == 0) W[ridx[r]] = (T)s;
}

// ---------------------------------------------------------------------------------
// Graph path: one launch per phase.
// ---------------------------------------------------------------------------------
// Step n of every active instance with n < M (FIRST: n = 0).
// Work unit u of the ghost rules (units [0, bc_blocks): 256 items each) and interpolation
// (the remaining units: 256 / lanes receivers each) at one level; tid in [0, 256).
template <typename T, int ORDER, bool CG>
__device__ __forceinline__ void gather_unit(int u, int tid, const BcItem *__restrict__ bc,
                                            int nbc, int bc_blocks,
                                            const int32_t *__restrict__ didx,
                                            const double *__restrict__ dw,
                                            const int64_t *__restrict__ ridx,
                                            const int32_t *__restrict__ rinst, int nrecv, T *W,
                                            const T *__restrict__ F,
                                            const InstDev *__restrict__ inst, int level,
                                            double fs) {
  if (u < bc_blocks) {
    const int k = u * 256 + tid;
    if (k >= nbc) return;
    const BcItem it = bc[k];
    const InstDev &I = inst[it.inst];
    if (I.active && level <= I.M) bc_item<T, CG>(it, W, F, fs * I.cosn[level]);
    return;
  }
  constexpr int LANES = ORDER == 4 ? 8 : 4;
  const int r = ((u - bc_blocks) * 256 + tid) / LANES;
  bool live = r < nrecv;
  if (live) {
    const InstDev &I = inst[rinst[r]];
    live = I.active && level <= I.M;
  }
  gather_group<T, ORDER, CG>(r, tid % LANES, live, didx, dw, ridx, W);
}

// Five resident blocks per SM (registers capped at 48, a few spilled): the FP64 march is
// FP64-pipe bound but stalls on memory latency, and the fifth block hides more of it than
// the spills cost (disk workload +7%; six blocks measured slower there).
template <typename T, int ORDER, bool FIRST, bool NOF = false>
__global__ void __launch_bounds__(kTileX *kTileY, 5)
    march_kernel(const DevGrid *__restrict__ grids, const Tile *__restrict__ tiles, int ntiles,
                 const int8_t *__restrict__ mask, const T *Wn, const T *Wprev, T *Wout,
                 const T *__restrict__ F, const T *__restrict__ Wt, double *V,
                 const InstDev *__restrict__ inst, int n, double fs, GatherArgs ga) {
  pdl_wait();
  const int tid = (int)threadIdx.y * kTileX + (int)threadIdx.x;
  // tiles by ticket when ga.ctl is set (the next ticket is fetched while a tile is computed,
  // and blocks that finish early take more tiles), else by grid stride
  __shared__ int s_tile;
  if (ga.ctl && tid == 0) s_tile = atomicAdd(&ga.ctl[1], 1);
  __syncthreads();
  int tile = ga.ctl ? s_tile : (int)blockIdx.x;
  __syncthreads();
  while (tile < ntiles) {
    if (ga.ctl && tid == 0) s_tile = atomicAdd(&ga.ctl[1], 1);
    const Tile t = tiles[tile];
    const DevGrid &G = grids[t.grid];
    const InstDev &I = inst[G.inst];
    const int i = t.i0 + (int)threadIdx.x;
    if (I.active && n < I.M && i < G.n0) {
      const T fc = step_fc<T>(I, n, fs, FIRST);
      const double wf_new = I.wf[n + 1], wf_cur = I.wf[n];
      const double fcos1 = fs * I.cosn[n + 1];
      if (sizeof(T) == 4 && G.stencil == kConstCross && !G.per0 && !G.per1) {
        // FP32 march, constant weights, no wrap: the ghost layers (width order/2) hold every
        // neighbour, so neighbour addresses are fixed offsets from the point (same
        // arithmetic, in the same order, as march_point).  Measured on the disk workload:
        // +20% for the latency-bound FP32 march, -5% for the ALU-bound FP64 march, which
        // keeps march_point.
        const int64_t pitch = G.pitch, n1 = G.n1;
        const int64_t b0 = G.base + (int64_t)G.g1 * pitch + G.g0 + i;
        const T c0 = grid_w<T>(G, 0), x1 = grid_w<T>(G, 1), x2 = grid_w<T>(G, 2);
        const T y1 = grid_w<T>(G, 3), y2 = grid_w<T>(G, 4);
#pragma unroll
        for (int m = 0; m < kPY; ++m) {
          const int j = t.j0 + (int)threadIdx.y + m * kTileY;
          if (j >= n1) continue;
          const int64_t p = b0 + j * pitch;
          const int8_t mk = mask[p];
          if (mk == 2) {
            V[p] = fma(wf_cur, to_f64(Wn[p]), V[p]);
            continue;
          }
          if (mk == 3) {
            if (G.gb) dirichlet_step(G, p, Wn, Wout, V, wf_cur, fcos1);
            continue;
          }
          if (mk != 1) continue;
          T a = FIRST ? c0 * Wn[p] : fma(c0, Wn[p], -Wprev[p]);
          a = fma(x1, Wn[p - 1], a);
          a = fma(x1, Wn[p + 1], a);
          a = fma(y1, Wn[p - pitch], a);
          a = fma(y1, Wn[p + pitch], a);
          if (ORDER == 4) {
            a = fma(x2, Wn[p - 2], a);
            a = fma(x2, Wn[p + 2], a);
            a = fma(y2, Wn[p - 2 * pitch], a);
            a = fma(y2, Wn[p + 2 * pitch], a);
          }
          if (FIRST) a *= (T)0.5;
          if (!NOF) a = fma(-fc, F[p], a);
          Wout[p] = a;
          V[p] = fma(wf_new, to_f64(a), V[p]);
        }
      } else {
#pragma unroll
        for (int m = 0; m < kPY; ++m) {
          const int j = t.j0 + (int)threadIdx.y + m * kTileY;
          if (j < G.n1)
            march_point<T, ORDER, FIRST, NOF>(G, i, j, mask, Wn, Wprev, Wout, F, Wt, V, fc,
                                              wf_new, wf_cur, fcos1);
        }
      }
    }
    if (ga.nunits && t.pad_) {  // a gather unit reads this tile's level n + 1: signal it
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        atomicExch(&ga.tile_done[tile], n + 1);
      }
    }
    if (ga.ctl) {
      __syncthreads();
      tile = s_tile;
      __syncthreads();
    } else {
      tile += gridDim.x;
    }
  }
  if (ga.ctl && tid == 0 && atomicAdd(&ga.ctl[2], 1) == (int)gridDim.x - 1) {
    atomicExch(&ga.ctl[1], 0);  // last block out: tickets start at zero in the next launch
    atomicExch(&ga.ctl[2], 0);
  }
  // The folded ghost rules and interpolation of level n + 1 (the graph path passes no tile
  // tickets with them): unit u on block nb - 1 - u (the blocks with the fewest march
  // tiles), after its source tiles have signalled.  Blocks only wait here, after their own
  // march tiles, and the grid is one resident wave, so every awaited tile is computed; each
  // wait is bounded all the same.  (Tiles and units both by ticket measured -25%.)
  __shared__ int s_fail;
  for (int u = (int)gridDim.x - 1 - (int)blockIdx.x; u < ga.nunits; u += gridDim.x) {
    if (tid == 0) s_fail = 0;
    __syncthreads();
    for (int64_t e = ga.udep_off[u] + tid; e < ga.udep_off[u + 1]; e += kTileX * kTileY) {
      volatile int *flag = (volatile int *)&ga.tile_done[ga.udep_tile[e]];
      unsigned long long it = 0;
      while (*flag < n + 1) {
        if (++it > ga.spin_limit) {
          atomicExch(ga.err, 1);
          s_fail = 1;
          break;
        }
        if (it > 64) __nanosleep(32);
      }
      __threadfence();
    }
    __syncthreads();
    if (s_fail) return;
    gather_unit<T, ORDER, true>(u, tid, ga.bc, ga.nbc, ga.bc_blocks, ga.didx, ga.dw, ga.ridx,
                                ga.rinst, ga.nrecv, Wout, F, inst, n + 1, fs);
  }
}

// ---------------------------------------------------------------------------------
// TMA-staged march.  A block of the fast role walks its share of the fast tiles with two
// shared-memory stages: while it computes tile k from one stage, the five boxes of tile k+1
// (W^n with halo, W^{n-1}, F, V, mask) arrive in the other through cp.async.bulk.tensor on
// that stage's mbarrier.  Out-of-range box parts are zero-filled and only feed points that
// are not computed.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// Shared-memory stages of the TMA-staged march: tiles prefetched while one is computed.
constexpr int kTmaStages = 2;

// Byte layout of one stage (every box 128-byte aligned).
template <typename T, int ORDER>
struct TmaStage {
  static constexpr int HY = kTileY * kPY + ORDER;  // tile rows + halo 2 x order/2
  static constexpr int kWnBytes = kBoxX * HY * (int)sizeof(T);
  static constexpr int kCtrBytes = kBoxX * kTileY * kPY * (int)sizeof(T);
  static constexpr int kVBytes = kBoxX * kTileY * kPY * 8;
  static constexpr int kMBytes = kMaskBoxX * kTileY * kPY;
  static constexpr int kWn = 0;
  static constexpr int kWp = (kWnBytes + 127) / 128 * 128;
  static constexpr int kF = kWp + (kCtrBytes + 127) / 128 * 128;
  static constexpr int kV = kF + (kCtrBytes + 127) / 128 * 128;
  static constexpr int kM = kV + (kVBytes + 127) / 128 * 128;
  static constexpr int kBytes = kM + (kMBytes + 127) / 128 * 128;
  static constexpr uint32_t kTx = kWnBytes + 2 * kCtrBytes + kVBytes + kMBytes;
  static constexpr size_t kSmem =
      kTmaStages * (size_t)kBytes + 128 + 8 * kTmaStages;  // + alignment, the mbarriers
};

// Per-tile scalars of the TMA-staged march, read one tile ahead by the issuing thread.
template <typename T>
struct TmaTileInfo {
  int64_t p0;     // state index of the tile's first point (grid point (i0, j0))
  int64_t pitch;
  double wf_new, wf_cur;
  T fc, c0, x1, x2, y1, y2;
  int ni, nj;     // points of the tile inside the grid (ragged edges)
  int live;       // 0: the tile's instance is past its M or switched off
  const double *gb;  // the grid's Dirichlet data (or null) and its factor at t^{n+1}
  double fcos1;
};

// Every block first walks its strided share of the fast tiles (blockIdx.x, + gridDim.x, ...;
// the next tile is known, so its copies and its scalars are fetched while the current one is
// computed), then takes general tiles by ticket, so blocks that finish early absorb the
// costlier tiles.  ctl[0]: sticky error flag; ctl[1]: next general ticket; ctl[2]: blocks
// done (the last one resets ctl[1] and ctl[2] for the next launch).
template <typename T, int ORDER, bool FIRST>
__global__ void __launch_bounds__(kTileX *kTileY)
    march_tma_kernel(const DevGrid *__restrict__ grids, const Tile *__restrict__ ftiles,
                     int nfast, const CUtensorMap *__restrict__ maps,
                     const Tile *__restrict__ gtiles, int ngen, const int8_t *__restrict__ mask,
                     T *Wa, T *Wb, const T *__restrict__ F, const T *__restrict__ Wt, double *V,
                     const InstDev *__restrict__ inst, int n, double fs, int *ctl,
                     unsigned long long spin_limit, GatherArgs ga) {
  using S = TmaStage<T, ORDER>;
  constexpr int R = ORDER / 2;
  pdl_wait();
  const T *Wn = (n & 1) ? Wb : Wa;
  T *Wout = (n & 1) ? Wa : Wb;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  uint64_t *bar = (uint64_t *)(sm + kTmaStages * S::kBytes);
  __shared__ int s_next, s_fail;
  __shared__ TmaTileInfo<T> s_info[kTmaStages];
  const int tid = threadIdx.y * kTileX + threadIdx.x;
  const int nb = (int)gridDim.x;
  const int nmy = nfast > (int)blockIdx.x ? (nfast - 1 - (int)blockIdx.x) / nb + 1 : 0;
  // thread 0: fetch the scalars of this block's k-th fast tile and start its copies, both
  // into stage k % kTmaStages
  auto issue = [&](int k) {
    const int stage = k % kTmaStages;
    const Tile t = ftiles[blockIdx.x + k * nb];
    const DevGrid &G = grids[t.grid];
    const InstDev &I = inst[G.inst];
    TmaTileInfo<T> &f = s_info[stage];
    f.live = I.active && n < I.M;
    if (!f.live) {
      mbar_arrive_tx(&bar[stage], 0);  // nothing to copy: completes the phase
      return;
    }
    f.pitch = G.pitch;
    f.p0 = G.base + (int64_t)(t.j0 + R) * G.pitch + (t.i0 + R);
    f.wf_new = I.wf[n + 1];
    f.wf_cur = I.wf[n];
    f.fc = step_fc<T>(I, n, fs, FIRST);
    f.gb = G.gb;
    f.fcos1 = fs * I.cosn[n + 1];
    f.c0 = grid_w<T>(G, 0);
    f.x1 = grid_w<T>(G, 1);
    f.x2 = grid_w<T>(G, 2);
    f.y1 = grid_w<T>(G, 3);
    f.y2 = grid_w<T>(G, 4);
    f.ni = min(kTileX, G.n0 - t.i0);
    f.nj = min(kTileY * kPY, G.n1 - t.j0);
    unsigned char *st = sm + stage * S::kBytes;
    const CUtensorMap *mp = maps + (int64_t)t.pad_ * kMapsPerGrid;
    const int x = t.i0, yh = t.j0, yc = t.j0 + R;  // extended coordinates (ghost width R)
    fence_proxy_async_smem();  // the stage's earlier generic reads precede the new copies
    mbar_arrive_tx(&bar[stage], S::kTx);
    tma_load_2d(st + S::kWn, mp + ((n & 1) ? kMapWbHalo : kMapWaHalo), x, yh, &bar[stage]);
    tma_load_2d(st + S::kWp, mp + ((n & 1) ? kMapWaCtr : kMapWbCtr), x, yc, &bar[stage]);
    tma_load_2d(st + S::kF, mp + kMapF, x, yc, &bar[stage]);
    tma_load_2d(st + S::kV, mp + kMapV, x, yc, &bar[stage]);
    tma_load_2d(st + S::kM, mp + kMapMask, x, yc, &bar[stage]);
  };
  if (tid == 0) {
    for (int q = 0; q < kTmaStages; ++q) mbar_init(&bar[q], 1);
    mbar_init_fence();
    s_fail = 0;
    for (int q = 0; q < kTmaStages - 1 && q < nmy; ++q) issue(q);
  }
  __syncthreads();
  for (int k = 0; k < nmy; ++k) {
    const int stage = k % kTmaStages;
    // refill the stage read in iteration k - 1
    if (tid == 0 && k + kTmaStages - 1 < nmy) issue(k + kTmaStages - 1);
    unsigned long long it = 0;
    while (!mbar_try_wait(&bar[stage], (uint32_t)((k / kTmaStages) & 1))) {
      if (++it > spin_limit) {
        s_fail = 1;
        break;
      }
    }
    __syncthreads();
    if (s_fail) {
      // let the copies still in flight land before the block (and its shared memory) goes:
      // this drain is bounded on its own scale (about a second), not by the caller's spin
      // limit, which may be set tiny to provoke the timeout; then report and leave
      if (tid == 0) {
        atomicExch(&ctl[0], 1);
        for (int q = k; q < k + kTmaStages && q < nmy; ++q) {
          unsigned long long w = 0;
          while (!mbar_try_wait(&bar[q % kTmaStages], (uint32_t)((q / kTmaStages) & 1)) &&
                 ++w < (1ull << 22))
            __nanosleep(256);
        }
      }
      return;
    }
    const TmaTileInfo<T> &f = s_info[stage];
    const int li = (int)threadIdx.x;
    if (f.live && li < f.ni) {
      const unsigned char *st = sm + stage * S::kBytes;
      const T *sWn = (const T *)(st + S::kWn);
      const T *sWp = (const T *)(st + S::kWp);
      const T *sF = (const T *)(st + S::kF);
      const double *sV = (const double *)(st + S::kV);
      const int8_t *sM = (const int8_t *)(st + S::kM);
      const T fc = f.fc, c0 = f.c0, x1 = f.x1, x2 = f.x2, y1 = f.y1, y2 = f.y2;
      const double wf_new = f.wf_new, wf_cur = f.wf_cur;
      const int64_t pitch = f.pitch, p0 = f.p0 + li;
      const int c = li + R;  // box column of the thread's grid column
#pragma unroll
      for (int m = 0; m < kPY; ++m) {
        const int lj = (int)threadIdx.y + m * kTileY;
        if (lj >= f.nj) continue;
        const int8_t mk = sM[lj * kMaskBoxX + c];
        const int64_t p = p0 + (int64_t)lj * pitch;
        const T *w = sWn + (lj + R) * kBoxX + c;
        const int q = lj * kBoxX + c;
        if (mk == 2) {
          V[p] = fma(wf_cur, to_f64(w[0]), sV[q]);
          continue;
        }
        if (mk == 3) {
          if (f.gb) {
            V[p] = fma(wf_cur, to_f64(w[0]), sV[q]);
            Wout[p] = (T)(f.fcos1 * f.gb[p]);
          }
          continue;
        }
        if (mk != 1) continue;
        T a = FIRST ? c0 * w[0] : fma(c0, w[0], -sWp[q]);
        a = fma(x1, w[-1], a);
        a = fma(x1, w[1], a);
        a = fma(y1, w[-kBoxX], a);
        a = fma(y1, w[kBoxX], a);
        if (ORDER == 4) {
          a = fma(x2, w[-2], a);
          a = fma(x2, w[2], a);
          a = fma(y2, w[-2 * kBoxX], a);
          a = fma(y2, w[2 * kBoxX], a);
        }
        if (FIRST) a *= (T)0.5;
        a = fma(-fc, sF[q], a);
        Wout[p] = a;
        V[p] = fma(wf_new, to_f64(a), sV[q]);
      }
    }
    __syncthreads();  // this stage is read; it is refilled by the issue of iteration k + 1
    if (ga.nunits && tid == 0) {  // fast tile blockIdx + k nb has written level n + 1
      __threadfence();
      atomicAdd(&ga.tile_done[blockIdx.x + k * nb], 1);
    }
  }
  // general tiles by ticket, exactly as march_kernel.  When they are few next to the blocks
  // (one annulus beside a large background), a ticket is a quarter tile (8 rows, one point
  // per thread): their points' memory round trips then run in parallel blocks instead of
  // one after another in the same threads (measured +17% on the disk workload in FP32; with
  // many general tiles whole tiles are better).
  const int gsplit = ngen * kPY <= 2 * nb ? kPY : 1;
  while (true) {
    if (tid == 0) s_next = atomicAdd(&ctl[1], 1);
    __syncthreads();
    const int g = s_next;
    __syncthreads();
    if (g >= gsplit * ngen) break;
    const Tile t = gtiles[g / gsplit];
    const int m0 = gsplit == 1 ? 0 : g % gsplit, m1 = gsplit == 1 ? kPY : m0 + 1;
    const DevGrid &G = grids[t.grid];
    const InstDev &I = inst[G.inst];
    const int i = t.i0 + (int)threadIdx.x;
    if (I.active && n < I.M && i < G.n0) {
      const T fc = step_fc<T>(I, n, fs, FIRST);
      const double wf_new = I.wf[n + 1], wf_cur = I.wf[n];
      for (int m = m0; m < m1; ++m) {
        const int j = t.j0 + (int)threadIdx.y + m * kTileY;
        if (j < G.n1)
          march_point<T, ORDER, FIRST>(G, i, j, mask, Wn, Wout, Wout, F, Wt, V, fc, wf_new,
                                       wf_cur, fs * I.cosn[n + 1]);
      }
    }
    if (ga.nunits) {  // one of the general tile's gsplit parts has written level n + 1
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        atomicAdd(&ga.tile_done[nfast + g / gsplit], 1);
      }
    }
  }
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&ctl[2], 1) == nb - 1) {  // last block out: reset the tickets
      atomicExch(&ctl[1], 0);
      atomicExch(&ctl[2], 0);
    }
  }
  if (!ga.nunits) return;
  // Level n + 1's ghost rules and interpolation folded in, as in march_kernel: unit u on
  // block nb - 1 - u after its tiles.  Tile flags count the parts written in this iteration
  // (one per step for a fast tile, gsplit per step for a general one), so a source tile t
  // has written level n + 1 once its flag reaches parts(t) (n + 1).
  for (int u = nb - 1 - (int)blockIdx.x; u < ga.nunits; u += nb) {
    if (tid == 0) s_fail = 0;
    __syncthreads();
    for (int64_t e = ga.udep_off[u] + tid; e < ga.udep_off[u + 1]; e += kTileX * kTileY) {
      const int dt = ga.udep_tile[e];
      const int need = (dt < nfast ? 1 : gsplit) * (n + 1);
      volatile int *flag = (volatile int *)&ga.tile_done[dt];
      unsigned long long it = 0;
      while (*flag < need) {
        if (++it > ga.spin_limit) {
          atomicExch(ga.err, 1);
          s_fail = 1;
          break;
        }
        if (it > 64) __nanosleep(32);
      }
      __threadfence();
    }
    __syncthreads();
    if (s_fail) return;
    gather_unit<T, ORDER, true>(u, tid, ga.bc, ga.nbc, ga.bc_blocks, ga.didx, ga.dw, ga.ridx,
                                ga.rinst, ga.nrecv, Wout, F, inst, n + 1, fs);
  }
}

// Ghost rules (blocks [0, bc_blocks)) and interpolation (the remaining blocks) of one
// time level W.  The two are independent: ghost rules read only discretization/Dirichlet
// points and donors are never ghosts or receivers.
// Level `level` of every active instance with level <= M.
template <typename T, int ORDER>
__global__ void __launch_bounds__(256)
    bc_gather_kernel(const BcItem *__restrict__ bc, int nbc, int bc_blocks,
                     const int32_t *__restrict__ didx, const double *__restrict__ dw,
                     const int64_t *__restrict__ ridx, const int32_t *__restrict__ rinst,
                     int nrecv, T *W, const T *__restrict__ F,
                     const InstDev *__restrict__ inst, int level, double fs) {
  pdl_wait();
  gather_unit<T, ORDER, false>((int)blockIdx.x, (int)threadIdx.x, bc, nbc, bc_blocks, didx, dw,
                               ridx, rinst, nrecv, W, F, inst, level, fs);
}

// W^0 = v on discretization and interpolation points, 0 elsewhere (ghosts included);
// V = w_0 W^0 on discretization points, 0 elsewhere.  One thread per extended point.
template <typename T>
__device__ __forceinline__ void init_point(const DevGrid *__restrict__ grids, int ngrids,
                                           const int8_t *__restrict__ mask,
                                           const double *v, T *W0, double *V,
                                           int64_t p, const InstDev *__restrict__ inst,
                                           double fs) {
  int g = 0;
  while (g + 1 < ngrids && p >= grids[g + 1].base) ++g;
  const DevGrid &G = grids[g];
  const InstDev &I = inst[G.inst];
  if (!I.active) return;
  const double w0 = I.wf[0];
  const int64_t o = p - G.base;
  const int j = (int)(o / G.pitch) - G.g1;
  const int i = (int)(o % G.pitch) - G.g0;
  const int8_t m = mask[p];
  double val = 0.0;
  if ((m == 1 || m == 2) && i >= 0 && i < G.n0 && j >= 0 && j < G.n1)
    val = v[G.cbase + (int64_t)j * G.n0 + i];
  else if (m == 3 && G.gb)  // Dirichlet data at t = 0
    val = fs * G.gb[p];
  W0[p] = (T)val;
  V[p] = m == 1 ? w0 * (double)(T)val : 0.0;
}

template <typename T>
__global__ void init_kernel(const DevGrid *__restrict__ grids, int ngrids,
                            const int8_t *__restrict__ mask, const double *__restrict__ v,
                            T *W0, double *V, int64_t total, const InstDev *__restrict__ inst,
                            double fs) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < total) init_point<T>(grids, ngrids, mask, v, W0, V, p, inst, fs);
}

// v_out (compact) = V at active points, 0 at unused points; interpolation points first
// receive the filter contribution wf_M W^M of their instance's last level M (in Wa when
// M is even).  Inactive instances leave v_out untouched.
template <typename T>
__device__ __forceinline__ void finish_point(const DevGrid *__restrict__ grids, int ngrids,
                                             const int8_t *__restrict__ mask, const double *V,
                                             const T *Wa, const T *Wb,
                                             const InstDev *__restrict__ inst, double *vout,
                                             int64_t c) {
  int g = 0;
  while (g + 1 < ngrids && c >= grids[g + 1].cbase) ++g;
  const DevGrid &G = grids[g];
  const InstDev &I = inst[G.inst];
  if (!I.active) return;
  const int64_t o = c - G.cbase;
  const int j = (int)(o / G.n0), i = (int)(o % G.n0);
  const int64_t p = G.base + (int64_t)(j + G.g1) * G.pitch + (i + G.g0);
  const int8_t m = mask[p];
  const T *WM = (I.M % 2 == 0) ? Wa : Wb;
  const bool last = m == 2 || (m == 3 && G.gb);  // their level M is not in V yet
  vout[c] = last ? fma(I.wf[I.M], to_f64(WM[p]), V[p]) : (m != 0 ? V[p] : 0.0);
}

template <typename T>
__global__ void finish_kernel(const DevGrid *__restrict__ grids, int ngrids,
                              const int8_t *__restrict__ mask, const double *__restrict__ V,
                              const T *Wa, const T *Wb, const InstDev *__restrict__ inst,
                              double *vout, int64_t ncompact) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncompact) finish_point<T>(grids, ngrids, mask, V, Wa, Wb, inst, vout, c);
}

// ---------------------------------------------------------------------------------
// Persistent path: one cooperative launch runs a whole WaveHoltz iteration -- init, the
// t = 0 ghost rules and interpolation, M steps of (march | grid barrier | ghost rules +
// interpolation | grid barrier), and the output -- so that no step pays a kernel launch,
// ramp-up or tail.  All blocks are co-resident (cooperative launch).  The grid barrier
// spins a bounded number of times; on timeout it records an error and every block leaves
// the kernel, and the host returns WH_ERR_TIMEOUT.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ bool grid_sync(GridBarrier *b, unsigned nblocks,
                                          unsigned long long spin_limit) {
  // one arrival counter and a generation word; the last arriver resets the counter and
  // advances the generation, the others poll it (bounded)
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    volatile unsigned *vgen = &b->gen[0];
    volatile int *verr = &b->err[0];
    const unsigned g = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&b->count[0], 1u) == nblocks - 1) {
      b->count[0] = 0;
      __threadfence();
      atomicAdd(&b->gen[0], 1u);
    } else {
      unsigned long long it = 0;
      while (*vgen == g) {
        if (*verr) {
          ok = 0;
          break;
        }
        if (++it > spin_limit) {
          atomicExch(&b->err[0], 1);
          ok = 0;
          break;
        }
        if (it > 4096) __nanosleep(32);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Value of ghost G1 (which = 0) or G2 (which = 1) of a ghost-rule item at one level.
template <typename T>
__device__ __forceinline__ double bc_value(const BcItem &it, const T *W, const T *__restrict__ F,
                                           double fcos, int which) {
  const double U0 = to_f64(W[it.u[0]]), U1 = to_f64(W[it.u[1]]);
  if (it.type == 0) return U1;
  const double U2 = to_f64(W[it.u[2]]), U3 = to_f64(W[it.u[3]]);
  const double E = -10.0 * U0 + 10.0 * U1 - 5.0 * U2 + U3;
  double G1;
  if (it.type == 1) {
    G1 = (18.0 * U1 - 10.0 * U0 - 6.0 * U2 + U3) * (1.0 / 3.0);
  } else {
    const double Fb = (to_f64(F[it.u[0]]) + it.fg) * fcos;
    G1 = (Fb - it.A2 * (-30.0 * U0 + 16.0 * U1 - U2) - it.B1 * (8.0 * U1 - U2) +
          (it.A2 - it.B1) * E) * it.inv;
  }
  return which == 0 ? G1 : 5.0 * G1 + E;
}

// Level value of receiver r from its donors (one thread, all donors).
template <typename T, int ORDER>
__device__ __forceinline__ double recv_value(int64_t r, const int32_t *__restrict__ didx,
                                             const double *__restrict__ dw, const T *W) {
  constexpr int ND = (ORDER + 1) * (ORDER + 1);
  const int32_t *di = didx + r * ND;
  const double *wi = dw + r * ND;
  double s = 0.0;
#pragma unroll
  for (int d = 0; d < ND; ++d) s = fma(wi[d], to_f64(W[di[d]]), s);
  return s;
}

// One WaveHoltz iteration in one cooperative launch, one grid barrier per time step.
// Step n of a 32 x 32 tile: stage W^n of the tile and its halo in shared memory; patch the
// halo and tile positions that are ghost points or receivers with their level-n values
// (ghost rules from the boundary columns, receivers from their donors -- all final after
// the previous barrier); then advance the tile's discretization points from shared memory
// and add the receivers' level-n filter contribution.  Receiver and ghost values never go
// back to global memory: every tile computes the ones its stencils read.
template <typename T, int ORDER>
__global__ void __launch_bounds__(kTileX *kTileY)
    iteration_kernel(IterArgs A, const double *__restrict__ v_in, double *v_out,
                     GridBarrier *bar) {
  constexpr int R = ORDER / 2;
  constexpr int SX = kTileX + 2 * R;          // 36 (order 4)
  constexpr int SY = kTileY * kPY + 2 * R;    // 36
  __shared__ T sw[SY][SX];
  const unsigned nb = gridDim.x;
  const int tid = threadIdx.y * kTileX + threadIdx.x;
  const int64_t gtid = (int64_t)blockIdx.x * (kTileX * kTileY) + tid;
  const int64_t nthreads = (int64_t)nb * (kTileX * kTileY);
  const T *F = (const T *)A.F;
  const T *Wt = (const T *)A.Wt;
  T *Wa = (T *)A.Wa, *Wb = (T *)A.Wb;
  const int M = A.M;
  // init: W^0 = v, V = w_0 W^0 (receivers' V accumulates from the first step on); no tile
  // has completed a step
  for (int64_t p = gtid; p < A.total; p += nthreads)
    init_point<T>(A.grids, A.ngrids, A.mask, v_in, Wa, A.V, p, A.inst, A.fs);
  for (int64_t t = gtid; t < A.ntiles; t += nthreads) A.tile_done[t] = 0;
  if (!grid_sync(bar, nb, A.spin_limit)) return;
  // Dataflow over tickets k = n * ntiles + tile, handed out in increasing order.  Ticket
  // (n, tile) waits until every tile it depends on has completed step n - 1 (its level-n
  // values are written); those are lower tickets, so the lowest ticket in progress never
  // waits on an unfinished one and, with every block resident (cooperative launch), the
  // loop cannot deadlock.  Each wait is bounded all the same.
  __shared__ int s_fail;
  const unsigned long long nticket = (unsigned long long)M * (unsigned long long)A.ntiles;
  unsigned long long *ctr = &bar->ticket[0];
  __shared__ unsigned long long s_tk;
  if (tid == 0) {
    s_tk = atomicAdd(ctr, 1ull);
    s_fail = 0;
  }
  __syncthreads();
  unsigned long long tk = s_tk;
  __syncthreads();
  while (tk < nticket) {
    if (tid == 0) s_tk = atomicAdd(ctr, 1ull);  // next ticket, in flight during this tile
    const int n = (int)(tk / (unsigned long long)A.ntiles);
    const int tile = (int)(tk % (unsigned long long)A.ntiles);
    T *cur = (n & 1) ? Wb : Wa;
    T *oth = (n & 1) ? Wa : Wb;
    {
      const Tile t = A.tiles[tile];
      const DevGrid &G = A.grids[t.grid];
      const InstDev &I = A.inst[G.inst];
      if (!I.active || n >= I.M) {
        // block-uniform: nothing to compute and nothing to signal.  The flag is left alone:
        // every tile that reads this one belongs to the same instance and skips this step
        // too, and a skip that raised it could overtake this tile's last real step, still
        // running in another block.
        __syncthreads();
        tk = s_tk;
        __syncthreads();
        continue;
      }
      // wait for the level-n values this tile reads (one thread per dependency)
      for (int64_t e = A.dep_off[tile] + tid; e < A.dep_off[tile + 1]; e += kTileX * kTileY) {
        volatile int *flag = (volatile int *)&A.tile_done[A.dep_tile[e]];
        volatile int *verr = &bar->err[0];
        unsigned long long it = 0;
        while (*flag < n) {
          if (*verr) {
            s_fail = 1;
            break;
          }
          if (++it > A.spin_limit) {
            atomicExch(&bar->err[0], 1);
            s_fail = 1;
            break;
          }
          if (it > 64) __nanosleep(32);
        }
        __threadfence();
      }
      __syncthreads();
      if (s_fail) return;  // block-uniform after the barrier
      const T fc = step_fc<T>(I, n, A.fs, n == 0);
      const double fcos = A.fs * I.cosn[n];
      const double wf_new = I.wf[n + 1], wf_cur = I.wf[n];
      // stage W^n (tile + halo; wrapped on periodic axes, clamped into the extended array)
      for (int e = tid; e < SX * SY; e += kTileX * kTileY) {
        const int rr = e / SX, cc = e % SX;
        int ii = wrap(t.i0 - R + cc, G.n0, G.per0);
        ii = ii < -G.g0 ? -G.g0 : (ii >= G.n0 + G.g0 ? G.n0 + G.g0 - 1 : ii);
        sw[rr][cc] = cur[row_off(G, t.j0 - R + rr) + ii];
      }
      __syncthreads();
      // patch ghost and receiver positions with their level-n values
      for (int64_t e = A.patch_off[tile] + tid; e < A.patch_off[tile + 1];
           e += kTileX * kTileY) {
        const int32_t pos = A.patch_pos[e], item = A.patch_item[e];
        const int kind = pos >> 24, sidx = pos & 0xffffff;
        double v;
        if (kind == 2) v = recv_value<T, ORDER>(item, A.didx, A.dw, cur);
        else v = bc_value<T>(A.bc[item], cur, F, fcos, kind);
        (&sw[0][0])[sidx] = (T)v;
      }
      __syncthreads();
      const int i = t.i0 + (int)threadIdx.x;
      if (i < G.n0) {
#pragma unroll
        for (int m = 0; m < kPY; ++m) {
          const int r = (int)threadIdx.y + m * kTileY;
          const int j = t.j0 + r;
          if (j >= G.n1) continue;
          const int64_t p = row_off(G, j) + i;
          const int8_t mk = A.mask[p];
          const T wc = sw[r + R][threadIdx.x + R];
          if (mk == 2) {
            A.V[p] = fma(wf_cur, to_f64(wc), A.V[p]);
            continue;
          }
          if (mk == 3) {
            if (G.gb) {
              A.V[p] = fma(wf_cur, to_f64(wc), A.V[p]);
              oth[p] = (T)(A.fs * I.cosn[n + 1] * G.gb[p]);
            }
            continue;
          }
          if (mk != 1) continue;
          T a;
          if (G.stencil == kConstCross) {
            const T c0 = grid_w<T>(G, 0), x1 = grid_w<T>(G, 1), y1 = grid_w<T>(G, 3);
            a = n == 0 ? c0 * wc : fma(c0, wc, -oth[p]);
            a = fma(x1, sw[r + R][threadIdx.x + R - 1], a);
            a = fma(x1, sw[r + R][threadIdx.x + R + 1], a);
            a = fma(y1, sw[r + R - 1][threadIdx.x + R], a);
            a = fma(y1, sw[r + R + 1][threadIdx.x + R], a);
            if (ORDER == 4) {
              const T x2 = grid_w<T>(G, 2), y2 = grid_w<T>(G, 4);
              a = fma(x2, sw[r + R][threadIdx.x + R - 2], a);
              a = fma(x2, sw[r + R][threadIdx.x + R + 2], a);
              a = fma(y2, sw[r + R - 2][threadIdx.x + R], a);
              a = fma(y2, sw[r + R + 2][threadIdx.x + R], a);
            }
          } else if (G.stencil == kPointCross) {
            const int64_t q = G.wbase + (p - G.base), E = G.ext;
            a = n == 0 ? Wt[q] * wc : fma(Wt[q], wc, -oth[p]);
            int pl = 1;
#pragma unroll
            for (int k = -R; k <= R; ++k) {
              if (k == 0) continue;
              a = fma(Wt[q + pl * E], sw[r + R][threadIdx.x + R + k], a);
              ++pl;
            }
#pragma unroll
            for (int k = -R; k <= R; ++k) {
              if (k == 0) continue;
              a = fma(Wt[q + pl * E], sw[r + R + k][threadIdx.x + R], a);
              ++pl;
            }
          } else {
            const int64_t q = G.wbase + (p - G.base), E = G.ext;
            a = n == 0 ? (T)0 : -oth[p];
#pragma unroll
            for (int bb = -R; bb <= R; ++bb)
#pragma unroll
              for (int aa = -R; aa <= R; ++aa)
                a = fma(Wt[q + ((bb + R) * (2 * R + 1) + (aa + R)) * E],
                        sw[r + R + bb][threadIdx.x + R + aa], a);
          }
          if (n == 0) a *= (T)0.5;
          a = fma(-fc, F[p], a);
          oth[p] = a;
          A.V[p] = fma(wf_new, to_f64(a), A.V[p]);
        }
      }
    }
    __syncthreads();  // the tile's values are written; the staged box is reused next
    if (tid == 0) {
      __threadfence();
      atomicMax(&A.tile_done[tile], n + 1);  // (n, tile) waited for (n - 1, tile): in order
    }
    tk = s_tk;
    __syncthreads();
  }
  if (!grid_sync(bar, nb, A.spin_limit)) return;
  // output; receivers add their level-M contribution, computed from their donors
  for (int64_t c = gtid; c < A.ncompact; c += nthreads) {
    int g = 0;
    while (g + 1 < A.ngrids && c >= A.grids[g + 1].cbase) ++g;
    const DevGrid &G = A.grids[g];
    const InstDev &I = A.inst[G.inst];
    if (!I.active) continue;
    const T *WM = (I.M % 2 == 0) ? Wa : Wb;
    const int64_t o = c - G.cbase;
    const int j = (int)(o / G.n0), i = (int)(o % G.n0);
    const int64_t p = G.base + (int64_t)(j + G.g1) * G.pitch + (i + G.g0);
    const int8_t m = A.mask[p];
    double val = 0.0;
    if (m == 1 || (m == 3 && !G.gb)) val = A.V[p];
    else if (m == 3)  // Dirichlet data: the level-M contribution is not in V yet
      val = fma(I.wf[I.M], to_f64(WM[p]), A.V[p]);
    else if (m == 2)
      val = fma(I.wf[I.M], recv_value<T, ORDER>(A.recv_of[p], A.didx, A.dw, WM), A.V[p]);
    v_out[c] = val;
  }
}

// ---------------------------------------------------------------------------------
// Differentiation: the exact transpose of the discrete iteration map (FP64).
// With C the constraint map (ghost rules + interpolation), D the restriction to
// discretization points and A the stencil operator (rows of the march), the forward map is
//   X^0 = C E v,  X^1 = C D(A X^0 / 2 - ...),  X^{n+1} = C D(A X^n - X^{n-1} - ...),
//   W_h = sum_n w_n M X^n.
// Its transpose runs backwards: Y^n = w_n M lam + s_n A^T Z^{n+1} - Z^{n+2} (s_0 = 1/2),
// Z^n = D C^T Y^n, and S^T lam = Z^0.
// ---------------------------------------------------------------------------------

// locate the grid and (i, j) of extended point p; false on padding
__device__ __forceinline__ bool ext_locate(const DevGrid *__restrict__ grids, int ngrids,
                                           int64_t p, int &g, int &i, int &j) {
  g = 0;
  while (g + 1 < ngrids && p >= grids[g + 1].base) ++g;
  const DevGrid &G = grids[g];
  const int64_t o64 = p - G.base;
  if (o64 >= G.ext) return false;
  const int o = (int)o64;  // the whole state is below 2^31 entries (checked at layout)
  j = o / G.pitch - G.g1;
  i = o - (j + G.g1) * G.pitch - G.g0;
  return i < G.n0 + G.g0;
}

// Z value of a neighbour (i, j) if it is inside the grid's discretization range (else 0;
// Z vanishes off discretization points anyway)
__device__ __forceinline__ bool nb_index(const DevGrid &G, int i, int j, int64_t &p) {
  if (G.per0) i = wrap(i, G.n0, 1);
  else if (i < 0 || i >= G.n0) return false;
  if (G.per1) j = wrap(j, G.n1, 1);
  else if (j < 0 || j >= G.n1) return false;
  p = G.base + (int64_t)(j + G.g1) * G.pitch + (i + G.g0);
  return true;
}

// Neighbour (i + di, j + dj) of point q = (i, j): plain offsets for interior points (every
// neighbour of the stencil inside the discretization range, no wrap), else nb_index.
__device__ __forceinline__ bool nbr(const DevGrid &G, int64_t q, int i, int j, int di, int dj,
                                    bool interior, int64_t &p) {
  if (interior) {
    p = q + di + (int64_t)dj * G.pitch;
    return true;
  }
  return nb_index(G, i + di, j + dj, p);
}

// One reverse step at every extended point q:
//   Y = w_n lam (active points) + s (A^T Z1) - Z2,  Znew = D Y (Y at discretization points,
//   0 elsewhere; the constraint part of C^T is added afterwards by adj_post_kernel).
// In gradient mode (Xn != nullptr; Xprev, Xn, Xnext the forward states n-1, n, n+1, Xprev
// null at n = 0) discretization points also add the parameter gradients of the step
// n -> n+1: gf -= fc Z1, c^2 gc2 += s Z1 ((A Xn) - 2 Xn) (gc2 is accumulated times c^2
// and divided by it when the sweep ends).
template <int ORDER>
__global__ void adj_step_kernel(const DevGrid *__restrict__ grids, int ngrids,
                                const int8_t *__restrict__ mask, const double *__restrict__ Wt,
                                const double *__restrict__ lam, double wn, double sc,
                                const double *__restrict__ Z1, const double *__restrict__ Z2,
                                double *__restrict__ Y, double *__restrict__ Znew, int64_t total,
                                const double *__restrict__ Xprev, const double *__restrict__ Xn,
                                const double *__restrict__ Xnext, const double *__restrict__ F,
                                double fc, double *gc2, double *gf) {
  constexpr int R = ORDER / 2;
  pdl_wait();
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= total) return;
  int g, i, j;
  if (!ext_locate(grids, ngrids, q, g, i, j)) {
    Y[q] = 0.0;
    Znew[q] = 0.0;
    return;
  }
  const DevGrid &G = grids[g];
  const int8_t mk = mask[q];
  if (mk == 0 && i >= 0 && i < G.n0 && j >= 0 && j < G.n1) {
    // unused point inside the grid: not a discretization point and not a constrained
    // position (those are receivers and ghost lines), so its Y is never read
    Y[q] = 0.0;
    Znew[q] = 0.0;
    return;
  }
  const bool interior = i >= R && i < G.n0 - R && j >= R && j < G.n1 - R;
  double at = 0.0;  // (A^T Z1)[q] = sum_o A[q - o, q] Z1[q - o]
  if (G.stencil == kConstCross) {
    // constant symmetric weights: A^T Z = A Z
    int64_t pn;
    if (nbr(G, q, i, j, 0, 0, interior, pn)) at += G.cw[0] * Z1[pn];
#pragma unroll
    for (int k = 1; k <= R; ++k) {
      const double wx = G.cw[k], wy = G.cw[2 + k];
      if (nbr(G, q, i, j, -k, 0, interior, pn)) at += wx * Z1[pn];
      if (nbr(G, q, i, j, k, 0, interior, pn)) at += wx * Z1[pn];
      if (nbr(G, q, i, j, 0, -k, interior, pn)) at += wy * Z1[pn];
      if (nbr(G, q, i, j, 0, k, interior, pn)) at += wy * Z1[pn];
    }
  } else if (G.stencil == kPointCross) {
    const int64_t E = G.ext;
    int64_t pn;
    if (nbr(G, q, i, j, 0, 0, interior, pn)) at += Wt[G.wbase + (pn - G.base)] * Z1[pn];
    int pl = 1;
#pragma unroll
    for (int k = -R; k <= R; ++k) {  // axis-0 offset k of row p = q - k
      if (k == 0) continue;
      if (nbr(G, q, i, j, -k, 0, interior, pn))
        at += Wt[G.wbase + (pn - G.base) + pl * E] * Z1[pn];
      ++pl;
    }
#pragma unroll
    for (int k = -R; k <= R; ++k) {
      if (k == 0) continue;
      if (nbr(G, q, i, j, 0, -k, interior, pn))
        at += Wt[G.wbase + (pn - G.base) + pl * E] * Z1[pn];
      ++pl;
    }
  } else {
    const int64_t E = G.ext;
#pragma unroll
    for (int b = -R; b <= R; ++b)
#pragma unroll
      for (int a = -R; a <= R; ++a) {
        int64_t pn;
        if (nbr(G, q, i, j, -a, -b, interior, pn))
          at += Wt[G.wbase + (pn - G.base) + ((b + R) * (2 * R + 1) + (a + R)) * E] * Z1[pn];
      }
  }
  const bool active = mk == 1 || mk == 2 || mk == 3;
  const double y = fma(sc, at, active ? fma(wn, lam[q], -Z2[q]) : -Z2[q]);
  Y[q] = y;
  Znew[q] = mk == 1 ? y : 0.0;
  if (Xn && mk == 1) {
    // (A X^n)[q] - 2 X^n[q] from the forward step itself, which at a discretization point
    // is X^{n+1} = A X^n - X^{n-1} - fc F (n > 0) or X^1 = A X^0 / 2 - fc F (n = 0)
    const double xn = Xn[q], fx = fma(fc, F[q], Xnext[q]);
    const double ax = Xprev ? fx + Xprev[q] - 2.0 * xn : 2.0 * (fx - xn);
    const double z = Z1[q];
    gc2[q] = fma(sc * z, ax, gc2[q]);  // divided by c^2 once, after the sweep
    gf[q] -= fc * z;
  }
}

// After adj_step_kernel, two independent jobs split by block (no launch of its own each):
//  * blocks [0, fix_blocks): the constraint part of Z = D C^T Y.  Each listed discretization
//    point adds the Y values of the constrained positions (ghosts, receivers) that read it,
//    times the constraint coefficients; 8 lanes share a point's entries (a background donor
//    point sits in the donor blocks of dozens of receivers) and combine them with xor
//    shuffles.  Constrained positions are never discretization points, so Y there is final.
//  * the remaining blocks (gradient mode): the gradient terms of the Dirichlet order-4
//    compatibility rule at this level.  With t = Y[G1] + 5 Y[G2]: gf[b] += fcos inv t and
//    c^2_b gc2[b] -= F_b fcos inv t (times c^2, like adj_step_kernel).
constexpr int kFixLanes = 8;
__global__ void adj_post_kernel(const int64_t *__restrict__ fq, const int64_t *__restrict__ foff,
                                const int64_t *__restrict__ rpos,
                                const double *__restrict__ rcoef, const double *__restrict__ Y,
                                double *__restrict__ Z, int64_t nfix, int fix_blocks,
                                const BcItem *__restrict__ bc, int nbc,
                                const double *__restrict__ F, double fcos, double *gc2,
                                double *gf) {
  pdl_wait();
  if ((int)blockIdx.x < fix_blocks) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t k = t / kFixLanes;
    const int lane = (int)(t % kFixLanes);
    const bool live = k < nfix;
    double z = 0.0;
    if (live)
      for (int64_t e = foff[k] + lane; e < foff[k + 1]; e += kFixLanes)
        z = fma(rcoef[e], Y[rpos[e]], z);
#pragma unroll
    for (int off = kFixLanes / 2; off > 0; off >>= 1)
      z += __shfl_xor_sync(0xffffffffu, z, off, kFixLanes);
    if (live && lane == 0) Z[fq[k]] += z;
    return;
  }
  const int k = ((int)blockIdx.x - fix_blocks) * blockDim.x + threadIdx.x;
  if (k >= nbc) return;
  const BcItem it = bc[k];
  if (it.type != 2) return;
  const double t = Y[it.g[0]] + 5.0 * Y[it.g[1]];
  const int64_t b = it.u[0];
  gf[b] += fcos * it.inv * t;
  gc2[b] -= F[b] * fcos * it.inv * t;
}

// compact <-> extended copies at active points (ext -> compact optionally divides by div)
__global__ void compact_to_ext_kernel(const DevGrid *__restrict__ grids, int ngrids,
                                      const int8_t *__restrict__ mask, const double *__restrict__ v,
                                      double *x, int64_t total) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= total) return;
  int g, i, j;
  double val = 0.0;
  if (ext_locate(grids, ngrids, p, g, i, j) && mask[p] != 0 && i >= 0 && i < grids[g].n0 &&
      j >= 0 && j < grids[g].n1)
    val = v[grids[g].cbase + (int64_t)j * grids[g].n0 + i];
  x[p] = val;
}

__global__ void ext_to_compact_kernel(const DevGrid *__restrict__ grids, int ngrids,
                                      const int8_t *__restrict__ mask, const double *__restrict__ x,
                                      double *v, int64_t ncompact, int disc_only,
                                      const double *__restrict__ div) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncompact) return;
  int g = 0;
  while (g + 1 < ngrids && c >= grids[g + 1].cbase) ++g;
  const DevGrid &G = grids[g];
  const int64_t o = c - G.cbase;
  const int j = (int)(o / G.n0), i = (int)(o % G.n0);
  const int64_t p = G.base + (int64_t)(j + G.g1) * G.pitch + (i + G.g0);
  const int8_t m = mask[p];
  const bool on = disc_only ? m == 1 : m != 0;
  v[c] = on ? (div ? x[p] / div[p] : x[p]) : 0.0;
}

// ---------------------------------------------------------------------------------
// Operator precompute (mapping method, Sec. 3.1): per point a11, a12, a22, b1, b2 with
// c(x)^2 folded in, and the frozen-coefficient spectral bound
//   s = a11/dr1^2 + a22/dr2^2 + 2|a12|/(dr1 dr2)   (max over discretization points).
// ---------------------------------------------------------------------------------

template <int ORDER>
__device__ __forceinline__ double d1(const double *a, const DevGrid &G, int i, int j,
                                     int axis) {
  // first derivative of an extended array along an axis: D0 or D0 (1 - h^2/6 D+D-)
  auto at = [&](int ii, int jj) {
    ii = wrap(ii, G.n0, G.per0);
    jj = wrap(jj, G.n1, G.per1);
    return a[(int64_t)(jj + G.g1) * G.pitch + (ii + G.g0)];
  };
  const double h = axis == 0 ? G.h0 : G.h1;
  const int di = axis == 0, dj = axis == 1;
  if (ORDER == 2) return (at(i + di, j + dj) - at(i - di, j - dj)) / (2.0 * h);
  return (8.0 * (at(i + di, j + dj) - at(i - di, j - dj)) -
          (at(i + 2 * di, j + 2 * dj) - at(i - 2 * di, j - 2 * dj))) / (12.0 * h);
}

template <int ORDER>
__global__ void coef_kernel(const DevGrid *__restrict__ grids, int gidx,
                            const int8_t *__restrict__ mask, const double *__restrict__ rx,
                            const double *__restrict__ c2, double *coef,
                            unsigned long long *smax_bits) {
  const DevGrid &G = grids[gidx];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= G.n0 || j >= G.n1) return;
  const int64_t o = (int64_t)(j + G.g1) * G.pitch + (i + G.g0);
  const int8_t m = mask[G.base + o];
  if (m != 1 && m != 3) return;
  const double cc = c2[G.base + o];
  double s;
  if (G.kind == 0) {
    s = cc * (1.0 / (G.h0 * G.h0) + 1.0 / (G.h1 * G.h1));
  } else {
    const int64_t E = G.ext;
    const double *r = rx + G.kbase;  // 4 metric planes dr_k/dx_m at plane 2k+m
    double rr[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) rr[k] = r[k * E + o];
    const double a11 = rr[0] * rr[0] + rr[1] * rr[1];
    const double a12 = rr[0] * rr[2] + rr[1] * rr[3];
    const double a22 = rr[2] * rr[2] + rr[3] * rr[3];
    double b[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      double acc = 0.0;
#pragma unroll
      for (int mm = 0; mm < 2; ++mm)
#pragma unroll
        for (int l = 0; l < 2; ++l)
          acc += rr[2 * l + mm] * d1<ORDER>(r + (2 * k + mm) * E, G, i, j, l);
      b[k] = acc;
    }
    double *cf = coef + G.kbase;
    cf[o] = cc * a11;
    cf[E + o] = cc * a12;
    cf[2 * E + o] = cc * a22;
    cf[3 * E + o] = cc * b[0];
    cf[4 * E + o] = cc * b[1];
    s = cc * (a11 / (G.h0 * G.h0) + a22 / (G.h1 * G.h1));
    if (!G.ortho) s += 2.0 * cc * fabs(a12) / (G.h0 * G.h1);
  }
  if (m == 1) atomicMax(smax_bits + G.inst, (unsigned long long)__double_as_longlong(s));
}

// Per-point stencil weights (dt^2 folded, centre + 2).  Cartesian grids with c(x) use
// the cross with a11 = a22 = c^2 (physical spacing), no first-derivative terms.
template <typename T, int ORDER>
__global__ void weight_kernel(const DevGrid *__restrict__ grids, int gidx,
                              const int8_t *__restrict__ mask, const double *__restrict__ coef,
                              const double *__restrict__ c2, T *Wt, double dt2) {
  const DevGrid &G = grids[gidx];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= G.n0 || j >= G.n1) return;
  const int64_t o = (int64_t)(j + G.g1) * G.pitch + (i + G.g0);
  if (mask[G.base + o] != 1) return;
  constexpr int R = ORDER / 2;
  const int64_t E = G.ext;
  double A1, A2, B1 = 0.0, B2 = 0.0, A12 = 0.0;
  if (G.kind == 0) {
    A1 = A2 = c2[G.base + o];
  } else {
    const double *cf = coef + G.kbase;
    A1 = cf[o];
    A12 = G.ortho ? 0.0 : cf[E + o];
    A2 = cf[2 * E + o];
    B1 = cf[3 * E + o];
    B2 = cf[4 * E + o];
  }
  // 1-D weights: second derivative D2[k], first derivative D1[k], offsets -R..R
  double D2[2 * R + 1], D1[2 * R + 1];
  if (ORDER == 2) {
    D2[0] = 1.0; D2[1] = -2.0; D2[2] = 1.0;
    D1[0] = -0.5; D1[1] = 0.0; D1[2] = 0.5;
  } else {
    D2[0] = -1.0 / 12; D2[1] = 16.0 / 12; D2[2] = -30.0 / 12; D2[3] = 16.0 / 12; D2[4] = -1.0 / 12;
    D1[0] = 1.0 / 12; D1[1] = -8.0 / 12; D1[2] = 0.0; D1[3] = 8.0 / 12; D1[4] = -1.0 / 12;
  }
  const double h0 = G.h0, h1 = G.h1;
  T *w = Wt + G.wbase + o;
  if (G.stencil == kPointCross) {
    double wc = 2.0 + dt2 * (A1 * D2[R] / (h0 * h0) + A2 * D2[R] / (h1 * h1));
    w[0] = (T)wc;
    int pl = 1;
    for (int k = -R; k <= R; ++k) {
      if (k == 0) continue;
      w[pl * E] = (T)(dt2 * (A1 * D2[k + R] / (h0 * h0) + B1 * D1[k + R] / h0));
      ++pl;
    }
    for (int k = -R; k <= R; ++k) {
      if (k == 0) continue;
      w[pl * E] = (T)(dt2 * (A2 * D2[k + R] / (h1 * h1) + B2 * D1[k + R] / h1));
      ++pl;
    }
  } else {
    for (int b = -R; b <= R; ++b)
      for (int a = -R; a <= R; ++a) {
        double v = 2.0 * A12 * D1[a + R] * D1[b + R] / (h0 * h1);
        if (b == 0) v += A1 * D2[a + R] / (h0 * h0) + B1 * D1[a + R] / h0;
        if (a == 0) v += A2 * D2[b + R] / (h1 * h1) + B2 * D1[b + R] / h1;
        v *= dt2;
        if (a == 0 && b == 0) v += 2.0;
        w[((b + R) * (2 * R + 1) + (a + R)) * E] = (T)v;
      }
  }
}

// Dirichlet order-4 item coefficients from the operator coefficients of the boundary
// point: A2 = a_nn/(12 h^2), B1 = sgn b_n/(12 h) (sgn = -1 on a high side).
__global__ void bc_coef_kernel(BcItem *bc, int nbc, const int32_t *__restrict__ item_grid,
                               const int32_t *__restrict__ item_axis,
                               const int32_t *__restrict__ item_hi,
                               const DevGrid *__restrict__ grids,
                               const double *__restrict__ coef, const double *__restrict__ c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nbc || bc[k].type != 2) return;
  const DevGrid &G = grids[item_grid[k]];
  const int a = item_axis[k];
  const int64_t p = bc[k].u[0];
  const double h = a == 0 ? G.h0 : G.h1;
  double ann, bn;
  if (G.kind == 0) {
    ann = c2[p];
    bn = 0.0;
  } else {
    const int64_t o = G.kbase + (p - G.base);
    ann = coef[o + (a == 0 ? 0 : 2) * G.ext];
    bn = coef[o + (3 + a) * G.ext];
  }
  const double sgn = item_hi[k] ? -1.0 : 1.0;
  bc[k].A2 = ann / (12.0 * h * h);
  bc[k].B1 = sgn * bn / (12.0 * h);
  bc[k].inv = 1.0 / (11.0 * bc[k].A2 - 3.0 * bc[k].B1);
}

// ---------------------------------------------------------------------------------
// Reductions for GMRES (Sec. 4.3): FP64, warp-shuffle partial sums per block, then one
// deterministic second pass.  `nv` vectors X[k] (stride ldx) against y.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double s) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

__global__ void __launch_bounds__(kRedThreads)
    multidot_partial(const double *__restrict__ X, int64_t ldx, int nv,
                     const double *__restrict__ y, int64_t n, double *partial) {
  // partial[k * gridDim.x + block] = sum over this block's grid-stride share
  __shared__ double red[kRedThreads / 32];
  for (int k = 0; k < nv; ++k) {
    const double *x = X + k * ldx;
    double s = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
      s = fma(x[q], y[q], s);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
      double t = threadIdx.x < kRedThreads / 32 ? red[threadIdx.x] : 0.0;
      t = warp_sum(t);
      if (threadIdx.x == 0) partial[(int64_t)k * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kRedThreads)
    partial_finish(const double *__restrict__ partial, int nblocks, int nv, double *out) {
  // one block per vector, fixed order
  __shared__ double red[kRedThreads / 32];
  const int k = blockIdx.x;
  if (k >= nv) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(int64_t)k * nblocks + b];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < kRedThreads / 32 ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) out[k] = t;
  }
}

// y -= sum_k h[k] X[k]   (h on the device)
__global__ void multi_axpy(const double *__restrict__ X, int64_t ldx, int nv,
                           const double *__restrict__ h, double *y, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    double s = y[q];
    for (int k = 0; k < nv; ++k) s = fma(-h[k], X[k * ldx + q], s);
    y[q] = s;
  }
}

// y = a x + b y
__global__ void axpby(double a, const double *__restrict__ x, double b, double *y, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    y[q] = a * x[q] + b * y[q];
}

// y = x - z
__global__ void sub(const double *__restrict__ x, const double *__restrict__ z, double *y,
                    int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    y[q] = x[q] - z[q];
}

// y += X^T c  (c on the device, nv entries)
__global__ void gemv_acc(const double *__restrict__ X, int64_t ldx, int nv,
                         const double *__restrict__ c, double *y, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    double s = y[q];
    for (int k = 0; k < nv; ++k) s = fma(c[k], X[k * ldx + q], s);
    y[q] = s;
  }
}

// ---------------------------------------------------------------------------------
// Host launchers (the only entry points the host code uses).
// ---------------------------------------------------------------------------------

// Launches of the iteration graph's kernels ask for programmatic serialization while
// set_pdl(true) is in effect on this thread (the graph capture).
static thread_local bool t_pdl = false;
void set_pdl(bool on) { t_pdl = on; }

template <typename... KArgs, typename... Args>
static void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t s, Args... args) {
  if (!t_pdl) {
    kernel<<<grid, block, smem, s>>>(args...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

void launch_march(bool fp32, int order, bool first, int nblocks, int ntiles, cudaStream_t s,
                  const DevGrid *grids, const Tile *tiles, const int8_t *mask, const void *Wn,
                  void *Wout, const void *F, const void *Wt, double *V, const InstDev *inst,
                  int n, double fs, const void *Wprev, const GatherArgs *gather) {
  const dim3 tb(kTileX, kTileY);
  if (!Wprev) Wprev = Wout;
  GatherArgs ga{};
  if (gather) ga = *gather;
#define WH_MARCH(T, O, FI, NF)                                                             \
  launch_k(march_kernel<T, O, FI, NF>, dim3(nblocks), tb, 0, s, grids, tiles, ntiles, mask, \
           (const T *)Wn, (const T *)Wprev, (T *)Wout, (const T *)F, (const T *)Wt, V, inst,  \
           n, fs, ga)
#define WH_MARCH3(T, O)                                                                    \
  do {                                                                                     \
    if (first) WH_MARCH(T, O, true, false);                                                \
    else if (fs == 0.0) WH_MARCH(T, O, false, true);                                       \
    else WH_MARCH(T, O, false, false);                                                     \
  } while (0)
  if (fp32) {
    if (order == 4) WH_MARCH3(float, 4);
    else            WH_MARCH3(float, 2);
  } else {
    if (order == 4) WH_MARCH3(double, 4);
    else            WH_MARCH3(double, 2);
  }
#undef WH_MARCH3
#undef WH_MARCH
}

size_t march_tma_smem(bool fp32, int order) {
  if (fp32) return order == 4 ? TmaStage<float, 4>::kSmem : TmaStage<float, 2>::kSmem;
  return order == 4 ? TmaStage<double, 4>::kSmem : TmaStage<double, 2>::kSmem;
}

template <typename T, int O, bool FI>
static void tma_attr() {
  cudaFuncSetAttribute(march_tma_kernel<T, O, FI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)TmaStage<T, O>::kSmem);
}

int march_tma_blocks_per_sm(bool fp32, int order) {
  const int threads = kTileX * kTileY;
  int nb = 0;
  if (fp32) {
    if (order == 4) {
      tma_attr<float, 4, false>();
      tma_attr<float, 4, true>();
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, march_tma_kernel<float, 4, false>,
                                                    threads, TmaStage<float, 4>::kSmem);
    } else {
      tma_attr<float, 2, false>();
      tma_attr<float, 2, true>();
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, march_tma_kernel<float, 2, false>,
                                                    threads, TmaStage<float, 2>::kSmem);
    }
  } else {
    if (order == 4) {
      tma_attr<double, 4, false>();
      tma_attr<double, 4, true>();
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, march_tma_kernel<double, 4, false>,
                                                    threads, TmaStage<double, 4>::kSmem);
    } else {
      tma_attr<double, 2, false>();
      tma_attr<double, 2, true>();
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, march_tma_kernel<double, 2, false>,
                                                    threads, TmaStage<double, 2>::kSmem);
    }
  }
  return nb < 1 ? 1 : nb;
}

void launch_march_tma(bool fp32, int order, bool first, int nblocks, cudaStream_t s,
                      const DevGrid *grids, const Tile *ftiles, int nfast, const CUtensorMap *maps,
                      const Tile *gtiles, int ngen, const int8_t *mask, void *Wa, void *Wb,
                      const void *F, const void *Wt, double *V, const InstDev *inst, int n,
                      double fs, int *ctl, unsigned long long spin_limit,
                      const GatherArgs *gather) {
  const dim3 tb(kTileX, kTileY);
  GatherArgs ga{};
  if (gather) ga = *gather;
#define WH_TMA(T, O, FI)                                                                       \
  launch_k(march_tma_kernel<T, O, FI>, dim3(nblocks), tb, TmaStage<T, O>::kSmem, s, grids,     \
           ftiles, nfast, maps, gtiles, ngen, mask, (T *)Wa, (T *)Wb, (const T *)F,            \
           (const T *)Wt, V, inst, n, fs, ctl, spin_limit, ga)
  if (fp32) {
    if (order == 4) { if (first) WH_TMA(float, 4, true); else WH_TMA(float, 4, false); }
    else            { if (first) WH_TMA(float, 2, true); else WH_TMA(float, 2, false); }
  } else {
    if (order == 4) { if (first) WH_TMA(double, 4, true); else WH_TMA(double, 4, false); }
    else            { if (first) WH_TMA(double, 2, true); else WH_TMA(double, 2, false); }
  }
#undef WH_TMA
}

void launch_bc_gather(bool fp32, int order, int blocks, cudaStream_t s, const BcItem *bc,
                      int nbc, int bc_blocks, const int32_t *didx, const double *dw,
                      const int64_t *ridx, const int32_t *rinst, int nrecv, void *W,
                      const void *F, const InstDev *inst, int level, double fs) {
#define WH_BCG(T, O)                                                                       \
  launch_k(bc_gather_kernel<T, O>, dim3(blocks), dim3(256), 0, s, bc, nbc, bc_blocks, didx, dw, \
           ridx, rinst, nrecv, (T *)W, (const T *)F, inst, level, fs)
  if (fp32) { if (order == 4) WH_BCG(float, 4); else WH_BCG(float, 2); }
  else      { if (order == 4) WH_BCG(double, 4); else WH_BCG(double, 2); }
#undef WH_BCG
}

void launch_init(bool fp32, unsigned blocks, cudaStream_t s, const DevGrid *grids, int ngrids,
                 const int8_t *mask, const double *v, void *W0, double *V, int64_t total,
                 const InstDev *inst, double fs) {
  if (fp32)
    init_kernel<float><<<blocks, 256, 0, s>>>(grids, ngrids, mask, v, (float *)W0, V, total, inst,
                                              fs);
  else
    init_kernel<double><<<blocks, 256, 0, s>>>(grids, ngrids, mask, v, (double *)W0, V, total,
                                               inst, fs);
}

void launch_finish(bool fp32, unsigned blocks, cudaStream_t s, const DevGrid *grids, int ngrids,
                   const int8_t *mask, const double *V, const void *Wa, const void *Wb,
                   const InstDev *inst, double *vout, int64_t ncompact) {
  if (fp32)
    finish_kernel<float><<<blocks, 256, 0, s>>>(grids, ngrids, mask, V, (const float *)Wa,
                                                (const float *)Wb, inst, vout, ncompact);
  else
    finish_kernel<double><<<blocks, 256, 0, s>>>(grids, ngrids, mask, V, (const double *)Wa,
                                                 (const double *)Wb, inst, vout, ncompact);
}

int march_blocks_per_sm(bool fp32, int order) {
  int nb = 0;
  const int threads = kTileX * kTileY;
  if (fp32) {
    if (order == 4) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, march_kernel<float, 4, false>, threads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, march_kernel<float, 2, false>, threads, 0);
  } else {
    if (order == 4) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, march_kernel<double, 4, false>, threads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, march_kernel<double, 2, false>, threads, 0);
  }
  return nb > 0 ? nb : 1;
}

int iteration_blocks_per_sm(bool fp32, int order) {
  int nb = 0;
  const int threads = kTileX * kTileY;
  if (fp32) {
    if (order == 4) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, iteration_kernel<float, 4>, threads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, iteration_kernel<float, 2>, threads, 0);
  } else {
    if (order == 4) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, iteration_kernel<double, 4>, threads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, iteration_kernel<double, 2>, threads, 0);
  }
  return nb;
}

cudaError_t launch_iteration(bool fp32, int order, int nblocks, cudaStream_t s,
                             const IterArgs &A, const double *v_in, double *v_out,
                             GridBarrier *bar) {
  IterArgs a = A;
  void *args[] = {(void *)&a, (void *)&v_in, (void *)&v_out, (void *)&bar};
  const dim3 tb(kTileX, kTileY), gb(nblocks);
  const void *fn;
  if (fp32) fn = order == 4 ? (const void *)iteration_kernel<float, 4> : (const void *)iteration_kernel<float, 2>;
  else fn = order == 4 ? (const void *)iteration_kernel<double, 4> : (const void *)iteration_kernel<double, 2>;
  return cudaLaunchCooperativeKernel(fn, gb, tb, args, 0, s);
}

void launch_coef(int order, dim3 gb, dim3 tb, cudaStream_t s, const DevGrid *grids, int gidx,
                 const int8_t *mask, const double *rx, const double *c2, double *coef,
                 unsigned long long *smax) {
  if (order == 4) coef_kernel<4><<<gb, tb, 0, s>>>(grids, gidx, mask, rx, c2, coef, smax);
  else coef_kernel<2><<<gb, tb, 0, s>>>(grids, gidx, mask, rx, c2, coef, smax);
}

void launch_weight(bool fp32, int order, dim3 gb, dim3 tb, cudaStream_t s, const DevGrid *grids,
                   int gidx, const int8_t *mask, const double *coef, const double *c2, void *Wt,
                   double dt2) {
  if (fp32) {
    if (order == 4) weight_kernel<float, 4><<<gb, tb, 0, s>>>(grids, gidx, mask, coef, c2, (float *)Wt, dt2);
    else weight_kernel<float, 2><<<gb, tb, 0, s>>>(grids, gidx, mask, coef, c2, (float *)Wt, dt2);
  } else {
    if (order == 4) weight_kernel<double, 4><<<gb, tb, 0, s>>>(grids, gidx, mask, coef, c2, (double *)Wt, dt2);
    else weight_kernel<double, 2><<<gb, tb, 0, s>>>(grids, gidx, mask, coef, c2, (double *)Wt, dt2);
  }
}

void launch_bc_coef(int nbc, cudaStream_t s, BcItem *bc, const int32_t *ig, const int32_t *ia,
                    const int32_t *ih, const DevGrid *grids, const double *coef,
                    const double *c2) {
  bc_coef_kernel<<<(nbc + 255) / 256, 256, 0, s>>>(bc, nbc, ig, ia, ih, grids, coef, c2);
}

void launch_adj_step(int order, cudaStream_t s, const DevGrid *grids, int ngrids,
                     const int8_t *mask, const double *Wt, const double *lam, double wn,
                     double sc, const double *Z1, const double *Z2, double *Y, double *Znew,
                     int64_t total, const double *Xprev, const double *Xn, const double *Xnext,
                     const double *F, double fc, double *gc2, double *gf) {
  const unsigned nb = (unsigned)((total + 255) / 256);
  if (order == 4)
    launch_k(adj_step_kernel<4>, dim3(nb), dim3(256), 0, s, grids, ngrids, mask, Wt, lam, wn, sc,
             Z1, Z2, Y, Znew, total, Xprev, Xn, Xnext, F, fc, gc2, gf);
  else
    launch_k(adj_step_kernel<2>, dim3(nb), dim3(256), 0, s, grids, ngrids, mask, Wt, lam, wn, sc,
             Z1, Z2, Y, Znew, total, Xprev, Xn, Xnext, F, fc, gc2, gf);
}

void launch_adj_post(cudaStream_t s, const int64_t *fq, const int64_t *foff, const int64_t *rpos,
                     const double *rcoef, const double *Y, double *Z, int64_t nfix,
                     const BcItem *bc, int nbc, const double *F, double fcos, double *gc2,
                     double *gf) {
  const int fix_blocks = (int)((nfix * kFixLanes + 255) / 256);
  const int bc_blocks = gc2 ? (nbc + 255) / 256 : 0;
  if (fix_blocks + bc_blocks)
    launch_k(adj_post_kernel, dim3(fix_blocks + bc_blocks), dim3(256), 0, s, fq, foff, rpos,
             rcoef, Y, Z, nfix, fix_blocks, bc, gc2 ? nbc : 0, F, fcos, gc2, gf);
}

void launch_compact_to_ext(cudaStream_t s, const DevGrid *grids, int ngrids, const int8_t *mask,
                           const double *v, double *x, int64_t total) {
  compact_to_ext_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(grids, ngrids, mask, v, x,
                                                                        total);
}

void launch_ext_to_compact(cudaStream_t s, const DevGrid *grids, int ngrids, const int8_t *mask,
                           const double *x, double *v, int64_t ncompact, int disc_only,
                           const double *div) {
  ext_to_compact_kernel<<<(unsigned)((ncompact + 255) / 256), 256, 0, s>>>(
      grids, ngrids, mask, x, v, ncompact, disc_only, div);
}

void launch_multidot(int nb, cudaStream_t s, const double *X, int64_t ldx, int nv,
                     const double *y, int64_t n, double *partial, double *out) {
  multidot_partial<<<nb, kRedThreads, 0, s>>>(X, ldx, nv, y, n, partial);
  partial_finish<<<nv, kRedThreads, 0, s>>>(partial, nb, nv, out);
}

void launch_multi_axpy(unsigned nb, cudaStream_t s, const double *X, int64_t ldx, int nv,
                       const double *h, double *y, int64_t n) {
  multi_axpy<<<nb, 256, 0, s>>>(X, ldx, nv, h, y, n);
}

// Y_c = sum_j X_j Z[j + c m] for c < p: a tall basis (m vectors of n values, X_j at X + j ldx)
// times a small m x p matrix (column-major, device).  One thread per row i, kGemmCols output
// columns per block row (blockIdx.y picks the column chunk), that chunk of Z in shared
// memory; X is read once per chunk, coalesced.  Y may not alias X.
constexpr int kGemmCols = 8;
__global__ void __launch_bounds__(256) gemm_tall_kernel(const double *__restrict__ X, int64_t ldx,
                                                         int m, const double *__restrict__ Z,
                                                         int p, double *__restrict__ Y,
                                                         int64_t ldy, int64_t n) {
  extern __shared__ double sz[];  // m x kGemmCols, row j = Z[j, c0 .. c0 + 7]
  const int c0 = blockIdx.y * kGemmCols;
  for (int t = threadIdx.x; t < m * kGemmCols; t += blockDim.x) {
    const int j = t / kGemmCols, c = t % kGemmCols;
    sz[t] = c0 + c < p ? Z[j + (int64_t)(c0 + c) * m] : 0.0;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc[kGemmCols];
#pragma unroll
    for (int c = 0; c < kGemmCols; ++c) acc[c] = 0.0;
    for (int j = 0; j < m; ++j) {
      const double x = X[j * ldx + i];
#pragma unroll
      for (int c = 0; c < kGemmCols; ++c) acc[c] = fma(x, sz[j * kGemmCols + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < kGemmCols; ++c)
      if (c0 + c < p) Y[(c0 + c) * ldy + i] = acc[c];
  }
}

void launch_gemm_tall(cudaStream_t s, const double *X, int64_t ldx, int m, const double *Z,
                      int p, double *Y, int64_t ldy, int64_t n) {
  if (m < 1 || p < 1 || n < 1) return;
  static int attr_bytes = 0;
  const int bytes = m * kGemmCols * (int)sizeof(double);
  if (bytes > 48 * 1024 && bytes > attr_bytes) {
    cudaFuncSetAttribute(gemm_tall_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    attr_bytes = bytes;
  }
  int64_t nb = (n + 255) / 256;
  nb = nb > 152 * 8 ? 152 * 8 : nb;
  const dim3 grid((unsigned)nb, (unsigned)((p + kGemmCols - 1) / kGemmCols));
  gemm_tall_kernel<<<grid, 256, bytes, s>>>(X, ldx, m, Z, p, Y, ldy, n);
}

// out[i] = to_f64(x[i]): the filter's widening, run on its own for testing.
__global__ void widen_kernel(const float *__restrict__ x, double *__restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = to_f64(x[i]);
}

void launch_widen(cudaStream_t s, const float *x, double *y, int64_t n) {
  int64_t nb = (n + 255) / 256;
  nb = nb < 1 ? 1 : (nb > 152 * 16 ? 152 * 16 : nb);
  widen_kernel<<<(unsigned)nb, 256, 0, s>>>(x, y, n);
}

// FP64 FMA throughput probe: every thread runs kChains independent dependent chains
// a <- fma(a, b, c) for `iters` rounds (nothing else in the loop), then stores their sum so
// that no chain is dead code.  2 FLOP per FMA.
constexpr int kChains = 8;
__global__ void __launch_bounds__(256) dfma_probe_kernel(double b, double c, int iters,
                                                         double *out) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  double sum = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) sum += a[k];
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = sum;
}

int64_t launch_dfma_probe(cudaStream_t s, int blocks, int iters, double *out) {
  dfma_probe_kernel<<<blocks, 256, 0, s>>>(0.9999999, 1e-7, iters, out);
  return (int64_t)blocks * 256 * iters * kChains;  // FMAs issued
}

void launch_axpby(unsigned nb, cudaStream_t s, double a, const double *x, double b, double *y,
                  int64_t n) {
  axpby<<<nb, 256, 0, s>>>(a, x, b, y, n);
}

void launch_sub(unsigned nb, cudaStream_t s, const double *x, const double *z, double *y,
                int64_t n) {
  sub<<<nb, 256, 0, s>>>(x, z, y, n);
}

void launch_gemv_acc(unsigned nb, cudaStream_t s, const double *X, int64_t ldx, int nv,
                     const double *c, double *y, int64_t n) {
  gemv_acc<<<nb, 256, 0, s>>>(X, ldx, nv, c, y, n);
}

}  // namespace wh
