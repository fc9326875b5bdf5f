// wh3_internal.h -- the three-dimensional path of libwaveholtz (second order; fourth order on
// Cartesian grids): device data structures, kernel launchers and the host context (not part
// of the ABI).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/waveholtz.h"

namespace wh3 {

// Stencil storage of a 3D grid in the march kernel.
enum Stencil3 : int32_t {
  kConst7 = 0,   // Cartesian grid, c = 1: four constant weights in Grid3Dev::cw
  kPoint7 = 1,   // per-point weights on the 7-point cross (all axis pairs orthogonal, or c(x))
  kPoint19 = 2,  // per-point weights on the 19-point box (a non-orthogonal axis pair)
  kConst13 = 3,  // fourth order, Cartesian grid, c = 1: seven constant weights in cw
  kPoint13 = 4   // fourth order, Cartesian grid with c(x): per-point weights, 13 planes
};
// Per-point weight planes, in this order: centre (with the "2"), then the face neighbours
// -x +x -y +y -z +z, then (kPoint19) the edge neighbours of pairs (x,y), (x,z), (y,z), each
// as (-,-) (+,-) (-,+) (+,+).
// kPoint13: centre, then per axis a the offsets -1, +1, -2, +2 (planes 1 + 4a .. 4 + 4a).
constexpr int kNw7 = 7, kNw19 = 19, kNw13 = 13;
// Coefficient planes of curvilinear grids (c^2 folded in).
enum { kA00 = 0, kA11, kA22, kA01, kA02, kA12, kB0, kB1, kB2, kNcoef };

// March block: 32 x 8 threads, each marching kTZ points along axis 2.
constexpr int kTX = 32, kTY = 8, kTZ = 8;

// One component grid in device memory.  Extended arrays (ghosts included, ghost width p/2 on
// non-periodic axes at order p) are stored with axis 0 fastest: (i, j, k) is at
// base + ((k + g2) * e1 + (j + g1)) * e0 + (i + g0).
struct Grid3Dev {
  int32_t n0, n1, n2;
  int32_t g0, g1, g2;
  int32_t e0, e1, e2;
  int32_t per;      // bit a: axis a periodic
  int32_t stencil;  // Stencil3
  int32_t nw;       // weight planes (point stencils)
  int32_t kind;     // WH_CARTESIAN / WH_CURVILINEAR
  int32_t ortho;    // orthogonal axis pairs: bit 0 (0,1), bit 1 (0,2), bit 2 (1,2)
  int64_t base;     // offset of the extended array in the state arrays
  int64_t ext;      // e0 * e1 * e2
  int64_t cbase;    // offset in compact vectors
  int64_t wbase;    // offset of weight plane 0 (plane stride ext)
  int64_t kbase;    // offset of coefficient plane 0 (plane stride ext), curvilinear only
  int64_t rbase;    // offset of metric plane 0 (9 planes, stride ext), curvilinear only
  double h[3];
  double cw[7];     // kConst7: centre, axis-0, axis-1, axis-2 neighbour weights (dt^2
                    // folded); kConst13: centre, then per axis a the +-1 and +-2 weights
                    // at 1 + 2a and 2 + 2a
  float cwf[7];     // the same rounded to FP32
};

// One march tile: 32 x 8 points of the (axis 0, axis 1) plane, kTZ planes deep.
struct Tile3 {
  int32_t grid, i0, j0, k0;
};

// Temporal blocking of the FP32 march (constant-weight, non-periodic grids): a unit is a
// box of kTX x kUY points of the (axis 0, axis 1) plane and up to `depth` planes along axis 2
// (a union of march tiles) that advances K time steps in one launch from the two levels
// before them, recomputing a K-point halo (overlapped tiling).  Its (K-1)-dilated box holds
// no receiver and no ghost that a rule rewrites, so every point the K steps read is either
// marched or constant.  flags bit 0: write every intermediate level (a coupled tile or a
// donor reads them), else only the last two.
constexpr int kUY = 16;
struct Unit3 {
  int32_t grid, i0, j0, k0, nz, flags;
};

// Fourth-order ghost rule of one boundary point of a Dirichlet or Neumann face: the points
// along the inward normal are U_k = W[q0 + k s], k = 0..3, the ghosts G1 = W[q0 - s] and
// G2 = W[q0 - 2 s].  a2 = c^2 / (12 h_n^2) of the boundary point for a Dirichlet face, 0
// for a Neumann face.
struct Ghost4 {
  int64_t q0;
  int64_t s;
  double a2;
};

// Per-step tables of the prepared frequency.
struct Tab3 {
  const double *fc;  // dt^2 cos(omega_e t^n), n = 0..M
  const double *wf;  // filter weights of level n
  const float *fcf;  // fc rounded to FP32
  double dt2h;       // dt^2 / 2
  float dt2hf;
};

// Launchers (wh_kernels3.cu).  T is double unless fp32; void pointers carry T arrays.
void launch_coef3(cudaStream_t s, const Grid3Dev *grids, int gidx, const Grid3Dev &G,
                  const int8_t *mask, const double *rx, const double *c2, double *coef,
                  unsigned long long *smax);
void launch_weight3(bool fp32, cudaStream_t s, const Grid3Dev *grids, int gidx,
                    const Grid3Dev &G, const int8_t *mask, const double *coef, const double *c2,
                    void *Wt, double dt2);
void launch_init3(bool fp32, cudaStream_t s, const Grid3Dev *grids, int ngrids,
                  int64_t max_ext, const int8_t *mask, const double *v, void *W0, double *V,
                  const double *wf);
// One step n -> n + 1 over `tiles`: W^{n+1} -> Wout from W^n (Wn) and W^{n-1} (Wprev, which
// may be Wout itself: the two-level in-place layout).
void launch_march3(bool fp32, cudaStream_t s, int ntiles, const Grid3Dev *grids,
                   const Tile3 *tiles, const int8_t *mask, const void *Wn, const void *Wprev,
                   void *Wout, const void *F, const void *Wt, double *V, Tab3 tab, int n,
                   double fs);
// K steps n -> n + K (K = 2, 3 or 4) of the FP32 march over `nunits` units.  ring holds L
// levels of the FP32 state, level l at ring + (l % L) * stride; levels n - 1 and n are read,
// levels n + 1 .. n + K written (only n + K - 1 and n + K for units without the export
// flag).  FM: the FP32 forcing at discretization points, NaN elsewhere
// (launch_forcing_mask).  Same arithmetic, in the same order, as launch_march3's.
void launch_march3_block(int K, cudaStream_t s, int nunits, const Grid3Dev *grids,
                         const Unit3 *units, const float *FM, float *ring, int64_t stride,
                         int L, double *V, Tab3 tab, int n, double fs);
void launch_forcing_mask(cudaStream_t s, const float *F, const int8_t *mask, float *FM,
                         int64_t n);
size_t march3_block_threads(int K);
// Receiver r of R: donor (i0 + a, j0 + b, k0 + c) at gbase[r] + goff[a R + r] +
// goff[(3 + b) R + r] + goff[(6 + c) R + r] with weight gw[a R + r] gw[(3 + b) R + r]
// gw[(6 + c) R + r] (planes of wx, wy, wz).
void launch_gather3(bool fp32, cudaStream_t s, int64_t nrecv, int64_t nghost,
                    const int64_t *ridx, const int32_t *gbase, const int32_t *goff,
                    const double *gw, const int32_t *gdst, const int32_t *gsrc, void *W,
                    double *V, const double *wf, int level);
void launch_finish3(cudaStream_t s, const Grid3Dev *grids, int ngrids, int64_t max_compact,
                    const double *V, double *vout);
// Dirichlet points with boundary data at one level: W[idx[t]] = gfac g[t], V += wf[level] W.
void launch_dirichlet3(bool fp32, cudaStream_t s, int64_t n, const int64_t *idx,
                       const double *g, void *W, double *V, double gfac, const double *wf,
                       int level);
// Fourth order (Cartesian grids): per-point weights of kPoint13 grids, one step of the
// 13-point march (same arguments as launch_march3), and the level's ghost rules and
// width-5 interpolation: receiver r's donor (i0 + a, j0 + b, k0 + c) at gbase[r] +
// goff[a R + r] + goff[(5 + b) R + r] + goff[(10 + c) R + r], weights likewise in gw;
// each Ghost4 item solves its two ghosts with the forcing term fcl F[q0] (fcl = the forcing
// switch times cos(omega_e t^level); F the FP64 forcing in the state layout).
void launch_weight3o4(bool fp32, cudaStream_t s, const Grid3Dev *grids, int gidx,
                      const Grid3Dev &G, const int8_t *mask, const double *c2, void *Wt,
                      double dt2);
void launch_march3o4(bool fp32, cudaStream_t s, int ntiles, const Grid3Dev *grids,
                     const Tile3 *tiles, const int8_t *mask, const void *Wn, const void *Wprev,
                     void *Wout, const void *F, const void *Wt, double *V, Tab3 tab, int n,
                     double fs);
void launch_gather3o4(bool fp32, cudaStream_t s, int64_t nrecv, int64_t nitems,
                      const int64_t *ridx, const int32_t *gbase, const int32_t *goff,
                      const double *gw, const Ghost4 *items, const double *F, double fcl,
                      void *W, double *V, const double *wf, int level);
// vout (compact) = W (extended, FP64) at discretization points, zero elsewhere.
void launch_disc3(cudaStream_t s, const Grid3Dev *grids, int ngrids, int64_t max_compact,
                  const int8_t *mask, const double *W, double *vout);
void launch_to_precision(bool fp32, cudaStream_t s, const double *src, void *dst, int64_t n);

// Host context of a three-dimensional problem (wh_api3.cu).
struct Ctx3;
Ctx3 *create();
void destroy(Ctx3 *c);
wh_status add_grid(Ctx3 *c, const wh_grid3_desc *d, int order, int32_t *id, std::string &err);
wh_status set_interp(Ctx3 *c, const wh_interp3_desc *d, std::string &err);
wh_status set_forcing(Ctx3 *c, int32_t gid, const double *f, std::string &err);
// Dirichlet boundary data of one grid (compact, read at its Dirichlet points; null removes
// them): those points hold g cos(omega_e t) while the forcing is on.
wh_status set_boundary_data(Ctx3 *c, int32_t gid, const double *g, std::string &err);
bool has_boundary_data(const Ctx3 *c);
// Prepare one frequency: upload (first time), coefficients, CFL bound, time tables, stencil
// weights; with fp32 also the FP32 march arrays.  Returns the time setup and sizes.
wh_status prepare(Ctx3 *c, const wh_options &opt, double omega, cudaStream_t s,
                  wh_time_info *ti, int64_t *ncompact, int64_t *nactive, std::string &err);
// v_out = W_h(v_in, f or 0) on the device with the FP64 or the FP32 march.
wh_status iterate(Ctx3 *c, bool fp32, int forcing, const double *vin, double *vout,
                  cudaStream_t s, int64_t *launches, std::string &err);
int ngrids(const Ctx3 *c);
// The masks (WH_DISC, ...) and the forcing (zero where none was set) of every grid in the
// compact order (grids one after another, each (n2, n1, n0) row-major).
void compact_mask(const Ctx3 *c, std::vector<int8_t> &m);
void compact_forcing(const Ctx3 *c, std::vector<double> &f);
// One first step of the FP64 march from y (compact) with zero forcing and the ghost rules
// applied to y (no interpolation): wy = y and w1 = W^1 = y + dt^2/2 c^2 L_h y, both at
// discretization points and zero elsewhere (compact).  Uses the FP64 state and filter
// arrays as scratch.
wh_status first_step(Ctx3 *c, const double *y, double *wy, double *w1, cudaStream_t s,
                     std::string &err);
// Temporal blocking of the FP32 march: depth K in [1, 4] (1 = single steps) and unit depth
// (planes, a multiple of 8 in [8, 256]); -1 = the library's choice.  Takes effect at once
// when the FP32 march is prepared, else at the next prepare.
wh_status set_blocking(Ctx3 *c, int K, int uz, std::string &err);
// The plan in use: depth, unit depth, points and units that advance K steps per launch.
void blocking(const Ctx3 *c, int *K, int *uz, int64_t *points, int64_t *units);
// Device time per launch (ms) and launches per iteration of [0] the single-step march, [1]
// the ghost-rule + interpolation kernel and [2] the K-step blocked march, each launch timed
// on its own with events over reps iterations.
wh_status profile(Ctx3 *c, bool fp32, cudaStream_t s, int reps, double *ms, int32_t *counts,
                  std::string &err);

}  // namespace wh3
