// wh_internal.h -- device-side data structures of libwaveholtz (not part of the ABI).
#pragma once
#include <cstdint>
#include <cuda.h>  // CUtensorMap (type only; maps are encoded through the runtime entry point)
#include <cuda_runtime.h>

#include <complex>
#include <vector>

namespace wh {

constexpr int kMaxOrder = 4;
constexpr int kTileX = 32;  // march block: 32 x 8 threads
constexpr int kTileY = 8;
constexpr int kPY = 4;      // points per thread along axis 1: a 32 x 32 tile per block

// Stencil storage of a grid in the march kernels.
enum StencilKind : int32_t {
  kConstCross = 0,  // Cartesian, constant c: weights in DevGrid::cw
  kPointCross = 1,  // per-point weights on the 2p+1 cross (orthogonal grids, c(x))
  kPointBox = 2     // per-point weights on the (p+1)^2 box (non-orthogonal grids)
};

// One component grid in device memory.  Extended arrays (ghosts included) are stored
// row-major with row stride `pitch`; element (i, j), i in [-g0, n0+g0), starts at
// base + (j + g1) * pitch + (i + g0).
struct DevGrid {
  int32_t n0, n1, g0, g1;
  int32_t pitch;
  int32_t per0, per1;       // periodic axes
  int32_t stencil;          // StencilKind
  int32_t nw;               // weights per point (per-point stencils)
  int32_t kind;             // WH_CARTESIAN / WH_CURVILINEAR
  int32_t ortho;
  int32_t inst;             // instance (independent Helmholtz problem) of this grid
  int64_t base;             // offset of the extended array in the state arrays
  int64_t ext;              // pitch * (n1 + 2 g1)
  int64_t cbase;            // offset in compact vectors
  int64_t wbase;            // offset of weight plane 0 in the weight array (stride ext)
  int64_t kbase;            // offset of coefficient plane 0 (5 planes, stride ext)
  double h0, h1;
  // constant cross weights (kConstCross), dt^2 folded in, centre includes the "2":
  // [centre, axis0 offset 1, axis0 offset 2, axis1 offset 1, axis1 offset 2]
  double cw[5];
  float cwf[5];  // the same weights rounded to FP32 (the FP32 march reads these)
  // Dirichlet boundary data g (FP64, indexed by state index like the state arrays), or
  // null when the grid has none: Dirichlet points then hold g cos(omega_e t) with the
  // forcing on
  const double *gb;
};

// One ghost-rule item: the ghost points next to one boundary point (Sec. 3.2 ghost
// rules; see the library source for the formulas).
struct BcItem {
  int64_t u[4];      // state indices of U0..U3 (boundary point and three inward)
  int64_t g[2];      // state indices of G1, G2 (G2 unused at order 2)
  int32_t type;      // 0: Neumann order 2, 1: Neumann order 4, 2: Dirichlet order 4
  int32_t inst;      // instance of the item's grid
  double A2, B1;     // Dirichlet order 4: a_nn/(12 h^2), +-b_n/(12 h) (c^2 folded)
  double inv;        // 1 / (11 A2 - 3 B1)
  double fg;         // Dirichlet order 4 with boundary data: -omega^2 g_b - c^2 (D_tt g)_b,
                     // added to f_b on the compatibility condition's right side (0 without)
};

// Time tables of one instance on the device (Recipe OmegaTildeExplicit per instance).
struct InstDev {
  const double *fc;    // dt^2 cos(omega_e t^n), n = 0..M
  const double *cosn;  // cos(omega_e t^n)
  const double *wf;    // filter weights of level n
  double dt2;
  int M;               // steps of one iteration; steps n >= M are skipped
  int active;          // 0: the instance is skipped entirely (converged in a batched solve)
  const float *fcf;    // fc rounded to FP32 (the FP32 march reads these)
  float dt2hf;         // dt^2 / 2 rounded to FP32 (first step)
};

// One tile of the march: a 32 x (8 kPY) block of points of one grid.  For tiles of the
// TMA-staged march, pad_ is the index of the grid's block of tensor maps.
struct Tile {
  int32_t grid, i0, j0, pad_;
};

// TMA-staged march (non-periodic grids with constant cross weights, ghost width = order/2):
// per grid 7 tensor maps over its extended arrays; every box is kBoxX elements wide starting
// at extended column i0 (= grid column i0 - order/2, 16-byte aligned since i0 % 32 == 0).
enum { kMapWaHalo = 0, kMapWbHalo, kMapWaCtr, kMapWbCtr, kMapF, kMapV, kMapMask, kMapsPerGrid };
constexpr int kBoxX = 36;      // state/forcing/filter box columns (tile 32 + halo 2 x 2)
constexpr int kMaskBoxX = 48;  // mask box columns (bytes; 16-byte multiple covering 2 + 32)

// Grid-wide barrier state of the persistent kernel (zeroed before every launch); each
// word on its own 128-byte line.
struct GridBarrier {
  unsigned count[32];
  unsigned gen[32];
  int err[32];
  unsigned long long ticket[16];  // dataflow tickets: ticket k is step k / ntiles, tile k % ntiles
};

// The ghost rules and interpolation of level n + 1 folded into the march launch of step n
// (nunits = 0: not folded).  Unit u (as a block of the separate kernel) runs after the tiles
// udep_tile[udep_off[u] .. udep_off[u+1]) have written level n + 1 (tile_done >= n + 1);
// tiles whose Tile::pad_ is 1 signal.  tile_done is zero at the start of each iteration.
struct GatherArgs {
  const BcItem *bc;
  const int32_t *didx;
  const double *dw;
  const int64_t *ridx;
  const int32_t *rinst;
  const int64_t *udep_off;
  const int32_t *udep_tile;
  int32_t *tile_done;
  int *err;
  // march tiles by ticket (non-null: ctl[1] next ticket, ctl[2] blocks done; the last
  // block out resets both) instead of the fixed grid stride
  int *ctl;
  unsigned long long spin_limit;
  int nbc, bc_blocks, nunits, nrecv;
};

// Everything the persistent iteration kernel reads (device pointers, per-step tables).
struct IterArgs {
  const DevGrid *grids;
  int ngrids;
  int ntiles;
  const Tile *tiles;
  const int8_t *mask;
  void *Wa, *Wb;
  const void *F, *Wt;
  double *V;
  const BcItem *bc;
  int64_t nbc;
  const int32_t *didx;
  const double *dw;
  const int64_t *ridx;
  int64_t nrecv;
  const InstDev *inst;
  const int32_t *rinst;  // instance of each receiver
  double fs;             // 1 with forcing, 0 without
  int M;                 // largest instance M
  int pad_;
  int64_t total, ncompact;
  unsigned long long spin_limit;
  // per-tile patch lists: entries [patch_off[t], patch_off[t+1]) of tile t; patch_pos holds
  // (kind << 24) | shared-memory index, kind 0/1 = ghost G1/G2 of BC item patch_item,
  // kind 2 = receiver patch_item
  const int64_t *patch_off;
  const int32_t *patch_pos;
  const int32_t *patch_item;
  const int32_t *recv_of;  // receiver index at each extended point, -1 elsewhere
  // dataflow: tile t at step n waits until tile_done[d] >= n for d in
  // dep_tile[dep_off[t] .. dep_off[t+1]), and sets tile_done[t] = n + 1 when done
  const int64_t *dep_off;
  const int32_t *dep_tile;
  int32_t *tile_done;
};

// Host launchers (wh_kernels.cu).  T is double unless fp32 is set; pointers typed void
// carry T arrays.
// While on, launches of the iteration graph's kernels (march, TMA march, ghost rules +
// interpolation) made from this thread ask for programmatic dependent launch.
void set_pdl(bool on);
void launch_march(bool fp32, int order, bool first, int nblocks, int ntiles, cudaStream_t s,
                  const DevGrid *grids, const Tile *tiles, const int8_t *mask, const void *Wn,
                  void *Wout, const void *F, const void *Wt, double *V, const InstDev *inst,
                  int n, double fs, const void *Wprev = nullptr,  // W^{n-1}: Wout if null
                  const GatherArgs *gather = nullptr);            // fold level n + 1's gather
int march_blocks_per_sm(bool fp32, int order);
// TMA-staged march, one launch per step: each block walks a strided share of the fast tiles
// (double-buffered TMA boxes on mbarriers, bounded waits), then takes general tiles by
// ticket (as launch_march).  Same arithmetic, in the same order.  ctl: int[3] in device memory, zero before the first
// launch (error flag, ticket counter, blocks done; the kernel leaves the last two at zero).
size_t march_tma_smem(bool fp32, int order);
int march_tma_blocks_per_sm(bool fp32, int order);
void launch_march_tma(bool fp32, int order, bool first, int nblocks, cudaStream_t s,
                      const DevGrid *grids, const Tile *ftiles, int nfast, const CUtensorMap *maps,
                      const Tile *gtiles, int ngen, const int8_t *mask, void *Wa, void *Wb,
                      const void *F, const void *Wt, double *V, const InstDev *inst, int n,
                      double fs, int *ctl, unsigned long long spin_limit,
                      const GatherArgs *gather = nullptr);  // fold level n + 1's gather
void launch_bc_gather(bool fp32, int order, int blocks, cudaStream_t s, const BcItem *bc,
                      int nbc, int bc_blocks, const int32_t *didx, const double *dw,
                      const int64_t *ridx, const int32_t *rinst, int nrecv, void *W,
                      const void *F, const InstDev *inst, int level, double fs);
int iteration_blocks_per_sm(bool fp32, int order);
cudaError_t launch_iteration(bool fp32, int order, int nblocks, cudaStream_t s,
                             const IterArgs &A, const double *v_in, double *v_out,
                             GridBarrier *bar);
void launch_init(bool fp32, unsigned blocks, cudaStream_t s, const DevGrid *grids, int ngrids,
                 const int8_t *mask, const double *v, void *W0, double *V, int64_t total,
                 const InstDev *inst, double fs);
void launch_finish(bool fp32, unsigned blocks, cudaStream_t s, const DevGrid *grids, int ngrids,
                   const int8_t *mask, const double *V, const void *Wa, const void *Wb,
                   const InstDev *inst, double *vout, int64_t ncompact);
void launch_coef(int order, dim3 gb, dim3 tb, cudaStream_t s, const DevGrid *grids, int gidx,
                 const int8_t *mask, const double *rx, const double *c2, double *coef,
                 unsigned long long *smax);
void launch_weight(bool fp32, int order, dim3 gb, dim3 tb, cudaStream_t s, const DevGrid *grids,
                   int gidx, const int8_t *mask, const double *coef, const double *c2, void *Wt,
                   double dt2);
void launch_bc_coef(int nbc, cudaStream_t s, BcItem *bc, const int32_t *ig, const int32_t *ia,
                    const int32_t *ih, const DevGrid *grids, const double *coef,
                    const double *c2);
void launch_adj_step(int order, cudaStream_t s, const DevGrid *grids, int ngrids,
                     const int8_t *mask, const double *Wt, const double *lam, double wn,
                     double sc, const double *Z1, const double *Z2, double *Y, double *Znew,
                     int64_t total, const double *Xprev, const double *Xn, const double *Xnext,
                     const double *F, double fc, double *gc2, double *gf);
// Z += the constraint part of D C^T Y at the listed points; with gc2 non-null also the
// Dirichlet compatibility gradient terms of this level (fcos = cos(omega_e t^n)).
void launch_adj_post(cudaStream_t s, const int64_t *fq, const int64_t *foff, const int64_t *rpos,
                     const double *rcoef, const double *Y, double *Z, int64_t nfix,
                     const BcItem *bc, int nbc, const double *F, double fcos, double *gc2,
                     double *gf);
void launch_compact_to_ext(cudaStream_t s, const DevGrid *grids, int ngrids, const int8_t *mask,
                           const double *v, double *x, int64_t total);
void launch_ext_to_compact(cudaStream_t s, const DevGrid *grids, int ngrids, const int8_t *mask,
                           const double *x, double *v, int64_t ncompact, int disc_only,
                           const double *div = nullptr);
constexpr int kRedThreads = 256;
void launch_multidot(int nb, cudaStream_t s, const double *X, int64_t ldx, int nv,
                     const double *y, int64_t n, double *partial, double *out);
void launch_multi_axpy(unsigned nb, cudaStream_t s, const double *X, int64_t ldx, int nv,
                       const double *h, double *y, int64_t n);
void launch_axpby(unsigned nb, cudaStream_t s, double a, const double *x, double b, double *y,
                  int64_t n);
void launch_sub(unsigned nb, cudaStream_t s, const double *x, const double *z, double *y,
                int64_t n);
void launch_gemv_acc(unsigned nb, cudaStream_t s, const double *X, int64_t ldx, int nv,
                     const double *c, double *y, int64_t n);
// Y_c = sum_{j < m} X_j Z[j + c m], c < p (tall basis times a small column-major matrix on
// the device; m <= 2048; Y may not alias X)
void launch_gemm_tall(cudaStream_t s, const double *X, int64_t ldx, int m, const double *Z,
                      int p, double *Y, int64_t ldy, int64_t n);
// Eigenvalues w (complex) and unit eigenvectors V (complex, column i for w[i], row-major
// m x m) of the real m x m row-major matrix A (host, wh_dense.cpp); false if the QR
// algorithm does not converge.
bool dense_eig(int m, const double *A, std::vector<std::complex<double>> &w,
               std::vector<std::complex<double>> &V);
// A real orthonormal basis Q (column-major m x p) of the invariant subspace of the `want`
// eigenvalues of largest modulus of the real m x m row-major A (a complex pair kept whole),
// from its complex Schur form reordered to put them first, widened to the real span of
// that subspace and its conjugate (so p >= want: one more per nearly real conjugate pair
// split by the selection); w gets the selected eigenvalues.  Returns p, or -1 if the QR
// algorithm does not converge.
int invariant_basis(int m, const double *A, int want, std::vector<double> &Q,
                    std::vector<std::complex<double>> &w);
// y[i] = the filter's FP32 -> FP64 widening of x[i] (testing aid)
void launch_widen(cudaStream_t s, const float *x, double *y, int64_t n);
// FP64 FMA throughput probe (blocks x 256 threads, out: one double per thread); returns the
// number of FMAs issued
int64_t launch_dfma_probe(cudaStream_t s, int blocks, int iters, double *out);

}  // namespace wh
