// wh_api.cu -- host side of libwaveholtz: the C ABI declared in include/waveholtz.h.
//
// Responsibilities: validate and upload the overset grid description, prepare one
// frequency (operator coefficients and stability bound on the device, the explicit time
// correction of Recipe OmegaTildeExplicit, alpha_d of Eq. alphad, per-point stencil
// weights, per-step tables), issue one WaveHoltz iteration as a CUDA graph of
// 2M + 1 kernels (M time steps of Algorithm 2) plus an input and an output kernel, and
// drive the fixed-point iteration (Algorithm 1) or GMRES (Sec. 4.3).
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/waveholtz.h"
#include "wh_internal.h"
#include "wh3_internal.h"

using namespace wh;

namespace {

struct HostGrid {
  wh_grid_desc d;
  std::vector<int8_t> mask;
  std::vector<double> rx, c2, f;
  std::vector<double> gdata;  // Dirichlet boundary data (compact), empty when none
  int g0 = 0, g1 = 0;
};

// The arrays of one march precision: state levels, forcing, stencil weights and the two
// captured iteration graphs (forcing off / on).
struct MarchSet {
  void *Wa = nullptr, *Wb = nullptr, *F = nullptr, *Wt = nullptr;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  bool fp32 = false, present = false;
  int march_blocks = 0, iter_blocks = 0;
  // TMA-staged march: tensor maps of the fast grids over this set's arrays
  CUtensorMap *maps = nullptr;
  bool tma = false;
  int tma_blocks = 0;
};

}  // namespace

struct wh_ctx {
  wh_options opt{};
  // 0 until the first grid is added, then 2 or 3; three-dimensional problems live in c3
  int dim = 0;
  // deflation set of wh_solve(WH_FPI): caller-owned device eigenvectors, host eigenvalues,
  // and the compact forcing for the final inflation
  int defl_k = 0;
  const double *defl_phi = nullptr;
  std::vector<double> defl_lam2;
  double *d_fcompact = nullptr;
  bool defl_on = false;  // apply_A projects the set out of W_h(x, 0) (deflated GMRES)
  // the set as an S-invariant basis with its Rayleigh matrix T = Q^T S Q (row-major k x k):
  // the inflation is then exact, u = v + Q (I - T)^{-1} Q^T W_h(v, f)
  bool defl_basis = false;
  std::vector<double> defl_T;
  // a solve that stopped at its product budget, for wh_get_state, or one loaded by
  // wh_set_state for the next wh_solve to continue (resume)
  struct SavedSolve {
    bool valid = false, resume = false;
    int method = 0, restart = 0, phase = 0;  // phase 1: FP32 wave solves of an FP32 context
    int products[2] = {0, 0};
    int fpi_k = 0;
    double bnorm = 0.0, prev = 0.0, residual = 0.0, dmin = 0.0;
    bool cycle = false;  // stopped inside an Arnoldi cycle after kk steps
    int kk = 0;
    double beta = 0.0;
    std::vector<double> H, cs, sn, g;
  } saved;
  double *d_saved = nullptr;  // device: [0] the iterate (the cycle's start inside a cycle), [1] b
  wh3::Ctx3 *c3 = nullptr;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  std::string err;
  std::vector<HostGrid> grids;
  // interpolation (host copies)
  int64_t nrecv = 0;
  std::vector<int32_t> rg, ri, rj, dg, di, dj;
  std::vector<double> wx, wy;
  // device layout
  bool dirty = true;
  bool prepared = false;
  int64_t total = 0;     // extended points, all grids (with alignment gaps)
  int64_t ncompact = 0;  // compact vector length
  int64_t nactive = 0;
  int64_t nplanes5 = 0, nweights = 0;
  std::vector<DevGrid> hgrids;
  std::vector<Tile> htiles;
  // march tiles split for the TMA-staged march: fast (non-periodic constant-weight grids,
  // pad_ = the grid's map slot) and general
  std::vector<Tile> hftiles, hgtiles;
  std::vector<int32_t> fast_grids;  // grid of each map slot
  Tile *d_ftiles = nullptr, *d_gtiles = nullptr;
  // batches: the same tile lists ordered by their instance's step count M (descending), so
  // that the tiles of the instances still marching at step n form a prefix; mpre_*[n] is
  // its length.  Used by the graph path when the gather is not folded (the folded gather
  // numbers tiles in the original lists).
  Tile *d_tiles_m = nullptr, *d_ftiles_m = nullptr, *d_gtiles_m = nullptr;
  std::vector<int32_t> mpre_t, mpre_f, mpre_g;
  bool msorted = false;
  // the same for the separate ghost-rule + interpolation launch: items and receivers by
  // descending M, prefix lengths per level (level L runs for instances with M >= L); the
  // host copies of the receivers' donor lists that the ordering starts from
  BcItem *d_bc_m = nullptr;
  // Dirichlet boundary data of every grid in the state layout (null when no grid has any)
  double *d_gb = nullptr;
  int32_t *d_didx_m = nullptr, *d_rinst_m = nullptr;
  double *d_dw_m = nullptr;
  int64_t *d_ridx_m = nullptr;
  std::vector<int32_t> mpre_bc, mpre_r;
  std::vector<int32_t> h_didx, h_rinst;
  std::vector<double> h_dw;
  std::vector<int64_t> h_ridx;
  // march control: [0] sticky error flag, [1] tile ticket, [2] blocks done
  int *d_err = nullptr;
  // launch layout fixed by wh_set_tuning / wh_autotune (-1: the library's choice)
  int tune_fold = -1, tune_tickets = -1, tune_tma = -1, tune_pdl = -1;
  // ghost rules + interpolation folded into the march launch (march_kernel sets)
  int nunits = 0;
  std::vector<int64_t> udep_off;
  std::vector<int32_t> udep_tile;
  int64_t *d_udep_off = nullptr;
  int32_t *d_udep_tile = nullptr;
  // the same dependencies numbered as the TMA-staged march's tiles (fast, then general)
  std::vector<int32_t> udep_tile_tma;
  int32_t *d_udep_tile_tma = nullptr;
  std::vector<BcItem> hbc;
  std::vector<int32_t> hbc_grid, hbc_axis, hbc_hi;
  std::vector<void *> allocs;
  DevGrid *d_grids = nullptr;
  Tile *d_tiles = nullptr;
  int8_t *d_mask = nullptr;
  // the active march set's arrays (mirrors of set[active]); set[0] is FP64, set[1] the
  // FP32 march of WH_FP32 contexts
  void *d_Wa = nullptr, *d_Wb = nullptr, *d_F = nullptr, *d_Wt = nullptr;
  MarchSet set[2];
  int active = 0;
  double *d_V = nullptr, *d_c2 = nullptr, *d_rx = nullptr, *d_coef = nullptr;
  BcItem *d_bc = nullptr;
  int32_t *d_bc_grid = nullptr, *d_bc_axis = nullptr, *d_bc_hi = nullptr;
  int32_t *d_didx = nullptr;
  double *d_dw = nullptr;
  int64_t *d_ridx = nullptr;
  unsigned long long *d_smax = nullptr;
  // time setup: one per instance (ti mirrors instance 0)
  wh_time_info ti{};
  int ninst = 1;
  std::vector<wh_time_info> iti;
  std::vector<int64_t> icstart, icend, inact;  // compact segment and active points
  std::vector<InstDev> hinst;                  // device structs (device table pointers)
  std::vector<int8_t> iactive;
  InstDev *d_inst = nullptr;
  double *d_tabs = nullptr;
  float *d_ftabs = nullptr;  // per instance fc[0..M] rounded to FP32
  int64_t tabs_cap = 0;
  int32_t *d_rinst = nullptr;
  int maxM = 0;
  // differentiation: transpose constraint lists (CSR over the discretization points that
  // constrained positions read: d_fq the points, d_roff their entry ranges) and buffers;
  // built on the first adjoint call after wh_prepare
  bool adj_ready = false;
  bool adjoint_mode = false;  // apply_A uses S^T (adjoint GMRES)
  int64_t nfix = 0;
  int64_t *d_fq = nullptr, *d_roff = nullptr, *d_rpos = nullptr;
  double *d_rcoef = nullptr;
  double *d_adj = nullptr;   // lam, Y, Z x3, gc2, gf (extended)
  double *d_ckpt = nullptr;  // checkpoints and segment states
  int64_t ckpt_cap = 0;
  cudaGraphExec_t adj_graph = nullptr;  // the S^T sweep (lam -> Z^0), captured once
  double *adj_z0 = nullptr;              // where that graph leaves Z^0
  double *d_traj = nullptr;  // the whole forward trajectory X^0 .. X^M (when it fits)
  int64_t traj_cap = 0;

  // solver workspace
  double *d_q = nullptr;  // Krylov basis
  int64_t q_cap = 0;
  double *d_work = nullptr;  // 3 vectors
  double *d_partial = nullptr, *d_red = nullptr;
  int partial_blocks = 0, red_cap = 0;
  int64_t launches = 0;
  int march_blocks = 0;
  // persistent path
  int iter_blocks = 0;
  GridBarrier *d_bar = nullptr;
  int *h_err = nullptr;       // pinned copy of the barrier error flag
  int64_t *d_patch_off = nullptr;
  int32_t *d_patch_pos = nullptr, *d_patch_item = nullptr, *d_recv_of = nullptr;
  int64_t *d_dep_off = nullptr;  // dataflow dependencies of each tile (CSR)
  int32_t *d_dep_tile = nullptr;
  int32_t *d_tile_done = nullptr;  // steps completed by each tile in the current launch
  bool persistent = true;
  bool fold_failed = false;  // a folded launch timed out: use the separate gather kernel
  unsigned long long opt_spin_limit = 1ull << 22;
  cudaEvent_t err_ev = nullptr;
  bool err_pending = false;
};

namespace {

constexpr int kWorkVectors = 5;

wh_status fail(wh_ctx *c, wh_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(ctx, WH_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

template <typename T>
wh_status dalloc(wh_ctx *ctx, T **p, size_t n) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
  if (e != cudaSuccess)
    return fail(ctx, WH_ERR_NOMEM, "cudaMalloc of %zu bytes failed: %s", n * sizeof(T),
                cudaGetErrorString(e));
  ctx->allocs.push_back((void *)*p);
  // the zero fill runs on the legacy stream, which the context's non-blocking stream does
  // not wait for: finish it here so that no later copy or kernel can be overtaken by it
  e = cudaMemset(*p, 0, n * sizeof(T));
  if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
  if (e != cudaSuccess) return fail(ctx, WH_ERR_CUDA, "cudaMemset: %s", cudaGetErrorString(e));
  return WH_OK;
}

// Host-to-device copy ordered on the context's stream; returns once the copy is complete,
// so the host buffer may be released and every later launch on the stream sees the data.
wh_status h2d(wh_ctx *ctx, void *dst, const void *src, size_t bytes) {
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return WH_OK;
}

// Free one buffer from dalloc before the context is reset.
template <typename T>
void dfree(wh_ctx *ctx, T **p) {
  if (!*p) return;
  for (size_t k = 0; k < ctx->allocs.size(); ++k)
    if (ctx->allocs[k] == (void *)*p) {
      ctx->allocs.erase(ctx->allocs.begin() + k);
      break;
    }
  cudaFree(*p);
  *p = nullptr;
}

void drop_graphs(wh_ctx *ctx) {
  for (auto &S : ctx->set)
    for (auto &g : S.gexec)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
  if (ctx->adj_graph) {
    cudaGraphExecDestroy(ctx->adj_graph);
    ctx->adj_graph = nullptr;
  }
}

void free_device(wh_ctx *ctx) {
  drop_graphs(ctx);
  for (auto &S : ctx->set) {
    S.Wa = S.Wb = S.F = S.Wt = nullptr;
    S.present = false;
  }
  for (void *p : ctx->allocs) cudaFree(p);
  ctx->allocs.clear();
  ctx->d_grids = nullptr;
  ctx->d_q = nullptr;
  ctx->q_cap = 0;
  ctx->d_work = nullptr;
  ctx->d_partial = ctx->d_red = nullptr;
  ctx->red_cap = 0;
  ctx->d_tabs = nullptr;
  ctx->d_ftabs = nullptr;
  ctx->tabs_cap = 0;
  ctx->adj_ready = false;
  ctx->nfix = 0;
  ctx->d_fq = ctx->d_roff = ctx->d_rpos = nullptr;
  ctx->d_rcoef = ctx->d_adj = ctx->d_ckpt = ctx->d_traj = nullptr;
  ctx->ckpt_cap = ctx->traj_cap = 0;
  ctx->d_bar = nullptr;
  ctx->d_tiles_m = ctx->d_ftiles_m = ctx->d_gtiles_m = nullptr;
  ctx->d_gb = nullptr;
  ctx->d_bc_m = nullptr;
  ctx->d_didx_m = ctx->d_rinst_m = nullptr;
  ctx->d_dw_m = nullptr;
  ctx->d_ridx_m = nullptr;
  ctx->msorted = false;
  // buffers allocated on first use must be allocated again after a new layout
  ctx->d_fcompact = nullptr;
  ctx->d_saved = nullptr;
  ctx->saved = wh_ctx::SavedSolve{};  // a stopped solve refers to the old layout
  for (auto &S : ctx->set) S.maps = nullptr;
}

inline int64_t ext_index(const DevGrid &G, int i, int j) {
  return G.base + (int64_t)(j + G.g1) * G.pitch + (i + G.g0);
}

bool is_fp32(const wh_ctx *c) { return c->set[c->active].fp32; }

// Make march set k (0: FP64, 1: FP32) the one the launch code uses.
void use_set(wh_ctx *c, int k) {
  c->active = k;
  const MarchSet &S = c->set[k];
  c->d_Wa = S.Wa;
  c->d_Wb = S.Wb;
  c->d_F = S.F;
  c->d_Wt = S.Wt;
  c->march_blocks = S.march_blocks;
  c->iter_blocks = S.iter_blocks;
}
int default_set(const wh_ctx *c) { return c->opt.precision == WH_FP32 ? 1 : 0; }

// Tensor maps of the TMA-staged march: per fast grid, over its extended arrays (width pitch,
// height n1 + 2 g1, rows pitch elements apart), boxes of kBoxX columns starting at extended
// column i0: W^n with halo (tile rows + 2R) from either state array, W^{n-1} (tile rows)
// from either, F, V (FP64) and the mask (kMaskBoxX bytes).  Out-of-range parts of a box
// are zero-filled.
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

wh_status encode_maps(wh_ctx *ctx, MarchSet &S, int order) {
  static EncodeTiled encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return fail(ctx, WH_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    encode = (EncodeTiled)fn;
  }
  const int R = order / 2, TY = kTileY * kPY;
  const size_t ts = S.fp32 ? 4 : 8;
  const CUtensorMapDataType dt = S.fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                        : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  std::vector<CUtensorMap> maps(ctx->fast_grids.size() * kMapsPerGrid);
  for (size_t k = 0; k < ctx->fast_grids.size(); ++k) {
    const DevGrid &G = ctx->hgrids[ctx->fast_grids[k]];
    const cuuint64_t dims[2] = {(cuuint64_t)G.pitch, (cuuint64_t)(G.n1 + 2 * G.g1)};
    const cuuint32_t estr[2] = {1, 1};
    auto enc = [&](int which, CUtensorMapDataType type, size_t es, void *base, int bx, int by) {
      const cuuint64_t strides[1] = {(cuuint64_t)G.pitch * es};
      const cuuint32_t box[2] = {(cuuint32_t)bx, (cuuint32_t)by};
      void *addr = (char *)base + (size_t)G.base * es;
      return encode(&maps[k * kMapsPerGrid + which], type, 2, addr, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    };
    CUresult r = CUDA_SUCCESS;
    if (!r) r = enc(kMapWaHalo, dt, ts, S.Wa, kBoxX, TY + 2 * R);
    if (!r) r = enc(kMapWbHalo, dt, ts, S.Wb, kBoxX, TY + 2 * R);
    if (!r) r = enc(kMapWaCtr, dt, ts, S.Wa, kBoxX, TY);
    if (!r) r = enc(kMapWbCtr, dt, ts, S.Wb, kBoxX, TY);
    if (!r) r = enc(kMapF, dt, ts, S.F, kBoxX, TY);
    if (!r) r = enc(kMapV, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, ctx->d_V, kBoxX, TY);
    if (!r) r = enc(kMapMask, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, ctx->d_mask, kMaskBoxX, TY);
    if (r) return fail(ctx, WH_ERR_CUDA, "tensor map of grid %d: error %d", ctx->fast_grids[k], (int)r);
  }
  wh_status st;
  if ((st = dalloc(ctx, &S.maps, std::max<size_t>(maps.size(), 1)))) return st;
  CK(cudaMemcpy(S.maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
  return WH_OK;
}

// Build the device layout, upload everything that does not depend on omega.
wh_status build_layout(wh_ctx *ctx) {
  free_device(ctx);
  const int order = ctx->opt.order, R = order / 2;
  int64_t off = 0, coff = 0, k5 = 0, woff = 0, nact = 0;
  ctx->hgrids.clear();
  ctx->htiles.clear();
  for (size_t g = 0; g < ctx->grids.size(); ++g) {
    const HostGrid &H = ctx->grids[g];
    DevGrid G{};
    G.n0 = H.d.n[0];
    G.n1 = H.d.n[1];
    G.g0 = H.g0;
    G.g1 = H.g1;
    G.pitch = (int32_t)(((G.n0 + 2 * G.g0) + 31) / 32 * 32);
    G.per0 = H.d.bc[0] == WH_BC_PERIODIC;
    G.per1 = H.d.bc[2] == WH_BC_PERIODIC;
    G.kind = H.d.kind;
    G.ortho = H.d.orthogonal;
    G.h0 = H.d.h[0];
    G.h1 = H.d.h[1];
    G.ext = (int64_t)G.pitch * (G.n1 + 2 * G.g1);
    G.base = off;
    off += (G.ext + 31) / 32 * 32;
    G.cbase = coff;
    coff += (int64_t)G.n0 * G.n1;
    bool varc = !H.c2.empty();
    if (G.kind == WH_CARTESIAN && !varc) {
      G.stencil = kConstCross;
      G.nw = 0;
    } else if (G.kind == WH_CARTESIAN || G.ortho) {
      G.stencil = kPointCross;
      G.nw = 4 * R + 1;
    } else {
      G.stencil = kPointBox;
      G.nw = (2 * R + 1) * (2 * R + 1);
    }
    G.wbase = woff;
    woff += (int64_t)G.nw * G.ext;
    G.kbase = -1;
    if (G.kind == WH_CURVILINEAR) {
      G.kbase = k5;
      k5 += 5 * G.ext;
    }
    for (size_t q = 0; q < H.mask.size(); ++q) nact += H.mask[q] != WH_UNUSED;
    // march tiles: only those holding a discretization or interpolation point
    const int TY = kTileY * kPY;
    for (int j0 = 0; j0 < G.n1; j0 += TY)
      for (int i0 = 0; i0 < G.n0; i0 += kTileX) {
        bool need = false;
        for (int j = j0; j < std::min(j0 + TY, G.n1) && !need; ++j)
          for (int i = i0; i < std::min(i0 + kTileX, G.n0) && !need; ++i) {
            const int8_t m = H.mask[(size_t)j * G.n0 + i];
            need = m == WH_DISC || m == WH_INTERP;
          }
        if (need) ctx->htiles.push_back(Tile{(int32_t)g, i0, j0, 0});
      }
    ctx->hgrids.push_back(G);
  }
  {
    // interleave the grids' tiles so that blocks taking tiles round-robin get a mix of
    // cheap (constant-weight) and expensive (per-point-weight) tiles
    std::vector<std::vector<Tile>> per(ctx->grids.size());
    for (const Tile &t : ctx->htiles) per[t.grid].push_back(t);
    std::vector<Tile> mixed;
    mixed.reserve(ctx->htiles.size());
    std::vector<double> taken(per.size(), 0.0);
    size_t left = ctx->htiles.size();
    std::vector<size_t> pos(per.size(), 0);
    while (left) {
      // take from the grid with the smallest fraction taken so far
      size_t best = 0;
      double bf = 2.0;
      for (size_t g = 0; g < per.size(); ++g)
        if (pos[g] < per[g].size()) {
          const double f = (double)pos[g] / per[g].size();
          if (f < bf) {
            bf = f;
            best = g;
          }
        }
      mixed.push_back(per[best][pos[best]++]);
      --left;
    }
    ctx->htiles.swap(mixed);
  }
  // the TMA-staged march keeps this interleaved order (grids mixed tile by tile)
  const std::vector<Tile> mixed_tiles = ctx->htiles;
  ctx->total = off;
  ctx->ncompact = coff;
  ctx->nactive = nact;
  // instances: contiguous runs of grids
  ctx->ninst = 0;
  ctx->icstart.clear();
  ctx->icend.clear();
  ctx->inact.clear();
  for (size_t g = 0; g < ctx->grids.size(); ++g) {
    const int k = ctx->grids[g].d.instance;
    if (k == ctx->ninst) {
      ctx->icstart.push_back(ctx->hgrids[g].cbase);
      ctx->icend.push_back(ctx->hgrids[g].cbase);
      ctx->inact.push_back(0);
      ++ctx->ninst;
    }
    ctx->hgrids[g].inst = k;
    ctx->icend[k] = ctx->hgrids[g].cbase + (int64_t)ctx->hgrids[g].n0 * ctx->hgrids[g].n1;
    for (int8_t m : ctx->grids[g].mask) ctx->inact[k] += m != WH_UNUSED;
  }
  ctx->iactive.assign(ctx->ninst, 1);
  ctx->nplanes5 = k5;
  ctx->nweights = woff;

  // host staging of extended arrays
  std::vector<int8_t> mask(off, 0);
  std::vector<double> c2(off, 1.0), f(off, 0.0), rx(std::max<int64_t>(k5, 1), 0.0);
  for (size_t g = 0; g < ctx->grids.size(); ++g) {
    const HostGrid &H = ctx->grids[g];
    const DevGrid &G = ctx->hgrids[g];
    for (int j = 0; j < G.n1; ++j)
      for (int i = 0; i < G.n0; ++i) {
        int64_t p = ext_index(G, i, j), c = (int64_t)j * G.n0 + i;
        mask[p] = H.mask[c];
        if (!H.c2.empty()) c2[p] = H.c2[c];
        if (!H.f.empty()) f[p] = H.f[c];
      }
    if (G.kind == WH_CURVILINEAR) {
      const int e0 = G.n0 + 2 * G.g0, e1 = G.n1 + 2 * G.g1;
      const int64_t E = (int64_t)e0 * e1;
      for (int k = 0; k < 4; ++k)
        for (int j = 0; j < e1; ++j)
          for (int i = 0; i < e0; ++i)
            rx[G.kbase + k * G.ext + (int64_t)j * G.pitch + i] = H.rx[k * E + (int64_t)j * e0 + i];
    }
  }

  // ghost-rule items
  ctx->hbc.clear();
  ctx->hbc_grid.clear();
  ctx->hbc_axis.clear();
  ctx->hbc_hi.clear();
  for (size_t g = 0; g < ctx->grids.size(); ++g) {
    const HostGrid &H = ctx->grids[g];
    const DevGrid &G = ctx->hgrids[g];
    for (int s = 0; s < 4; ++s) {
      const int code = H.d.bc[s];
      if (code != WH_BC_DIRICHLET && code != WH_BC_NEUMANN) continue;
      const int a = s / 2, hi = s % 2, nt = a == 0 ? G.n1 : G.n0, nn = a == 0 ? G.n0 : G.n1;
      for (int t = 0; t < nt; ++t) {
        auto pt = [&](int k) {
          int nrm = hi ? nn - 1 - k : k;
          return a == 0 ? ext_index(G, nrm, t) : ext_index(G, t, nrm);
        };
        const int8_t m = mask[pt(0)];
        BcItem it{};
        if (code == WH_BC_NEUMANN) {
          if (m != WH_DISC) continue;
          it.type = order == 2 ? 0 : 1;
        } else {
          if (m != WH_DIRICHLET || order == 2) continue;
          it.type = 2;
        }
        for (int k = 0; k < 4; ++k) {
          it.u[k] = pt(k);
          if (k > 0 || code == WH_BC_NEUMANN) {
            const int8_t mk = mask[pt(k)];
            if (k <= (order == 2 ? 1 : 3) && mk != WH_DISC && mk != WH_DIRICHLET)
              return fail(ctx, WH_ERR_GRID,
                          "grid %zu side %d: ghost rule at %d reads a non-discretization point",
                          g, s, t);
          }
        }
        it.g[0] = pt(-1);
        it.g[1] = order == 4 ? pt(-2) : pt(-1);
        it.inst = ctx->hgrids[g].inst;
        ctx->hbc.push_back(it);
        ctx->hbc_grid.push_back((int32_t)g);
        ctx->hbc_axis.push_back(a);
        ctx->hbc_hi.push_back(hi);
      }
    }
  }

  // interpolation: absolute donor indices and full tensor weights
  const int w = order + 1, ND = w * w;
  std::vector<int32_t> didx((size_t)std::max<int64_t>(ctx->nrecv, 1) * ND, 0);
  std::vector<double> dw((size_t)std::max<int64_t>(ctx->nrecv, 1) * ND, 0.0);
  std::vector<int64_t> ridx((size_t)std::max<int64_t>(ctx->nrecv, 1), 0);
  std::vector<int> seen(off, 0);
  if (off > INT32_MAX) return fail(ctx, WH_ERR_ARG, "grid too large for 32-bit donor indices");
  for (int64_t r = 0; r < ctx->nrecv; ++r) {
    const int rgr = ctx->rg[r], dgr = ctx->dg[r];
    const DevGrid &RG = ctx->hgrids[rgr], &DG = ctx->hgrids[dgr];
    if (ctx->ri[r] < 0 || ctx->ri[r] >= RG.n0 || ctx->rj[r] < 0 || ctx->rj[r] >= RG.n1)
      return fail(ctx, WH_ERR_GRID, "receiver %lld outside its grid", (long long)r);
    if (RG.inst != DG.inst)
      return fail(ctx, WH_ERR_GRID, "receiver %lld interpolates across instances", (long long)r);
    const int64_t q = ext_index(RG, ctx->ri[r], ctx->rj[r]);
    if (mask[q] != WH_INTERP)
      return fail(ctx, WH_ERR_GRID, "receiver %lld is not an interpolation point", (long long)r);
    if (seen[q]++)
      return fail(ctx, WH_ERR_GRID, "receiver %lld listed twice", (long long)r);
    ridx[r] = q;
    for (int b = 0; b < w; ++b)
      for (int a = 0; a < w; ++a) {
        int ii = ctx->di[r] + a, jj = ctx->dj[r] + b;
        if (DG.per0) ii = ((ii % DG.n0) + DG.n0) % DG.n0;
        if (DG.per1) jj = ((jj % DG.n1) + DG.n1) % DG.n1;
        if (ii < 0 || ii >= DG.n0 || jj < 0 || jj >= DG.n1)
          return fail(ctx, WH_ERR_GRID, "receiver %lld: donor (%d,%d) outside grid %d",
                      (long long)r, ii, jj, dgr);
        const int64_t p = ext_index(DG, ii, jj);
        if (mask[p] != WH_DISC && mask[p] != WH_DIRICHLET)
          return fail(ctx, WH_ERR_GRID,
                      "receiver %lld: donor (%d,%d) of grid %d is not a discretization point",
                      (long long)r, ii, jj, dgr);
        didx[r * ND + b * w + a] = (int32_t)p;
        dw[r * ND + b * w + a] = ctx->wx[r * w + a] * ctx->wy[r * w + b];
      }
  }
  for (size_t g = 0; g < ctx->grids.size(); ++g) {
    const DevGrid &G = ctx->hgrids[g];
    for (int j = 0; j < G.n1; ++j)
      for (int i = 0; i < G.n0; ++i) {
        int64_t p = ext_index(G, i, j);
        if (mask[p] == WH_INTERP && !seen[p])
          return fail(ctx, WH_ERR_GRID, "interpolation point (%d,%d) of grid %zu has no donor",
                      i, j, g);
      }
  }

  // Ghost rules and interpolation folded into the march launch: work units as the blocks of
  // the separate kernel (256 items, or 256 / lanes receivers), and for each unit the tiles
  // holding the values it reads (ghost-rule sources, donors).  Those tiles go first in the
  // march order (they are done early in the launch) and signal when written (pad_ = 1).
  {
    const int ntl = (int)ctx->htiles.size();
    std::vector<int32_t> owner(off, -1);
    for (int t = 0; t < ntl; ++t) {
      const Tile &T = ctx->htiles[t];
      const DevGrid &G = ctx->hgrids[T.grid];
      for (int j = T.j0; j < std::min(T.j0 + kTileY * kPY, G.n1); ++j)
        for (int i = T.i0; i < std::min(T.i0 + kTileX, G.n0); ++i) owner[ext_index(G, i, j)] = t;
    }
    const int lanes = order == 4 ? 8 : 4;
    const int nbc = (int)ctx->hbc.size();
    const int bc_blocks = (nbc + 255) / 256;
    const int g_blocks = (int)((ctx->nrecv * lanes + 255) / 256);
    ctx->nunits = bc_blocks + g_blocks;
    std::vector<std::vector<int32_t>> udep(ctx->nunits);
    std::vector<char> needed(ntl, 0);
    auto add = [&](int u, int64_t p) {
      if (p >= 0 && p < off && owner[p] >= 0) {
        udep[u].push_back(owner[p]);
        needed[owner[p]] = 1;
      }
    };
    for (int k = 0; k < nbc; ++k)
      for (int q = 0; q < 4; ++q) add(k / 256, ctx->hbc[k].u[q]);
    for (int64_t r = 0; r < ctx->nrecv; ++r)
      for (int d = 0; d < ND; ++d) add(bc_blocks + (int)(r * lanes / 256), didx[r * ND + d]);
    // stable partition: signalling tiles first
    std::vector<int32_t> newpos(ntl);
    std::vector<Tile> order_t;
    order_t.reserve(ntl);
    for (int pass = 0; pass < 2; ++pass)
      for (int t = 0; t < ntl; ++t)
        if ((needed[t] != 0) == (pass == 0)) {
          newpos[t] = (int32_t)order_t.size();
          Tile T = ctx->htiles[t];
          T.pad_ = needed[t] ? 1 : 0;
          order_t.push_back(T);
        }
    ctx->htiles.swap(order_t);
    ctx->udep_off.assign(ctx->nunits + 1, 0);
    ctx->udep_tile.clear();
    for (int u = 0; u < ctx->nunits; ++u) {
      std::vector<int32_t> &d = udep[u];
      for (int32_t &x : d) x = newpos[x];
      std::sort(d.begin(), d.end());
      d.erase(std::unique(d.begin(), d.end()), d.end());
      ctx->udep_tile.insert(ctx->udep_tile.end(), d.begin(), d.end());
      ctx->udep_off[u + 1] = (int64_t)ctx->udep_tile.size();
    }
  }
  {
    // TMA-staged march: tiles of non-periodic constant-weight grids whose ghost width is the
    // stencil radius (every TMA box then starts at a 16-byte aligned extended column)
    ctx->hftiles.clear();
    ctx->hgtiles.clear();
    ctx->fast_grids.clear();
    std::vector<int32_t> slot(ctx->hgrids.size(), -1);
    for (size_t g = 0; g < ctx->hgrids.size(); ++g) {
      const DevGrid &G = ctx->hgrids[g];
      if (G.stencil == kConstCross && !G.per0 && !G.per1 && G.g0 == R && G.g1 == R &&
          G.base % 32 == 0 && G.pitch % 32 == 0) {
        slot[g] = (int32_t)ctx->fast_grids.size();
        ctx->fast_grids.push_back((int32_t)g);
      }
    }
    for (const Tile &t : mixed_tiles) {
      if (slot[t.grid] >= 0 && t.i0 % 32 == 0) {
        Tile f = t;
        f.pad_ = slot[t.grid];
        ctx->hftiles.push_back(f);
      } else {
        ctx->hgtiles.push_back(t);
      }
    }
  }
  {
    // the folded gather's dependencies in the TMA march's numbering (fast tiles, then general)
    std::map<std::tuple<int, int, int>, int32_t> tma_index;
    for (size_t k = 0; k < ctx->hftiles.size(); ++k) {
      const Tile &t = ctx->hftiles[k];
      tma_index[std::make_tuple(t.grid, t.i0, t.j0)] = (int32_t)k;
    }
    for (size_t k = 0; k < ctx->hgtiles.size(); ++k) {
      const Tile &t = ctx->hgtiles[k];
      tma_index[std::make_tuple(t.grid, t.i0, t.j0)] = (int32_t)(ctx->hftiles.size() + k);
    }
    ctx->udep_tile_tma.resize(ctx->udep_tile.size());
    for (size_t e = 0; e < ctx->udep_tile.size(); ++e) {
      const Tile &t = ctx->htiles[ctx->udep_tile[e]];
      ctx->udep_tile_tma[e] = tma_index.at(std::make_tuple(t.grid, t.i0, t.j0));
    }
  }

  // persistent-kernel patch lists: ghost and receiver positions inside each tile's staged
  // box (tile + halo of order/2, corner blocks excluded: the cross stencil never reads
  // them; box stencils only occur on grids without ghosts or receivers in the halo corners
  // of ... every patched position is included regardless of stencil)
  std::vector<int32_t> kind_item(off, -1), recv_of(off, -1);
  for (size_t k = 0; k < ctx->hbc.size(); ++k) {
    kind_item[ctx->hbc[k].g[0]] = (0 << 24) | (int32_t)k;
    if (order == 4) kind_item[ctx->hbc[k].g[1]] = (1 << 24) | (int32_t)k;
  }
  for (int64_t r = 0; r < ctx->nrecv; ++r) {
    kind_item[ridx[r]] = (2 << 24) | (int32_t)r;
    recv_of[ridx[r]] = (int32_t)r;
  }
  std::vector<int64_t> patch_off(ctx->htiles.size() + 1, 0);
  std::vector<int32_t> patch_pos, patch_item;
  {
    const int SX = kTileX + 2 * R, SY = kTileY * kPY + 2 * R;
    for (size_t t = 0; t < ctx->htiles.size(); ++t) {
      const Tile &T = ctx->htiles[t];
      const DevGrid &G = ctx->hgrids[T.grid];
      const bool box = G.stencil == kPointBox;
      for (int rr = 0; rr < SY; ++rr)
        for (int cc = 0; cc < SX; ++cc) {
          const bool corner = (rr < R || rr >= SY - R) && (cc < R || cc >= SX - R);
          if (corner && !box) continue;
          int i = T.i0 - R + cc, j = T.j0 - R + rr;
          if (G.per0) i = ((i % G.n0) + G.n0) % G.n0;
          else if (i < -G.g0 || i >= G.n0 + G.g0) continue;
          if (G.per1) j = ((j % G.n1) + G.n1) % G.n1;
          else if (j < -G.g1 || j >= G.n1 + G.g1) continue;
          const int32_t ki = kind_item[ext_index(G, i, j)];
          if (ki < 0) continue;
          patch_pos.push_back(((ki >> 24) << 24) | (rr * SX + cc));
          patch_item.push_back(ki & 0xffffff);
        }
      patch_off[t + 1] = (int64_t)patch_pos.size();
    }
  }
  if (ctx->hbc.size() >= (1u << 24) || ctx->nrecv >= (1 << 24))
    return fail(ctx, WH_ERR_ARG, "too many ghost items or receivers for the patch encoding");

  // persistent-kernel dataflow dependencies: tile t at step n reads level-n values owned by
  // the tiles in deps(t) -- its staged box (halo included), the sources of the ghost rules
  // and the donors of the receivers it patches, and itself (W^{n-1} at its own points).  The
  // lists are closed under reversal: t also waits for every tile that reads t's points, so
  // W^{n+1} never overwrites a W^{n-1} value that a reader still needs.
  std::vector<int64_t> dep_off(ctx->htiles.size() + 1, 0);
  std::vector<int32_t> dep_tile;
  {
    const int ntl = (int)ctx->htiles.size();
    std::vector<int32_t> owner(off, -1);
    for (int t = 0; t < ntl; ++t) {
      const Tile &T = ctx->htiles[t];
      const DevGrid &G = ctx->hgrids[T.grid];
      for (int j = T.j0; j < std::min(T.j0 + kTileY * kPY, G.n1); ++j)
        for (int i = T.i0; i < std::min(T.i0 + kTileX, G.n0); ++i) owner[ext_index(G, i, j)] = t;
    }
    std::vector<std::vector<int32_t>> dep(ntl);
    const int SX = kTileX + 2 * R, SY = kTileY * kPY + 2 * R;
    for (int t = 0; t < ntl; ++t) {
      const Tile &T = ctx->htiles[t];
      const DevGrid &G = ctx->hgrids[T.grid];
      std::vector<int32_t> &d = dep[t];
      auto add = [&](int64_t p) {
        if (p >= 0 && p < off && owner[p] >= 0) d.push_back(owner[p]);
      };
      d.push_back(t);
      for (int rr = 0; rr < SY; ++rr)
        for (int cc = 0; cc < SX; ++cc) {
          int i = T.i0 - R + cc, j = T.j0 - R + rr;
          if (G.per0) i = ((i % G.n0) + G.n0) % G.n0;
          else if (i < -G.g0 || i >= G.n0 + G.g0) continue;
          if (G.per1) j = ((j % G.n1) + G.n1) % G.n1;
          else if (j < -G.g1 || j >= G.n1 + G.g1) continue;
          add(ext_index(G, i, j));
        }
      for (int64_t e = patch_off[t]; e < patch_off[t + 1]; ++e) {
        const int kind = patch_pos[e] >> 24, item = patch_item[e];
        if (kind == 2)
          for (int k = 0; k < ND; ++k) add(didx[(int64_t)item * ND + k]);
        else
          for (int k = 0; k < 4; ++k) add(ctx->hbc[item].u[k]);
      }
    }
    std::vector<std::vector<int32_t>> rev(ntl);
    for (int t = 0; t < ntl; ++t)
      for (int32_t x : dep[t]) rev[x].push_back(t);
    for (int t = 0; t < ntl; ++t) {
      std::vector<int32_t> &d = dep[t];
      d.insert(d.end(), rev[t].begin(), rev[t].end());
      std::sort(d.begin(), d.end());
      d.erase(std::unique(d.begin(), d.end()), d.end());
      dep_tile.insert(dep_tile.end(), d.begin(), d.end());
      dep_off[t + 1] = (int64_t)dep_tile.size();
    }
  }

  // device allocations
  wh_status st;
  for (int k = 0; k < 2; ++k) {
    MarchSet &S = ctx->set[k];
    S.fp32 = k == 1;
    S.present = k == 0 || ctx->opt.precision == WH_FP32;
    if (!S.present) continue;
    const size_t ts = S.fp32 ? sizeof(float) : sizeof(double);
    if ((st = dalloc(ctx, (char **)&S.Wa, off * ts)) ||
        (st = dalloc(ctx, (char **)&S.Wb, off * ts)) ||
        (st = dalloc(ctx, (char **)&S.F, off * ts)) ||
        (st = dalloc(ctx, (char **)&S.Wt, ctx->nweights * ts)))
      return st;
  }
  if ((st = dalloc(ctx, &ctx->d_grids, ctx->hgrids.size())) ||
      (st = dalloc(ctx, &ctx->d_tiles, ctx->htiles.size())) ||
      (st = dalloc(ctx, &ctx->d_ftiles, std::max<size_t>(ctx->hftiles.size(), 1))) ||
      (st = dalloc(ctx, &ctx->d_gtiles, std::max<size_t>(ctx->hgtiles.size(), 1))) ||
      (st = dalloc(ctx, &ctx->d_err, 3)) ||
      (st = dalloc(ctx, &ctx->d_udep_off, ctx->udep_off.size())) ||
      (st = dalloc(ctx, &ctx->d_udep_tile, std::max<size_t>(ctx->udep_tile.size(), 1))) ||
      (st = dalloc(ctx, &ctx->d_udep_tile_tma, std::max<size_t>(ctx->udep_tile.size(), 1))) ||
      (st = dalloc(ctx, &ctx->d_mask, off)) ||
      (st = dalloc(ctx, &ctx->d_V, off)) || (st = dalloc(ctx, &ctx->d_c2, off)) ||
      (st = dalloc(ctx, &ctx->d_rx, std::max<int64_t>(k5, 1))) ||
      (st = dalloc(ctx, &ctx->d_coef, std::max<int64_t>(k5, 1))) ||
      (st = dalloc(ctx, &ctx->d_bc, ctx->hbc.size())) ||
      (st = dalloc(ctx, &ctx->d_bc_grid, ctx->hbc.size())) ||
      (st = dalloc(ctx, &ctx->d_bc_axis, ctx->hbc.size())) ||
      (st = dalloc(ctx, &ctx->d_bc_hi, ctx->hbc.size())) ||
      (st = dalloc(ctx, &ctx->d_didx, didx.size())) || (st = dalloc(ctx, &ctx->d_dw, dw.size())) ||
      (st = dalloc(ctx, &ctx->d_ridx, ridx.size())) ||
      (st = dalloc(ctx, &ctx->d_smax, (size_t)ctx->ninst)) ||
      (st = dalloc(ctx, &ctx->d_inst, (size_t)ctx->ninst)) ||
      (st = dalloc(ctx, &ctx->d_rinst, ridx.size())) ||
      (st = dalloc(ctx, &ctx->d_patch_off, patch_off.size())) ||
      (st = dalloc(ctx, &ctx->d_patch_pos, std::max<size_t>(patch_pos.size(), 1))) ||
      (st = dalloc(ctx, &ctx->d_patch_item, std::max<size_t>(patch_item.size(), 1))) ||
      (st = dalloc(ctx, &ctx->d_recv_of, recv_of.size())) ||
      (st = dalloc(ctx, &ctx->d_dep_off, dep_off.size())) ||
      (st = dalloc(ctx, &ctx->d_dep_tile, std::max<size_t>(dep_tile.size(), 1))) ||
      (st = dalloc(ctx, &ctx->d_tile_done, std::max<size_t>(ctx->htiles.size(), 1))))
    return st;
  CK(cudaMemcpy(ctx->d_patch_off, patch_off.data(), patch_off.size() * 8, cudaMemcpyHostToDevice));
  if (!patch_pos.empty()) {
    CK(cudaMemcpy(ctx->d_patch_pos, patch_pos.data(), patch_pos.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_patch_item, patch_item.data(), patch_item.size() * 4,
                  cudaMemcpyHostToDevice));
  }
  CK(cudaMemcpy(ctx->d_recv_of, recv_of.data(), recv_of.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_dep_off, dep_off.data(), dep_off.size() * 8, cudaMemcpyHostToDevice));
  if (!dep_tile.empty())
    CK(cudaMemcpy(ctx->d_dep_tile, dep_tile.data(), dep_tile.size() * 4, cudaMemcpyHostToDevice));
  {
    std::vector<int32_t> rinst(ridx.size(), 0);
    for (int64_t r = 0; r < ctx->nrecv; ++r) rinst[r] = ctx->hgrids[ctx->rg[r]].inst;
    CK(cudaMemcpy(ctx->d_rinst, rinst.data(), rinst.size() * 4, cudaMemcpyHostToDevice));
    ctx->h_rinst = rinst;
  }
  ctx->h_didx = didx;
  ctx->h_dw = dw;
  ctx->h_ridx = ridx;
  CK(cudaMemcpy(ctx->d_tiles, ctx->htiles.data(), ctx->htiles.size() * sizeof(Tile),
                cudaMemcpyHostToDevice));
  if (!ctx->hftiles.empty())
    CK(cudaMemcpy(ctx->d_ftiles, ctx->hftiles.data(), ctx->hftiles.size() * sizeof(Tile),
                  cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_udep_off, ctx->udep_off.data(), ctx->udep_off.size() * 8,
                cudaMemcpyHostToDevice));
  if (!ctx->udep_tile.empty()) {
    CK(cudaMemcpy(ctx->d_udep_tile, ctx->udep_tile.data(), ctx->udep_tile.size() * 4,
                  cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_udep_tile_tma, ctx->udep_tile_tma.data(),
                  ctx->udep_tile_tma.size() * 4, cudaMemcpyHostToDevice));
  }
  if (!ctx->hgtiles.empty())
    CK(cudaMemcpy(ctx->d_gtiles, ctx->hgtiles.data(), ctx->hgtiles.size() * sizeof(Tile),
                  cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_mask, mask.data(), off, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_c2, c2.data(), off * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->set[0].F, f.data(), off * sizeof(double), cudaMemcpyHostToDevice));
  if (ctx->set[1].present) {
    std::vector<float> ff(f.begin(), f.end());
    CK(cudaMemcpy(ctx->set[1].F, ff.data(), off * sizeof(float), cudaMemcpyHostToDevice));
  }
  if (k5) CK(cudaMemcpy(ctx->d_rx, rx.data(), k5 * sizeof(double), cudaMemcpyHostToDevice));
  if (!ctx->hbc.empty()) {
    CK(cudaMemcpy(ctx->d_bc, ctx->hbc.data(), ctx->hbc.size() * sizeof(BcItem),
                  cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_bc_grid, ctx->hbc_grid.data(), ctx->hbc.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_bc_axis, ctx->hbc_axis.data(), ctx->hbc.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_bc_hi, ctx->hbc_hi.data(), ctx->hbc.size() * 4, cudaMemcpyHostToDevice));
  }
  CK(cudaMemcpy(ctx->d_didx, didx.data(), didx.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_dw, dw.data(), dw.size() * 8, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_ridx, ridx.data(), ridx.size() * 8, cudaMemcpyHostToDevice));
  {
    // Dirichlet boundary data: one FP64 array in the state layout, read at Dirichlet points
    bool any = false;
    for (const auto &H : ctx->grids) any |= !H.gdata.empty();
    if (any) {
      std::vector<double> gb((size_t)off, 0.0);
      for (size_t g = 0; g < ctx->grids.size(); ++g) {
        const HostGrid &H = ctx->grids[g];
        if (H.gdata.empty()) continue;
        const DevGrid &G = ctx->hgrids[g];
        for (int j = 0; j < G.n1; ++j)
          for (int i = 0; i < G.n0; ++i)
            if (H.mask[(size_t)j * G.n0 + i] == WH_DIRICHLET)
              gb[(size_t)ext_index(G, i, j)] = H.gdata[(size_t)j * G.n0 + i];
      }
      wh_status e;
      if ((e = dalloc(ctx, &ctx->d_gb, (size_t)off))) return e;
      CK(cudaMemcpy(ctx->d_gb, gb.data(), gb.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    for (size_t g = 0; g < ctx->grids.size(); ++g)
      ctx->hgrids[g].gb = ctx->grids[g].gdata.empty() ? nullptr : ctx->d_gb;
  }
  CK(cudaMemcpy(ctx->d_grids, ctx->hgrids.data(), ctx->hgrids.size() * sizeof(DevGrid),
                cudaMemcpyHostToDevice));
  {
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    for (auto &S : ctx->set) {
      if (!S.present) continue;
      S.march_blocks = sms * march_blocks_per_sm(S.fp32, order);
      S.iter_blocks = sms * iteration_blocks_per_sm(S.fp32, order);
      if (ctx->opt.resident_blocks > 0)
        S.iter_blocks = std::min(S.iter_blocks, ctx->opt.resident_blocks);
      S.tma = S.fp32 && !ctx->hftiles.empty();
      if (S.tma) {
        S.tma_blocks = sms * march_tma_blocks_per_sm(S.fp32, order);
        if ((st = encode_maps(ctx, S, order))) return st;
      }
    }
    CK(cudaGetLastError());
  }
  use_set(ctx, default_set(ctx));
  if ((st = dalloc(ctx, &ctx->d_bar, 1))) return st;
  ctx->dirty = false;
  return WH_OK;
}

// Ghost rules and interpolation folded into march_kernel's launch (see GatherArgs) when
// their work units are few next to the march blocks: each block then runs at most one unit
// after its tiles (disk workload: 235 units, 608 blocks, +6%).  With many units (a batch
// of instances) the separate, fully parallel kernel is faster (16 instances: folding -12%).
bool uses_tma(const wh_ctx *ctx) { return ctx->set[ctx->active].tma && ctx->tune_tma != 0; }

bool folds_gather(const wh_ctx *ctx) {
  if (ctx->nunits == 0 || ctx->fold_failed) return false;
  // the folded units wait for tiles of other blocks: the whole grid must be resident
  const int cap = ctx->opt.resident_blocks;
  const int grid = uses_tma(ctx) ? ctx->set[ctx->active].tma_blocks
                                 : std::min((int)ctx->htiles.size(), ctx->march_blocks);
  if (cap > 0 && grid > cap) return false;
  if (ctx->tune_fold >= 0) return ctx->tune_fold != 0;
  // the TMA march's units would start after its ticketed general tiles run out (a tail:
  // folding measured -6% on the FP32 disk workload), so it folds only when tuned to
  if (uses_tma(ctx)) return false;
  const int nb = std::min((int)ctx->htiles.size(), ctx->march_blocks);
  return 2 * ctx->nunits <= nb;
}

bool tile_tickets(const wh_ctx *ctx) { return ctx->tune_tickets != 0; }

GatherArgs gather_args(wh_ctx *ctx) {
  GatherArgs ga{};
  const int nbc = (int)ctx->hbc.size();
  ga.bc = ctx->d_bc;
  ga.didx = ctx->d_didx;
  ga.dw = ctx->d_dw;
  ga.ridx = ctx->d_ridx;
  ga.rinst = ctx->d_rinst;
  ga.udep_off = ctx->d_udep_off;
  ga.udep_tile = uses_tma(ctx) ? ctx->d_udep_tile_tma : ctx->d_udep_tile;
  ga.tile_done = ctx->d_tile_done;
  ga.err = ctx->d_err;
  // tiles by fixed stride: blocks with fewer tiles reach their gather unit early (tickets,
  // which keep every block on tiles until none are left, measured -8% here)
  ga.ctl = nullptr;
  ga.spin_limit = ctx->opt_spin_limit;
  ga.nbc = nbc;
  ga.bc_blocks = (nbc + 255) / 256;
  ga.nunits = ctx->nunits;
  ga.nrecv = (int)ctx->nrecv;
  return ga;
}

// One march step of the active set: the TMA-staged kernel when the set has tensor maps,
// else march_kernel (with level n + 1's ghost rules and interpolation folded in when
// `gather` is given).
void march_step(wh_ctx *ctx, int n, void *cur, void *oth, double fs,
                const GatherArgs *gather = nullptr) {
  const MarchSet &S = ctx->set[ctx->active];
  const int order = ctx->opt.order;
  // batches without the folded gather: only the prefix of instances still marching
  const bool pre = ctx->msorted && !(gather && gather->nunits);
  if (uses_tma(ctx)) {
    const int nf = pre ? ctx->mpre_f[n] : (int)ctx->hftiles.size();
    const int ngn = pre ? ctx->mpre_g[n] : (int)ctx->hgtiles.size();
    if (nf + ngn == 0) return;
    launch_march_tma(S.fp32, order, n == 0, std::min(S.tma_blocks, nf + ngn), ctx->stream,
                     ctx->d_grids, pre ? ctx->d_ftiles_m : ctx->d_ftiles, nf, S.maps,
                     pre ? ctx->d_gtiles_m : ctx->d_gtiles, ngn, ctx->d_mask, S.Wa, S.Wb, S.F,
                     S.Wt, ctx->d_V, ctx->d_inst, n, fs, ctx->d_err, ctx->opt_spin_limit,
                     gather && gather->nunits ? gather : nullptr);
    return;
  }
  const int ntiles = pre ? ctx->mpre_t[n] : (int)ctx->htiles.size();
  if (ntiles == 0) return;
  launch_march(S.fp32, order, n == 0, std::min(ntiles, ctx->march_blocks), ntiles, ctx->stream,
               ctx->d_grids, pre ? ctx->d_tiles_m : ctx->d_tiles, ctx->d_mask, cur, oth,
               ctx->d_F, ctx->d_Wt, ctx->d_V, ctx->d_inst, n, fs, nullptr, gather);
}

wh_status launch_steps(wh_ctx *ctx, int forcing) {
  // the body of one iteration after init: level-0 ghost rules + interpolation, then the
  // steps n = 0 .. maxM-1 (each instance stops after its own M steps)
  const int order = ctx->opt.order;
  const bool f32 = is_fp32(ctx);
  cudaStream_t s = ctx->stream;
  const double fs = forcing ? 1.0 : 0.0;
  const int nbc = (int)ctx->hbc.size();
  const int bc_blocks = (nbc + 255) / 256;
  const int lanes = order == 4 ? 8 : 4;
  const int g_blocks = (int)((ctx->nrecv * lanes + 255) / 256);
  const int bg_blocks = bc_blocks + g_blocks;
  void *Wa = ctx->d_Wa, *Wb = ctx->d_Wb;
  auto bcg = [&](void *W, int level) {
    if (bg_blocks == 0) return;
    if (ctx->msorted) {  // batches: the items and receivers of instances still marching
      const int nb_l = ctx->mpre_bc[(size_t)level], nr_l = ctx->mpre_r[(size_t)level];
      const int bcb = (nb_l + 255) / 256, gb = (nr_l * lanes + 255) / 256;
      if (bcb + gb == 0) return;
      launch_bc_gather(f32, order, bcb + gb, s, ctx->d_bc_m, nb_l, bcb, ctx->d_didx_m,
                       ctx->d_dw_m, ctx->d_ridx_m, ctx->d_rinst_m, nr_l, W, ctx->d_F,
                       ctx->d_inst, level, fs);
      return;
    }
    launch_bc_gather(f32, order, bg_blocks, s, ctx->d_bc, nbc, bc_blocks, ctx->d_didx, ctx->d_dw,
                     ctx->d_ridx, ctx->d_rinst, (int)ctx->nrecv, W, ctx->d_F, ctx->d_inst, level,
                     fs);
  };
  bcg(Wa, 0);
  const bool fold = folds_gather(ctx);
  const GatherArgs ga = gather_args(ctx);
  GatherArgs ga_tiles{};  // tiles by ticket, no folded gather (batches: +6% over the stride)
  ga_tiles.ctl = ctx->d_err;
  for (int n = 0; n < ctx->maxM; ++n) {
    void *cur = (n & 1) ? Wb : Wa;
    void *oth = (n & 1) ? Wa : Wb;
    if (fold) {
      march_step(ctx, n, cur, oth, fs, &ga);  // level n + 1's ghosts and receivers included
    } else {
      march_step(ctx, n, cur, oth, fs, tile_tickets(ctx) ? &ga_tiles : nullptr);
      bcg(oth, n + 1);
    }
  }
  return WH_OK;
}

wh_status build_graph(wh_ctx *ctx, int forcing) {
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  set_pdl(ctx->tune_pdl != 0);
  wh_status st = launch_steps(ctx, forcing);
  set_pdl(false);
  cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
  if (st != WH_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(ctx, WH_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&ctx->set[ctx->active].gexec[forcing], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess)
    return fail(ctx, WH_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return WH_OK;
}

// A timed-out grid barrier of an earlier persistent launch is reported by the first
// call that finds its flag copied back.
wh_status check_timeout(wh_ctx *ctx, bool wait) {
  if (!ctx->err_pending) return WH_OK;
  if (wait) {
    CK(cudaEventSynchronize(ctx->err_ev));
  } else if (cudaEventQuery(ctx->err_ev) != cudaSuccess) {
    return WH_OK;
  }
  ctx->err_pending = false;
  if (*ctx->h_err) {
    *ctx->h_err = 0;
    if (!ctx->persistent && folds_gather(ctx)) {
      // a folded gather unit gave up waiting (fewer blocks resident than the grid, e.g. a
      // GPU shared with other work): from now on the ghost rules and interpolation run as
      // their own kernel, which waits on nothing
      ctx->fold_failed = true;
      drop_graphs(ctx);
    }
    // the graph path's flag is sticky on the device: clear it once reported, so that the
    // context stays usable (the persistent path clears its own at every launch)
    if (ctx->d_err) CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    return fail(ctx, WH_ERR_TIMEOUT,
                "a bounded wait timed out (grid barrier, step flag or TMA stage of an "
                "iteration)");
  }
  return WH_OK;
}

wh_status iterate_persistent(wh_ctx *ctx, int forcing, const double *vin, double *vout) {
  wh_status st = check_timeout(ctx, false);
  if (st) return st;
  IterArgs A{};
  A.grids = ctx->d_grids;
  A.ngrids = (int)ctx->hgrids.size();
  A.ntiles = (int)ctx->htiles.size();
  A.tiles = ctx->d_tiles;
  A.mask = ctx->d_mask;
  A.Wa = ctx->d_Wa;
  A.Wb = ctx->d_Wb;
  A.F = ctx->d_F;
  A.Wt = ctx->d_Wt;
  A.V = ctx->d_V;
  A.bc = ctx->d_bc;
  A.nbc = (int64_t)ctx->hbc.size();
  A.didx = ctx->d_didx;
  A.dw = ctx->d_dw;
  A.ridx = ctx->d_ridx;
  A.nrecv = ctx->nrecv;
  A.inst = ctx->d_inst;
  A.rinst = ctx->d_rinst;
  A.fs = forcing ? 1.0 : 0.0;
  A.M = ctx->maxM;
  A.total = ctx->total;
  A.ncompact = ctx->ncompact;
  A.spin_limit = ctx->opt_spin_limit;
  A.patch_off = ctx->d_patch_off;
  A.patch_pos = ctx->d_patch_pos;
  A.patch_item = ctx->d_patch_item;
  A.recv_of = ctx->d_recv_of;
  A.dep_off = ctx->d_dep_off;
  A.dep_tile = ctx->d_dep_tile;
  A.tile_done = ctx->d_tile_done;
  CK(cudaMemsetAsync(ctx->d_bar, 0, sizeof(GridBarrier), ctx->stream));
  CK(launch_iteration(is_fp32(ctx), ctx->opt.order, ctx->iter_blocks, ctx->stream, A, vin, vout,
                      ctx->d_bar));
  CK(cudaMemcpyAsync(ctx->h_err, &ctx->d_bar->err, sizeof(int), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaEventRecord(ctx->err_ev, ctx->stream));
  ctx->err_pending = true;
  ctx->launches += 1;
  return WH_OK;
}

wh_status iterate_device(wh_ctx *ctx, int forcing, const double *vin, double *vout) {
  forcing = forcing ? 1 : 0;
  if (ctx->dim == 3)
    return wh3::iterate(ctx->c3, ctx->active == 1, forcing, vin, vout, ctx->stream,
                        &ctx->launches, ctx->err);
  if (ctx->persistent) return iterate_persistent(ctx, forcing, vin, vout);
  if (wh_status st = check_timeout(ctx, false)) return st;
  if (!ctx->set[ctx->active].gexec[forcing]) {
    wh_status st = build_graph(ctx, forcing);
    if (st) return st;
  }
  const int blk = 256;
  const int64_t nb = (ctx->total + blk - 1) / blk;
  const int ng = (int)ctx->hgrids.size();
  launch_init(is_fp32(ctx), (unsigned)nb, ctx->stream, ctx->d_grids, ng, ctx->d_mask, vin,
              ctx->d_Wa, ctx->d_V, ctx->total, ctx->d_inst, forcing ? 1.0 : 0.0);
  CK(cudaGetLastError());
  // tickets start at zero (the kernels also leave them so)
  CK(cudaMemsetAsync(ctx->d_err + 1, 0, 2 * sizeof(int), ctx->stream));
  if (folds_gather(ctx))  // the tiles' step flags start at zero in every iteration
    CK(cudaMemsetAsync(ctx->d_tile_done, 0, ctx->htiles.size() * sizeof(int32_t), ctx->stream));
  CK(cudaGraphLaunch(ctx->set[ctx->active].gexec[forcing], ctx->stream));
  if (uses_tma(ctx) || folds_gather(ctx)) {
    // bounded waits in the graph's kernels leave a sticky flag; reported by a later call
    CK(cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaEventRecord(ctx->err_ev, ctx->stream));
    ctx->err_pending = true;
  }
  const int64_t nc = (ctx->ncompact + blk - 1) / blk;
  launch_finish(is_fp32(ctx), (unsigned)nc, ctx->stream, ctx->d_grids, ng, ctx->d_mask, ctx->d_V,
                ctx->d_Wa, ctx->d_Wb, ctx->d_inst, vout, ctx->ncompact);
  CK(cudaGetLastError());
  // init, level 0's ghost rules + interpolation, the steps, output
  ctx->launches += 3 + (folds_gather(ctx) ? 1 : 2) * (int64_t)ctx->maxM;
  return WH_OK;
}

// ---- reductions ----
wh_status ensure_red(wh_ctx *ctx, int nv) {
  if (ctx->partial_blocks == 0) {
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ctx->partial_blocks = sms * 4;
  }
  if (nv > ctx->red_cap) {
    wh_status st;
    dfree(ctx, &ctx->d_partial);
    dfree(ctx, &ctx->d_red);
    if ((st = dalloc(ctx, &ctx->d_partial, (size_t)nv * ctx->partial_blocks)) ||
        (st = dalloc(ctx, &ctx->d_red, (size_t)nv)))
      return st;
    ctx->red_cap = nv;
  }
  return WH_OK;
}

// A Krylov basis of at least nv compact vectors in d_q (an old, smaller one is freed).
wh_status ensure_q(wh_ctx *ctx, int nv) {
  const int64_t need = (int64_t)nv * ctx->ncompact;
  if (ctx->q_cap >= need) return WH_OK;
  dfree(ctx, &ctx->d_q);
  ctx->q_cap = 0;
  wh_status st = dalloc(ctx, &ctx->d_q, (size_t)need);
  if (st) return st;
  ctx->q_cap = need;
  return WH_OK;
}

// out[k] = <X_k, y>, k < nv, on the device (d_red) and copied to host `out`.
wh_status multidot(wh_ctx *ctx, const double *X, int64_t ldx, int nv, const double *y, int64_t n,
                   double *out_host) {
  wh_status st = ensure_red(ctx, nv);
  if (st) return st;
  int nb = (int)std::min<int64_t>(ctx->partial_blocks, (n + kRedThreads - 1) / kRedThreads);
  if (nb < 1) nb = 1;
  launch_multidot(nb, ctx->stream, X, ldx, nv, y, n, ctx->d_partial, ctx->d_red);
  CK(cudaGetLastError());
  ctx->launches += 2;
  if (out_host) {
    CK(cudaMemcpyAsync(out_host, ctx->d_red, nv * sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return check_timeout(ctx, true);
  }
  return WH_OK;
}

wh_status ensure_stream(wh_ctx *ctx) {
  if (ctx->stream) return WH_OK;
  if (!ctx->own_stream) CK(cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking));
  ctx->stream = ctx->own_stream;
  return WH_OK;
}

// Mark instances active (1) or skipped (0) for the following iterations.
wh_status set_active(wh_ctx *ctx, const std::vector<int8_t> &act) {
  bool changed = false;
  for (int k = 0; k < ctx->ninst; ++k)
    if ((int)act[k] != ctx->hinst[k].active) {
      ctx->hinst[k].active = act[k];
      changed = true;
    }
  if (changed)
    CK(cudaMemcpyAsync(ctx->d_inst, ctx->hinst.data(), ctx->ninst * sizeof(InstDev),
                       cudaMemcpyHostToDevice, ctx->stream));
  ctx->iactive = act;
  return WH_OK;
}

unsigned grid1d(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (unsigned)std::min<int64_t>(b, 152 * 16);
}

}  // namespace

namespace {

// ---- GMRES (Sec. 4.3): A v = v - W_h(v, 0) with the active march set ----
struct SolveLog {
  double *history = nullptr;
  int cap = 0, n = 0;
  int products[2] = {0, 0};  // FP64 / FP32 march products
  void add(double r) {
    if (history && n < cap) history[n] = r;
    ++n;
  }
};

// y = A x = x - W_h(x, 0) (w0 is scratch)
wh_status apply_adjoint(wh_ctx *ctx, const double *x, double *y);

// w -= sum_m (w, phi_m) phi_m over the deflation set (Algorithm 3's deflation step)
wh_status defl_project(wh_ctx *ctx, double *w) {
  const int64_t n = ctx->ncompact;
  wh_status st = multidot(ctx, ctx->defl_phi, n, ctx->defl_k, w, n, nullptr);
  if (st) return st;
  launch_multi_axpy(grid1d(n), ctx->stream, ctx->defl_phi, n, ctx->defl_k, ctx->d_red, w, n);
  return WH_OK;
}

wh_status apply_A(wh_ctx *ctx, const double *x, double *y, double *w0, SolveLog &L) {
  wh_status st = ctx->adjoint_mode ? apply_adjoint(ctx, x, w0) : iterate_device(ctx, 0, x, w0);
  if (st) return st;
  L.products[ctx->active] += 1;
  // deflated GMRES: A_d x = x - P S x with P = I - Phi Phi^T
  if (ctx->defl_on && (st = defl_project(ctx, w0))) return st;
  launch_sub(grid1d(ctx->ncompact), ctx->stream, x, w0, y, ctx->ncompact);
  return WH_OK;
}

// One restart cycle of GMRES(m) on A x = rhs, starting from x, classical Gram-Schmidt
// applied twice, Givens rotations; stops early when the residual estimate drops to
// tol_abs or the product budget runs out.  scale converts residual norms into the
// relative values written to the log.
// FP32 contexts: relative residual at which a solve switches from FP32 to FP64 wave solves
// (an FP32 product is accurate to a few 1e-5 relative on the tested problems)
constexpr double kFp32Split = 1e-4;
// a deflated eigenvalue this close to omega^2 (relative) is refused: the inflation divides
// by omega^2 - lambda_m^2 and would amplify any error in (f, phi_m)
constexpr double kResonanceRel = 1e-12;
// divergence by growth: an FPI difference ||v_{k+1} - v_k|| above kGrowth x the smallest one
// so far, or a GMRES product ||A q|| (q a unit vector) above kGrowth x kOpBound.  A stable
// march gives |beta| <= 1 on every eigenmode, so ||A q|| = ||q - S q|| stays near 2.
constexpr double kGrowth = 10.0;
constexpr double kOpBound = 2.5;

wh_status gmres_cycle(wh_ctx *ctx, const double *rhs, double *x, bool x_is_zero, int m,
                      double tol_abs, int budget, double scale, SolveLog &L, double *res_out,
                      bool *finite, wh_ctx::SavedSolve *sv = nullptr) {
  const int64_t n = ctx->ncompact;
  cudaStream_t s = ctx->stream;
  double *w0 = ctx->d_work, *r = ctx->d_work + n;
  double *Q = ctx->d_q;
  wh_status st;
  *finite = true;
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0), y(m), h(m + 1);
  int k0 = 0;
  if (sv && sv->cycle) {
    // continue a cycle stopped after kk Arnoldi steps: x holds its starting iterate and
    // Q[0..kk] its basis; the rotations and the residual vector g come from the state
    H = sv->H;
    cs = sv->cs;
    sn = sv->sn;
    g = sv->g;
    k0 = sv->kk;
    *res_out = std::fabs(g[k0]);
    sv->cycle = false;
  } else {
    if (x_is_zero) {
      CK(cudaMemcpyAsync(r, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
      if ((st = apply_A(ctx, x, r, w0, L))) return st;
      launch_axpby(grid1d(n), s, 1.0, rhs, -1.0, r, n);  // r = rhs - A x
      --budget;
    }
    double rr;
    if ((st = multidot(ctx, r, 0, 1, r, n, &rr))) return st;
    const double beta = std::sqrt(rr);
    *res_out = beta;
    L.add(beta * scale);
    if (!std::isfinite(beta)) {
      *finite = false;
      return WH_OK;
    }
    if (beta <= tol_abs || budget <= 0) return WH_OK;
    g[0] = beta;
    launch_axpby(grid1d(n), s, 1.0 / beta, r, 0.0, Q, n);
  }
  int kk = k0;
  bool stopped = false;  // the budget ran out inside the cycle
  for (int k = k0; k < m; ++k) {
    if (budget <= 0) {
      stopped = true;
      break;
    }
    double *qk = Q + (int64_t)k * n, *w = Q + (int64_t)(k + 1) * n;
    if ((st = apply_A(ctx, qk, w, w0, L))) return st;
    --budget;
    for (int pass = 0; pass < 2; ++pass) {
      // h = Q^T w lands in d_red (device) and in h (host)
      if ((st = multidot(ctx, Q, n, k + 1, w, n, h.data()))) return st;
      launch_multi_axpy(grid1d(n), s, Q, n, k + 1, ctx->d_red, w, n);
      for (int i = 0; i <= k; ++i) H[(size_t)i * m + k] += h[i];
    }
    double ww;
    if ((st = multidot(ctx, w, 0, 1, w, n, &ww))) return st;
    const double hk1 = std::sqrt(ww);
    {  // ||A q_k||^2 = sum_i h_ik^2 + hk1^2 (q_k a unit vector)
      double col = ww;
      for (int i = 0; i <= k; ++i) col += H[(size_t)i * m + k] * H[(size_t)i * m + k];
      if (!(std::sqrt(col) <= kGrowth * kOpBound)) {
        *finite = false;
        *res_out = std::sqrt(col);
        return WH_OK;
      }
    }
    if (hk1 > 0) launch_axpby(grid1d(n), s, 0.0, w, 1.0 / hk1, w, n);
    for (int i = 0; i < k; ++i) {
      const double t = cs[i] * H[(size_t)i * m + k] + sn[i] * H[(size_t)(i + 1) * m + k];
      H[(size_t)(i + 1) * m + k] = -sn[i] * H[(size_t)i * m + k] + cs[i] * H[(size_t)(i + 1) * m + k];
      H[(size_t)i * m + k] = t;
    }
    const double hkk = H[(size_t)k * m + k];
    const double den = std::hypot(hkk, hk1);
    cs[k] = hkk / den;
    sn[k] = hk1 / den;
    H[(size_t)k * m + k] = den;
    g[k + 1] = -sn[k] * g[k];
    g[k] = cs[k] * g[k];
    kk = k + 1;
    const double est = std::fabs(g[k + 1]);
    *res_out = est;
    L.add(est * scale);
    if (!std::isfinite(est)) {
      *finite = false;
      return WH_OK;
    }
    if (est <= tol_abs || hk1 == 0) break;
    if (budget <= 0 && kk < m) {
      stopped = true;
      break;
    }
  }
  if (stopped && sv) {
    // keep what continuing this cycle needs: the starting iterate (x, before the update
    // below), the Arnoldi data, and the basis Q[0..kk] (stays in d_q)
    sv->cycle = true;
    sv->kk = kk;
    sv->H = H;
    sv->cs = cs;
    sv->sn = sn;
    sv->g = g;
    CK(cudaMemcpyAsync(ctx->d_saved, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  for (int i = kk - 1; i >= 0; --i) {
    double t = g[i];
    for (int j = i + 1; j < kk; ++j) t -= H[(size_t)i * m + j] * y[j];
    y[i] = t / H[(size_t)i * m + i];
  }
  if (kk) {
    CK(cudaMemcpyAsync(ctx->d_red, y.data(), kk * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_gemv_acc(grid1d(n), s, Q, n, kk, ctx->d_red, x, n);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));  // y is read by the copy above
  return WH_OK;
}

// ---- batched GMRES: one GMRES per instance, all advancing in lockstep around one
// batched wave solve per Arnoldi step (instances that are done are switched off) ----
struct InstGmres {
  int64_t off = 0, len = 0;
  double bnorm = 0.0, tol_abs = 0.0, res = 0.0;
  bool converged = false, in_cycle = false, finite = true;
  int kk = 0, products = 0, products32 = 0;
  std::vector<double> H, cs, sn, g, y;
};

// y = A x on the instances marked in `act` (w0 scratch); products counted per instance
wh_status apply_A_batch(wh_ctx *ctx, const double *x, double *y, double *w0,
                        std::vector<InstGmres> &I, const std::vector<int8_t> &act) {
  wh_status st = set_active(ctx, act);
  if (st) return st;
  if ((st = iterate_device(ctx, 0, x, w0))) return st;
  for (size_t k = 0; k < I.size(); ++k)
    if (act[k]) (ctx->active == 1 ? I[k].products32 : I[k].products) += 1;
  launch_sub(grid1d(ctx->ncompact), ctx->stream, x, w0, y, ctx->ncompact);
  return WH_OK;
}

// One lockstep restart cycle on A x = rhs for the instances with in_cycle set; each keeps
// going until its residual estimate reaches its tol_abs, then leaves the cycle.
wh_status gmres_cycle_batch(wh_ctx *ctx, const double *rhs, double *x, bool x_is_zero, int m,
                            int &budget, std::vector<InstGmres> &I) {
  const int64_t n = ctx->ncompact;
  const int K = (int)I.size();
  cudaStream_t s = ctx->stream;
  double *w0 = ctx->d_work, *r = ctx->d_work + n;
  double *Q = ctx->d_q;
  wh_status st;
  std::vector<int8_t> act(K, 0);
  for (int k = 0; k < K; ++k) act[k] = I[k].in_cycle;
  if (x_is_zero) {
    CK(cudaMemcpyAsync(r, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    if ((st = apply_A_batch(ctx, x, r, w0, I, act))) return st;
    launch_axpby(grid1d(n), s, 1.0, rhs, -1.0, r, n);
    --budget;
  }
  for (int k = 0; k < K; ++k) {
    InstGmres &G = I[k];
    if (!G.in_cycle) continue;
    double rr;
    if ((st = multidot(ctx, r + G.off, 0, 1, r + G.off, G.len, &rr))) return st;
    const double beta = std::sqrt(rr);
    G.res = beta;
    G.kk = 0;
    if (!std::isfinite(beta)) G.finite = false;
    if (!std::isfinite(beta) || beta <= G.tol_abs) {
      G.in_cycle = false;
      continue;
    }
    G.H.assign((size_t)(m + 1) * m, 0.0);
    G.cs.assign(m, 0.0);
    G.sn.assign(m, 0.0);
    G.g.assign(m + 1, 0.0);
    G.y.assign(m, 0.0);
    G.g[0] = beta;
    launch_axpby(grid1d(G.len), s, 1.0 / beta, r + G.off, 0.0, Q + G.off, G.len);
  }
  std::vector<double> h(m + 1);
  std::vector<int8_t> live(K);
  for (int k = 0; k < K; ++k) live[k] = I[k].in_cycle;
  for (int j = 0; j < m && budget > 0; ++j) {
    bool any = false;
    for (int k = 0; k < K; ++k) any |= live[k] != 0;
    if (!any) break;
    if ((st = apply_A_batch(ctx, Q + (int64_t)j * n, Q + (int64_t)(j + 1) * n, w0, I, live)))
      return st;
    --budget;
    for (int k = 0; k < K; ++k) {
      if (!live[k]) continue;
      InstGmres &G = I[k];
      double *Qs = Q + G.off, *w = Q + (int64_t)(j + 1) * n + G.off;
      for (int pass = 0; pass < 2; ++pass) {
        if ((st = multidot(ctx, Qs, n, j + 1, w, G.len, h.data()))) return st;
        launch_multi_axpy(grid1d(G.len), s, Qs, n, j + 1, ctx->d_red, w, G.len);
        for (int i = 0; i <= j; ++i) G.H[(size_t)i * m + j] += h[i];
      }
      double ww;
      if ((st = multidot(ctx, w, 0, 1, w, G.len, &ww))) return st;
      const double hk1 = std::sqrt(ww);
      if (hk1 > 0) launch_axpby(grid1d(G.len), s, 0.0, w, 1.0 / hk1, w, G.len);
      for (int i = 0; i < j; ++i) {
        const double t = G.cs[i] * G.H[(size_t)i * m + j] + G.sn[i] * G.H[(size_t)(i + 1) * m + j];
        G.H[(size_t)(i + 1) * m + j] =
            -G.sn[i] * G.H[(size_t)i * m + j] + G.cs[i] * G.H[(size_t)(i + 1) * m + j];
        G.H[(size_t)i * m + j] = t;
      }
      const double hjj = G.H[(size_t)j * m + j];
      const double den = std::hypot(hjj, hk1);
      G.cs[j] = hjj / den;
      G.sn[j] = hk1 / den;
      G.H[(size_t)j * m + j] = den;
      G.g[j + 1] = -G.sn[j] * G.g[j];
      G.g[j] = G.cs[j] * G.g[j];
      G.kk = j + 1;
      G.res = std::fabs(G.g[j + 1]);
      if (!std::isfinite(G.res)) {
        G.finite = false;
        live[k] = 0;
      } else if (G.res <= G.tol_abs || hk1 == 0) {
        live[k] = 0;
      }
    }
  }
  for (int k = 0; k < K; ++k) {
    InstGmres &G = I[k];
    if (!G.in_cycle || G.kk == 0 || !G.finite) continue;
    for (int i = G.kk - 1; i >= 0; --i) {
      double t = G.g[i];
      for (int jj = i + 1; jj < G.kk; ++jj) t -= G.H[(size_t)i * m + jj] * G.y[jj];
      G.y[i] = t / G.H[(size_t)i * m + i];
    }
    CK(cudaMemcpyAsync(ctx->d_red, G.y.data(), G.kk * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_gemv_acc(grid1d(G.len), s, Q + G.off, n, G.kk, ctx->d_red, x + G.off, G.len);
    CK(cudaStreamSynchronize(s));  // d_red is reused by the next instance
  }
  CK(cudaGetLastError());
  return WH_OK;
}

// ---- differentiation (single-instance contexts, FP64 march) ----
constexpr int kCkptEvery = 16;  // forward states are recomputed from checkpoints this far apart

wh_status adj_setup(wh_ctx *ctx) {
  if (ctx->adj_ready) return WH_OK;
  const int order = ctx->opt.order;
  const int64_t total = ctx->total;
  // the 2x2 solve coefficients of the ghost items live on the device (bc_coef_kernel)
  std::vector<BcItem> bc(ctx->hbc.size());
  if (!bc.empty())
    CK(cudaMemcpy(bc.data(), ctx->d_bc, bc.size() * sizeof(BcItem), cudaMemcpyDeviceToHost));
  // entries (source point, constrained position, coefficient)
  struct Ent {
    int64_t src, pos;
    double c;
  };
  std::vector<Ent> ent;
  const double e5[4] = {-10.0, 10.0, -5.0, 1.0};  // E = sum e5_k U_k, G2 = 5 G1 + E
  for (const BcItem &it : bc) {
    double a[4] = {0, 0, 0, 0};
    if (it.type == 0) {
      a[1] = 1.0;
    } else if (it.type == 1) {
      a[0] = -10.0 / 3; a[1] = 18.0 / 3; a[2] = -6.0 / 3; a[3] = 1.0 / 3;
    } else {
      a[0] = (20 * it.A2 + 10 * it.B1) * it.inv;
      a[1] = (-6 * it.A2 - 18 * it.B1) * it.inv;
      a[2] = (-4 * it.A2 + 6 * it.B1) * it.inv;
      a[3] = (it.A2 - it.B1) * it.inv;
    }
    for (int k = 0; k < 4; ++k) {
      if (a[k] != 0.0) ent.push_back({it.u[k], it.g[0], a[k]});
      if (order == 4 && it.type != 0) {
        const double b = 5.0 * a[k] + e5[k];
        if (b != 0.0) ent.push_back({it.u[k], it.g[1], b});
      }
    }
  }
  const int ND = (order + 1) * (order + 1);
  {
    std::vector<int32_t> didx((size_t)ctx->nrecv * ND);
    std::vector<double> dw((size_t)ctx->nrecv * ND);
    std::vector<int64_t> ridx((size_t)ctx->nrecv);
    if (ctx->nrecv) {
      CK(cudaMemcpy(didx.data(), ctx->d_didx, didx.size() * 4, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(dw.data(), ctx->d_dw, dw.size() * 8, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(ridx.data(), ctx->d_ridx, ridx.size() * 8, cudaMemcpyDeviceToHost));
    }
    for (int64_t r = 0; r < ctx->nrecv; ++r)
      for (int d = 0; d < ND; ++d) ent.push_back({didx[r * ND + d], ridx[r], dw[r * ND + d]});
  }
  // CSR over source points; only discretization sources are kept (D zeroes the rest)
  std::vector<int8_t> mask(total);
  CK(cudaMemcpy(mask.data(), ctx->d_mask, total, cudaMemcpyDeviceToHost));
  std::vector<int64_t> cnt(total, 0);
  for (const Ent &e : ent)
    if (mask[e.src] == WH_DISC) cnt[e.src]++;
  std::vector<int64_t> fq, off(1, 0), first(total, -1);
  for (int64_t q = 0; q < total; ++q)
    if (cnt[q]) {
      first[q] = off.back();
      fq.push_back(q);
      off.push_back(off.back() + cnt[q]);
    }
  std::vector<int64_t> pos(off.back());
  std::vector<double> coef(off.back());
  for (const Ent &e : ent) {
    if (mask[e.src] != WH_DISC) continue;
    const int64_t k = first[e.src]++;
    pos[k] = e.pos;
    coef[k] = e.c;
  }
  ctx->nfix = (int64_t)fq.size();
  wh_status st;
  if ((st = dalloc(ctx, &ctx->d_fq, std::max<size_t>(fq.size(), 1))) ||
      (st = dalloc(ctx, &ctx->d_roff, off.size())) ||
      (st = dalloc(ctx, &ctx->d_rpos, std::max<size_t>(pos.size(), 1))) ||
      (st = dalloc(ctx, &ctx->d_rcoef, std::max<size_t>(coef.size(), 1))) ||
      (!ctx->d_adj && (st = dalloc(ctx, &ctx->d_adj, 7 * (size_t)total))))
    return st;
  CK(cudaMemcpy(ctx->d_roff, off.data(), off.size() * 8, cudaMemcpyHostToDevice));
  if (!fq.empty()) {
    CK(cudaMemcpy(ctx->d_fq, fq.data(), fq.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_rpos, pos.data(), pos.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_rcoef, coef.data(), coef.size() * 8, cudaMemcpyHostToDevice));
  }
  CK(cudaStreamSynchronize(cudaStreamLegacy));  // land before the stream's adjoint launches
  ctx->adj_ready = true;
  return WH_OK;
}

// Host copy of instance 0's time tables.
void host_tables(const wh_ctx *ctx, std::vector<double> &fc, std::vector<double> &cosn,
                 std::vector<double> &wf) {
  const wh_time_info &ti = ctx->iti[0];
  const int M = ti.M;
  fc.resize(M + 1);
  cosn.resize(M + 1);
  wf.resize(M + 1);
  for (int n = 0; n <= M; ++n) {
    const double cn = std::cos(ti.omega_e * n * ti.dt);
    const double sig = (n == 0 || n == M) ? 0.5 : 1.0;
    fc[n] = ti.dt * ti.dt * cn;
    cosn[n] = cn;
    wf[n] = (2.0 / M) * sig * (cn - ti.alpha / 2.0);
  }
}

// One forward time step n on the FP64 set: X^{n+1} into Wout from Wn = X^n and
// Wprev = X^{n-1} (march, then ghost rules and interpolation of level n+1).
void forward_step(wh_ctx *ctx, int n, const double *Wn, const double *Wprev, double *Wout) {
  const int order = ctx->opt.order;
  cudaStream_t s = ctx->stream;
  const int nbc = (int)ctx->hbc.size();
  const int bc_blocks = (nbc + 255) / 256;
  const int bg_blocks = bc_blocks + (int)((ctx->nrecv * (order == 4 ? 8 : 4) + 255) / 256);
  const int ntiles = (int)ctx->htiles.size();
  launch_march(false, order, n == 0, std::min(ntiles, ctx->march_blocks), ntiles, s, ctx->d_grids,
               ctx->d_tiles, ctx->d_mask, Wn, Wout, ctx->d_F, ctx->d_Wt, ctx->d_V, ctx->d_inst,
               n, 1.0, Wprev);
  if (bg_blocks)
    launch_bc_gather(false, order, bg_blocks, s, ctx->d_bc, nbc, bc_blocks, ctx->d_didx, ctx->d_dw,
                     ctx->d_ridx, ctx->d_rinst, (int)ctx->nrecv, Wout, ctx->d_F, ctx->d_inst,
                     n + 1, 1.0);
}

// X^0 = C E u into W (input kernel, then ghost rules and interpolation of level 0).
void forward_start(wh_ctx *ctx, const double *u, double *W) {
  const int order = ctx->opt.order;
  cudaStream_t s = ctx->stream;
  const int ng = (int)ctx->hgrids.size();
  launch_init(false, (unsigned)((ctx->total + 255) / 256), s, ctx->d_grids, ng, ctx->d_mask, u, W,
              ctx->d_V, ctx->total, ctx->d_inst, 1.0);
  const int bc_blocks = ((int)ctx->hbc.size() + 255) / 256;
  const int bg_blocks = bc_blocks + (int)((ctx->nrecv * (order == 4 ? 8 : 4) + 255) / 256);
  if (bg_blocks)
    launch_bc_gather(false, order, bg_blocks, s, ctx->d_bc, (int)ctx->hbc.size(), bc_blocks,
                     ctx->d_didx, ctx->d_dw, ctx->d_ridx, ctx->d_rinst, (int)ctx->nrecv, W,
                     ctx->d_F, ctx->d_inst, 0, 1.0);
}

// The reverse sweep.  lam: extended adjoint source.  Without gradients: Z^0 = S^T lam is
// left in the returned buffer.  With gradients (u != nullptr, compact): the forward states
// X^n of the march from u (forcing on) are kept whole or recomputed from checkpoints, and
// d(lam . W_h)/df and c^2 d(lam . W_h)/dc^2 are accumulated (extended) into gf, gc2.
wh_status adj_sweep(wh_ctx *ctx, const double *lam, double **z0_out, const double *u,
                    double *gc2, double *gf) {
  const int order = ctx->opt.order, M = ctx->iti[0].M;
  const int64_t total = ctx->total;
  cudaStream_t s = ctx->stream;
  const int ng = (int)ctx->hgrids.size();
  std::vector<double> fc, cosn, wf;
  host_tables(ctx, fc, cosn, wf);
  double *Y = ctx->d_adj + total;
  double *Zb[3] = {ctx->d_adj + 2 * total, ctx->d_adj + 3 * total, ctx->d_adj + 4 * total};
  CK(cudaMemsetAsync(Zb[0], 0, total * sizeof(double), s));
  CK(cudaMemsetAsync(Zb[1], 0, total * sizeof(double), s));
  const bool grad = u != nullptr;
  const int nseg = (M + kCkptEvery - 1) / kCkptEvery;
  const double *F = (const double *)ctx->d_F;
  bool whole = false;
  double *ck = nullptr, *seg = nullptr;
  wh_status st;
  if (grad) {
    const int64_t need = (int64_t)(M + 1) * total;
    uint64_t cap = ctx->opt.trajectory_bytes;
    if (!cap) {
      size_t fr = 0, tot = 0;
      CK(cudaMemGetInfo(&fr, &tot));
      cap = (uint64_t)fr / 2 + (uint64_t)ctx->traj_cap * 8;  // a held buffer counts as free
    }
    whole = (uint64_t)need * 8 <= cap;
    if (whole && ctx->traj_cap < need) {
      dfree(ctx, &ctx->d_traj);
      ctx->traj_cap = 0;
      if ((st = dalloc(ctx, &ctx->d_traj, (size_t)need))) return st;
      ctx->traj_cap = need;
    }
  }
  if (grad && whole) {
    // X^n in slot n: the march writes each level into its own slot
    double *X = ctx->d_traj;
    forward_start(ctx, u, X);
    for (int n = 0; n < M; ++n)
      forward_step(ctx, n, X + (int64_t)n * total, X + (int64_t)(n ? n - 1 : 0) * total,
                   X + (int64_t)(n + 1) * total);
    CK(cudaGetLastError());
  } else if (grad) {
    // checkpoints (X^s, X^{s-1}) at s = 0, 16, ...; a segment buffer for X^{s-1} .. X^{s+16}
    const int64_t need = (2 * (int64_t)nseg + kCkptEvery + 2) * total;
    if (ctx->ckpt_cap < need) {
      dfree(ctx, &ctx->d_ckpt);
      ctx->ckpt_cap = 0;
      if ((st = dalloc(ctx, &ctx->d_ckpt, (size_t)need))) return st;
      ctx->ckpt_cap = need;
    }
    ck = ctx->d_ckpt;
    seg = ctx->d_ckpt + 2 * (int64_t)nseg * total;
    double *Wa = (double *)ctx->d_Wa, *Wb = (double *)ctx->d_Wb;
    forward_start(ctx, u, Wa);
    for (int n = 0; n < M; ++n) {
      double *cur = (n & 1) ? Wb : Wa, *oth = (n & 1) ? Wa : Wb;
      if (n % kCkptEvery == 0) {
        const int k = n / kCkptEvery;
        CK(cudaMemcpyAsync(ck + (2 * k) * total, cur, total * 8, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(ck + (2 * k + 1) * total, oth, total * 8, cudaMemcpyDeviceToDevice, s));
      }
      forward_step(ctx, n, cur, oth, oth);
    }
    CK(cudaGetLastError());
  }
  int s0 = 0;  // first level of the current segment (checkpoint mode)
  auto state = [&](int k) -> const double * {
    if (whole) return ctx->d_traj + (int64_t)k * total;
    return seg + (int64_t)(k - s0 + 1) * total;  // X^{s0-1} .. X^{e0+1}
  };
  // level M
  int iz_new = 2, iz1 = 0, iz2 = 1;  // Z^{n+1} in Zb[iz1], Z^{n+2} in Zb[iz2]
  launch_adj_step(order, s, ctx->d_grids, ng, ctx->d_mask, (const double *)ctx->d_Wt, lam, wf[M],
                  1.0, Zb[iz1], Zb[iz2], Y, Zb[iz_new], total, nullptr, nullptr, nullptr, F, 0.0,
                  gc2, gf);
  launch_adj_post(s, ctx->d_fq, ctx->d_roff, ctx->d_rpos, ctx->d_rcoef, Y, Zb[iz_new], ctx->nfix,
                  ctx->d_bc, (int)ctx->hbc.size(), F, cosn[M], grad ? gc2 : nullptr, gf);
  // rotate: Z^{M+2} <- Z^{M+1}, Z^{M+1} <- Z^M
  int t = iz2;
  iz2 = iz1;
  iz1 = iz_new;
  iz_new = t;
  for (int sidx = nseg - 1; sidx >= 0; --sidx) {
    s0 = sidx * kCkptEvery;
    const int e0 = std::min(s0 + kCkptEvery - 1, M - 1);
    if (grad && !whole) {
      // restore X^{s0}, X^{s0-1} and recompute X^{s0+1} .. X^{e0+1} into the segment slots
      CK(cudaMemcpyAsync(seg, ck + (2 * sidx + 1) * total, total * 8, cudaMemcpyDeviceToDevice,
                         s));
      CK(cudaMemcpyAsync(seg + total, ck + (2 * sidx) * total, total * 8,
                         cudaMemcpyDeviceToDevice, s));
      for (int n = s0; n <= e0; ++n)
        forward_step(ctx, n, state(n), state(n - 1), (double *)state(n + 1));
    }
    for (int n = e0; n >= s0; --n) {
      const double sc = n == 0 ? 0.5 : 1.0;
      const double fcn = n == 0 ? 0.5 * ctx->iti[0].dt * ctx->iti[0].dt : fc[n];
      const double *Xp = grad && n > 0 ? state(n - 1) : nullptr;
      const double *Xn = grad ? state(n) : nullptr, *Xx = grad ? state(n + 1) : nullptr;
      launch_adj_step(order, s, ctx->d_grids, ng, ctx->d_mask, (const double *)ctx->d_Wt, lam,
                      wf[n], sc, Zb[iz1], Zb[iz2], Y, Zb[iz_new], total, Xp, Xn, Xx, F, fcn, gc2,
                      gf);
      launch_adj_post(s, ctx->d_fq, ctx->d_roff, ctx->d_rpos, ctx->d_rcoef, Y, Zb[iz_new],
                      ctx->nfix, ctx->d_bc, (int)ctx->hbc.size(), F, cosn[n],
                      grad ? gc2 : nullptr, gf);
      t = iz2;
      iz2 = iz1;
      iz1 = iz_new;
      iz_new = t;
    }
  }
  CK(cudaGetLastError());
  *z0_out = Zb[iz1];
  return WH_OK;
}

// y = S^T x for compact x, y (the zero-forcing map's transpose).  The sweep between the
// fixed buffers lam and Z^0 is captured once per preparation as a CUDA graph (its kernels
// with programmatic dependent launch, as the forward iteration's) and replayed.
wh_status apply_adjoint(wh_ctx *ctx, const double *x, double *y) {
  wh_status st = adj_setup(ctx);
  if (st) return st;
  const int ng = (int)ctx->hgrids.size();
  double *lam = ctx->d_adj;
  if (!ctx->adj_graph) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    set_pdl(ctx->tune_pdl != 0);
    st = adj_sweep(ctx, lam, &ctx->adj_z0, nullptr, nullptr, nullptr);
    set_pdl(false);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (st) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return fail(ctx, WH_ERR_CUDA, "adjoint capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ctx->adj_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
      return fail(ctx, WH_ERR_CUDA, "adjoint graph: %s", cudaGetErrorString(e));
  }
  launch_compact_to_ext(ctx->stream, ctx->d_grids, ng, ctx->d_mask, x, lam, ctx->total);
  CK(cudaGraphLaunch(ctx->adj_graph, ctx->stream));
  launch_ext_to_compact(ctx->stream, ctx->d_grids, ng, ctx->d_mask, ctx->adj_z0, y,
                        ctx->ncompact, 1);
  CK(cudaGetLastError());
  return WH_OK;
}

}  // namespace

// =====================================================================================
// C ABI
// =====================================================================================
namespace {

// ---- eigenpairs of S for deflation (Sec. 4.4, Algorithm 3's deflation set) ----
//
// The paper computes the deflation set with a Krylov-Schur method (SLEPc) on the spatial
// pencil and notes that WaveHoltz itself can yield the eigenpairs.  Here a Krylov-Schur-
// style Arnoldi iteration runs on the zero-forcing map S = W_h(., 0) on the GPU: its
// eigenvectors are those of the constrained spatial operator (S is a polynomial of the
// one-step map) and its largest |beta| are exactly the slowest modes of the fixed-point
// iteration.  Products are library iterations; the basis lives in device memory; only the
// small projected matrices are on the host.

// splitmix64 (Steele, Lea and Flood, 2014): a counter-based generator for the start vectors.
uint64_t splitmix64(uint64_t &x) {
  x += 0x9E3779B97F4A7C15ull;
  uint64_t z = x;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// The real basis of the `want` eigenvalues of largest modulus of the m x m matrix A
// (row-major): their eigenvectors (real parts; a complex conjugate pair contributes its real
// and imaginary parts), in decreasing modulus, as columns of Z (column-major m x p).  order,
// w, Y receive the full eigen-decomposition.  Returns p (want, or want + 1 when the cut
// falls inside a complex pair), or -1 if the QR algorithm failed.
struct SmallEig {
  std::vector<std::complex<double>> w, Y;
  std::vector<int> order;
};
int real_basis(int m, const std::vector<double> &A, int want, SmallEig &E, std::vector<double> &Z,
               bool split_pairs) {
  if (!dense_eig(m, A.data(), E.w, E.Y)) return -1;
  E.order.resize(m);
  for (int i = 0; i < m; ++i) E.order[i] = i;
  std::stable_sort(E.order.begin(), E.order.end(),
                   [&](int a, int b) { return std::abs(E.w[a]) > std::abs(E.w[b]); });
  Z.assign((size_t)m * (want + 1), 0.0);
  int p = 0;
  for (int t = 0; t < m && p < want; ++t) {
    const int i = E.order[t];
    const std::complex<double> th = E.w[i];
    const bool cplx = std::fabs(th.imag()) > 1e-8 * std::abs(th);
    if (cplx && th.imag() < 0) continue;  // the pair is taken at its + member
    // rotate the eigenvector so that its largest entry is real and positive
    int rmax = 0;
    for (int r = 1; r < m; ++r)
      if (std::abs(E.Y[(size_t)r * m + i]) > std::abs(E.Y[(size_t)rmax * m + i])) rmax = r;
    const std::complex<double> ph = std::abs(E.Y[(size_t)rmax * m + i]) > 0
                                        ? std::conj(E.Y[(size_t)rmax * m + i]) /
                                              std::abs(E.Y[(size_t)rmax * m + i])
                                        : 1.0;
    for (int r = 0; r < m; ++r) Z[(size_t)p * m + r] = (E.Y[(size_t)r * m + i] * ph).real();
    ++p;
    if (cplx && (p < want || !split_pairs)) {
      for (int r = 0; r < m; ++r) Z[(size_t)p * m + r] = (E.Y[(size_t)r * m + i] * ph).imag();
      ++p;
    }
  }
  return p;
}

// T = Z^T A Z (A row-major m x m, Z column-major m x p, T row-major p x p).
std::vector<double> project(int m, const std::vector<double> &A, int p, const std::vector<double> &Z) {
  std::vector<double> AZ((size_t)m * p, 0.0), T((size_t)p * p, 0.0);
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < p; ++c) {
      double t = 0.0;
      for (int l = 0; l < m; ++l) t += A[(size_t)r * m + l] * Z[(size_t)c * m + l];
      AZ[(size_t)c * m + r] = t;
    }
  for (int a = 0; a < p; ++a)
    for (int c = 0; c < p; ++c) {
      double t = 0.0;
      for (int r = 0; r < m; ++r) t += Z[(size_t)a * m + r] * AZ[(size_t)c * m + r];
      T[(size_t)a * p + c] = t;
    }
  return T;
}

// y = P x (P = I - L L^T over the nl locked vectors L, orthonormal), in place
wh_status eig_project(wh_ctx *ctx, const double *Lk, int nl, double *x) {
  if (nl == 0) return WH_OK;
  const int64_t n = ctx->ncompact;
  wh_status st = multidot(ctx, Lk, n, nl, x, n, nullptr);
  if (st) return st;
  launch_multi_axpy(grid1d(n), ctx->stream, Lk, n, nl, ctx->d_red, x, n);
  return WH_OK;
}

// The masks and the forcing at discretization points (zero elsewhere) in the compact order,
// for two- and three-dimensional contexts.
void compact_disc(const wh_ctx *ctx, std::vector<int8_t> &m) {
  if (ctx->dim == 3) {
    wh3::compact_mask(ctx->c3, m);
    return;
  }
  m.clear();
  for (const auto &H : ctx->grids) m.insert(m.end(), H.mask.begin(), H.mask.end());
}

void compact_forcing_disc(const wh_ctx *ctx, std::vector<double> &f) {
  std::vector<int8_t> m;
  compact_disc(ctx, m);
  if (ctx->dim == 3) {
    wh3::compact_forcing(ctx->c3, f);
  } else {
    f.clear();
    for (const auto &H : ctx->grids) {
      const int64_t np = (int64_t)H.d.n[0] * H.d.n[1];
      if (H.f.empty())
        f.insert(f.end(), (size_t)np, 0.0);
      else
        f.insert(f.end(), H.f.begin(), H.f.begin() + np);
    }
  }
  for (size_t q = 0; q < f.size(); ++q)
    if (m[q] != WH_DISC) f[q] = 0.0;
}

struct EigPass {
  int k = 0;                // Schur vectors delivered
  std::vector<double> T;    // k x k row-major, T = Q^T S Q
  std::vector<std::complex<double>> theta;  // eigenvalues of T (the Ritz values)
  double maxres = 0.0;      // largest relative residual of the wanted Ritz pairs
  bool converged = false;
};

// One Krylov-Schur run on P S P (P = I - L L^T, or S alone when nl = 0): the orthonormal
// basis Q (k vectors into Qout, stride n) of the invariant subspace of the k eigenvalues of
// largest modulus, and T = Q^T S Q.  V: m + 1 basis vectors; W: m scratch vectors.
wh_status eig_pass(wh_ctx *ctx, int k, int m, double tol, int budget, uint64_t seed,
                   const double *Lk, int nl, double *V, double *W, double *Qout, EigPass &R,
                   int &products) {
  const int64_t n = ctx->ncompact;
  cudaStream_t s = ctx->stream;
  wh_status st;
  if ((st = ensure_red(ctx, std::max(m + 1, nl)))) return st;
  // start: uniform in (-1, 1) at discretization points (S ignores the others' values)
  {
    std::vector<double> v0((size_t)n, 0.0);
    std::vector<int8_t> mk;
    compact_disc(ctx, mk);
    uint64_t x = seed;
    for (int64_t q = 0; q < n; ++q) {
      const double r = (double)(splitmix64(x) >> 11) * (1.0 / 9007199254740992.0);
      if (mk[q] == WH_DISC) v0[q] = 2.0 * r - 1.0;
    }
    if ((st = h2d(ctx, V, v0.data(), n * sizeof(double)))) return st;
  }
  if ((st = eig_project(ctx, Lk, nl, V))) return st;
  double nn;
  if ((st = multidot(ctx, V, 0, 1, V, n, &nn))) return st;
  if (!(nn > 0)) return fail(ctx, WH_ERR_STATE, "wh_eigs: no discretization point to start from");
  launch_axpby(grid1d(n), s, 0.0, V, 1.0 / std::sqrt(nn), V, n);
  // H: (m + 1) x m, row-major with row stride m
  std::vector<double> H((size_t)(m + 1) * m, 0.0), h(m + 1);
  int p = 0;
  SmallEig E;
  std::vector<double> Z, Hm((size_t)m * m), Zd;
  double *dZ = nullptr;
  if ((st = dalloc(ctx, &dZ, (size_t)m * m))) return st;
  struct FreeZ {
    wh_ctx *c;
    double **p;
    ~FreeZ() { dfree(c, p); }
  } free_z{ctx, &dZ};
  int mm = m;  // basis size reached (smaller after an invariant-subspace breakdown)
  while (true) {
    mm = m;
    for (int j = p; j < m; ++j) {
      double *vj = V + (int64_t)j * n, *w = V + (int64_t)(j + 1) * n;
      if (budget - products <= 0) {
        mm = j;
        break;
      }
      if ((st = iterate_device(ctx, 0, vj, w))) return st;
      ++products;
      if ((st = eig_project(ctx, Lk, nl, w))) return st;
      for (int pass = 0; pass < 2; ++pass) {
        if ((st = multidot(ctx, V, n, j + 1, w, n, h.data()))) return st;
        launch_multi_axpy(grid1d(n), s, V, n, j + 1, ctx->d_red, w, n);
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] += h[i];
      }
      double ww;
      if ((st = multidot(ctx, w, 0, 1, w, n, &ww))) return st;
      const double hn = std::sqrt(ww);
      if (!std::isfinite(hn)) return fail(ctx, WH_ERR_DIVERGED, "wh_eigs: product not finite");
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn <= 1e-14) {  // invariant subspace: the basis cannot grow
        mm = j + 1;
        H[(size_t)(j + 1) * m + j] = 0.0;
        break;
      }
      launch_axpby(grid1d(n), s, 0.0, w, 1.0 / hn, w, n);
    }
    if (mm < std::min(k, m)) return fail(ctx, WH_ERR_NOT_CONVERGED, "wh_eigs: product budget too small for the basis");
    // the projected matrix and its eigenvalues
    Hm.assign((size_t)mm * mm, 0.0);
    for (int r = 0; r < mm; ++r)
      for (int c = 0; c < mm; ++c) Hm[(size_t)r * mm + c] = H[(size_t)r * m + c];
    const double hlast = mm < m + 1 && mm > 0 ? H[(size_t)mm * m + (mm - 1)] : 0.0;
    const int keep_final = std::min(k, mm);
    // the wanted eigenvalues' invariant subspace of H (an orthonormal Schur basis Z, stable
    // also for nearly defective pairs); S V Z = V Z T + v_{m+1} (h_{m,m-1} Z[m-1, :]), so its
    // residual ||S Q - Q T|| is |h_{m,m-1}| ||Z[m-1, :]||.  Small residuals of the single
    // Ritz pairs do not bound it when the eigenvectors are nearly parallel (clusters near 1,
    // measured: pairs at 1e-15, subspace at 2e-5), so convergence is judged on the subspace.
    std::vector<std::complex<double>> wsel;
    int pk = invariant_basis(mm, Hm.data(), keep_final, Z, wsel);
    for (int w = keep_final - 1; pk > k && w >= 1; --w) pk = invariant_basis(mm, Hm.data(), w, Z, wsel);
    if (pk < 0) return fail(ctx, WH_ERR_CUDA, "wh_eigs: the small eigenproblem did not converge");
    {
      double row = 0.0, thmax = 0.0;
      for (int c = 0; c < pk; ++c) row += Z[(size_t)c * mm + (mm - 1)] * Z[(size_t)c * mm + (mm - 1)];
      for (const auto &th : wsel) thmax = std::max(thmax, std::abs(th));
      R.maxres = std::fabs(hlast) * std::sqrt(row) / std::max(thmax, 1e-300);
    }
    R.converged = R.maxres <= tol;
    const bool out_of_budget = budget - products <= 0 || mm < m;
    if (R.converged || out_of_budget) {
      // deliver: Q = V Z, T = Z^T H Z
      Zd.assign((size_t)mm * pk, 0.0);
      for (int c = 0; c < pk; ++c)
        for (int r = 0; r < mm; ++r) Zd[(size_t)c * mm + r] = Z[(size_t)c * mm + r];
      CK(cudaMemcpyAsync(dZ, Zd.data(), Zd.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      launch_gemm_tall(s, V, n, mm, dZ, pk, Qout, n, n);
      CK(cudaGetLastError());
      CK(cudaStreamSynchronize(s));
      R.k = pk;
      R.T = project(mm, Hm, pk, Z);
      std::vector<std::complex<double>> tw, tY;
      dense_eig(pk, R.T.data(), tw, tY);
      R.theta = tw;
      return WH_OK;
    }
    // thick restart: keep the Schur basis of the Ritz values of largest modulus (the
    // invariant subspace of the small matrix, so S V Z = V Z T + v_{m+1} b^T holds exactly)
    int want = std::min(mm - 2, k + std::max(1, (m - k) / 2));
    int pnew = invariant_basis(mm, Hm.data(), want, Z, wsel);
    while (pnew > mm - 1 && want > 1) pnew = invariant_basis(mm, Hm.data(), --want, Z, wsel);
    if (pnew < 0) return fail(ctx, WH_ERR_CUDA, "wh_eigs: the small eigenproblem did not converge");
    std::vector<double> T = project(mm, Hm, pnew, Z);
    Zd.assign((size_t)mm * pnew, 0.0);
    for (int c = 0; c < pnew; ++c)
      for (int r = 0; r < mm; ++r) Zd[(size_t)c * mm + r] = Z[(size_t)c * mm + r];
    CK(cudaMemcpyAsync(dZ, Zd.data(), Zd.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_gemm_tall(s, V, n, mm, dZ, pnew, W, n, n);
    CK(cudaMemcpyAsync(V, W, (size_t)pnew * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(V + (int64_t)pnew * n, V + (int64_t)mm * n, n * sizeof(double),
                       cudaMemcpyDeviceToDevice, s));
    CK(cudaGetLastError());
    std::fill(H.begin(), H.end(), 0.0);
    for (int r = 0; r < pnew; ++r)
      for (int c = 0; c < pnew; ++c) H[(size_t)r * m + c] = T[(size_t)r * pnew + c];
    for (int c = 0; c < pnew; ++c) H[(size_t)pnew * m + c] = hlast * Z[(size_t)c * mm + (mm - 1)];
    p = pnew;
    CK(cudaStreamSynchronize(s));  // Zd is reused
  }
}

// lambda^2 of the eigenvector y (compact, device): -(y, c^2 L_h y) / (y, y) over
// discretization points, with the ghost rules applied to y first (no interpolation).
// c^2 L_h y comes from one first step of the FP64 march with zero forcing:
// W^1 = y + dt^2/2 c^2 L_h y at discretization points.  Uses the FP64 set's two state
// levels and the work vectors w0, w1.
wh_status rayleigh_lam2(wh_ctx *ctx, const double *y, double *w0, double *w1, double *lam2) {
  const int64_t n = ctx->ncompact;
  cudaStream_t s = ctx->stream;
  if (ctx->dim == 3) {
    if (wh_status e = wh3::first_step(ctx->c3, y, w0, w1, s, ctx->err)) return e;
    launch_axpby(grid1d(n), s, -1.0, w0, 1.0, w1, n);
    CK(cudaGetLastError());
    double d[2];
    if (wh_status e = multidot(ctx, w0, n, 2, w0, n, d)) return e;
    *lam2 = -(2.0 / (ctx->ti.dt * ctx->ti.dt)) * d[1] / d[0];
    return WH_OK;
  }
  MarchSet &S0 = ctx->set[0];
  const int order = ctx->opt.order;
  const int ng = (int)ctx->hgrids.size();
  const int64_t nb = (ctx->total + 255) / 256;
  launch_init(false, (unsigned)nb, s, ctx->d_grids, ng, ctx->d_mask, y, S0.Wa, ctx->d_V,
              ctx->total, ctx->d_inst, 0.0);
  const int nbc = (int)ctx->hbc.size();
  if (nbc > 0) {
    const int bcb = (nbc + 255) / 256;
    launch_bc_gather(false, order, bcb, s, ctx->d_bc, nbc, bcb, ctx->d_didx, ctx->d_dw,
                     ctx->d_ridx, ctx->d_rinst, 0, S0.Wa, S0.F, ctx->d_inst, 0, 0.0);
  }
  const int ntiles = (int)ctx->htiles.size();
  launch_march(false, order, true, std::min(ntiles, S0.march_blocks), ntiles, s, ctx->d_grids,
               ctx->d_tiles, ctx->d_mask, S0.Wa, S0.Wb, S0.F, S0.Wt, ctx->d_V, ctx->d_inst, 0,
               0.0);
  launch_ext_to_compact(s, ctx->d_grids, ng, ctx->d_mask, (const double *)S0.Wa, w0, n, 1);
  launch_ext_to_compact(s, ctx->d_grids, ng, ctx->d_mask, (const double *)S0.Wb, w1, n, 1);
  launch_axpby(grid1d(n), s, -1.0, w0, 1.0, w1, n);  // w1 = W^1 - y at discretization points
  CK(cudaGetLastError());
  double d[2];
  wh_status st = multidot(ctx, w0, n, 2, w0, n, d);  // (y, y), (W^1 - y, y)
  if (st) return st;
  const double dt = ctx->ti.dt;
  *lam2 = -(2.0 / (dt * dt)) * d[1] / d[0];
  return WH_OK;
}

}  // namespace


extern "C" {

wh_status wh_options_default(wh_options *opt) {
  if (!opt) return WH_ERR_ARG;
  opt->order = 4;
  opt->periods = 1;
  opt->cfl = 0.9;
  opt->alpha_mode = 0;
  opt->precision = WH_FP64;
  opt->launch_mode = WH_LAUNCH_GRAPH;
  opt->barrier_spin_limit = 0;
  opt->trajectory_bytes = 0;
  opt->resident_blocks = 0;
  return WH_OK;
}

wh_status wh_create(const wh_options *opt, wh_ctx **out) {
  if (!out) return WH_ERR_ARG;
  *out = nullptr;
  wh_options o;
  wh_options_default(&o);
  if (opt) o = *opt;
  if ((o.order != 2 && o.order != 4) || o.periods < 1 || !(o.cfl > 0.0 && o.cfl <= 2.0) ||
      o.resident_blocks < 0 ||
      (o.alpha_mode != 0 && o.alpha_mode != 1) ||
      (o.precision != WH_FP64 && o.precision != WH_FP32) ||
      (o.launch_mode != WH_LAUNCH_PERSISTENT && o.launch_mode != WH_LAUNCH_GRAPH))
    return WH_ERR_ARG;
  wh_ctx *ctx = new (std::nothrow) wh_ctx();
  if (!ctx) return WH_ERR_NOMEM;
  ctx->opt = o;
  ctx->persistent = o.launch_mode == WH_LAUNCH_PERSISTENT;
  if (o.barrier_spin_limit) ctx->opt_spin_limit = o.barrier_spin_limit;
  // the context's own stream is created on first device use, so that grid description
  // and validation work without a GPU
  *out = ctx;
  return WH_OK;
}

void wh_destroy(wh_ctx *ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_device(ctx);
  if (ctx->h_err) cudaFreeHost(ctx->h_err);
  if (ctx->err_ev) cudaEventDestroy(ctx->err_ev);
  if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
  wh3::destroy(ctx->c3);
  delete ctx;
}

const char *wh_last_error(const wh_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

wh_status wh_set_stream(wh_ctx *ctx, void *stream) {
  if (!ctx) return WH_ERR_ARG;
  if (!stream && !ctx->own_stream) {
    wh_status st = ensure_stream(ctx);
    if (st) return st;
  }
  cudaStream_t s = stream ? (cudaStream_t)stream : ctx->own_stream;
  if (s != ctx->stream) drop_graphs(ctx);
  ctx->stream = s;
  return WH_OK;
}

wh_status wh_add_grid(wh_ctx *ctx, const wh_grid_desc *gd, int32_t *grid_id) {
  if (!ctx || !gd || !gd->mask) return fail(ctx, WH_ERR_ARG, "null grid description");
  if (ctx->dim == 3) return fail(ctx, WH_ERR_STATE, "the context holds three-dimensional grids");
  const int order = ctx->opt.order;
  const int *bc = gd->bc;
  for (int s = 0; s < 4; ++s)
    if (bc[s] < WH_BC_NONE || bc[s] > WH_BC_PERIODIC)
      return fail(ctx, WH_ERR_ARG, "bad boundary code %d", bc[s]);
  if ((bc[0] == WH_BC_PERIODIC) != (bc[1] == WH_BC_PERIODIC) ||
      (bc[2] == WH_BC_PERIODIC) != (bc[3] == WH_BC_PERIODIC))
    return fail(ctx, WH_ERR_GRID, "periodic sides must come in pairs");
  if (gd->kind != WH_CARTESIAN && gd->kind != WH_CURVILINEAR)
    return fail(ctx, WH_ERR_ARG, "bad grid kind");
  if (gd->kind == WH_CURVILINEAR && !gd->rx)
    return fail(ctx, WH_ERR_ARG, "curvilinear grid without metrics");
  if (!(gd->h[0] > 0) || !(gd->h[1] > 0)) return fail(ctx, WH_ERR_ARG, "non-positive spacing");
  for (int a = 0; a < 2; ++a) {
    const bool per = bc[2 * a] == WH_BC_PERIODIC;
    if (gd->n[a] < (per ? order + 1 : 2 * order + 1))
      return fail(ctx, WH_ERR_ARG, "grid too small along axis %d", a);
  }
  bool phys = false, neu = false;
  for (int s = 0; s < 4; ++s) {
    phys |= bc[s] == WH_BC_DIRICHLET || bc[s] == WH_BC_NEUMANN;
    neu |= bc[s] == WH_BC_NEUMANN;
  }
  if (gd->kind == WH_CURVILINEAR && !gd->orthogonal && phys)
    return fail(ctx, WH_ERR_GRID, "non-orthogonal grid with a Dirichlet or Neumann side");
  if (neu)
    for (int s = 0; s < 4; ++s)
      for (int s2 = 0; s2 < 4; ++s2)
        if (s / 2 != s2 / 2 && bc[s] == WH_BC_NEUMANN &&
            (bc[s2] == WH_BC_DIRICHLET || bc[s2] == WH_BC_NEUMANN))
          return fail(ctx, WH_ERR_GRID, "a Neumann side meets another physical side");
  const int prev = ctx->grids.empty() ? -1 : ctx->grids.back().d.instance;
  if (gd->instance != prev && gd->instance != prev + 1)
    return fail(ctx, WH_ERR_ARG, "instance ids must be contiguous: got %d after %d",
                gd->instance, prev);
  if (ctx->grids.empty() && gd->instance != 0)
    return fail(ctx, WH_ERR_ARG, "the first grid belongs to instance 0");
  HostGrid H;
  H.d = *gd;
  const int64_t n = (int64_t)gd->n[0] * gd->n[1];
  H.mask.assign(gd->mask, gd->mask + n);
  for (int64_t q = 0; q < n; ++q)
    if (H.mask[q] < WH_UNUSED || H.mask[q] > WH_DIRICHLET)
      return fail(ctx, WH_ERR_GRID, "bad mask value %d", (int)H.mask[q]);
  H.g0 = bc[0] == WH_BC_PERIODIC ? 0 : order / 2;
  H.g1 = bc[2] == WH_BC_PERIODIC ? 0 : order / 2;
  if (gd->kind == WH_CURVILINEAR) {
    const int64_t E = (int64_t)(gd->n[0] + 2 * H.g0) * (gd->n[1] + 2 * H.g1);
    H.rx.assign(gd->rx, gd->rx + 4 * E);
    for (double v : H.rx)
      if (!std::isfinite(v)) return fail(ctx, WH_ERR_GRID, "non-finite metric");
  }
  if (gd->c2) {
    H.c2.assign(gd->c2, gd->c2 + n);
    for (double v : H.c2)
      if (!(v > 0) || !std::isfinite(v)) return fail(ctx, WH_ERR_ARG, "c^2 must be positive");
  }
  ctx->grids.push_back(std::move(H));
  ctx->dim = 2;
  ctx->dirty = true;
  ctx->prepared = false;
  if (grid_id) *grid_id = (int32_t)ctx->grids.size() - 1;
  return WH_OK;
}

wh_status wh_add_grid3(wh_ctx *ctx, const wh_grid3_desc *gd, int32_t *grid_id) {
  if (!ctx) return WH_ERR_ARG;
  if (ctx->dim == 2) return fail(ctx, WH_ERR_STATE, "the context holds two-dimensional grids");
  if (!ctx->c3 && !(ctx->c3 = wh3::create())) return fail(ctx, WH_ERR_NOMEM, "out of memory");
  wh_status st = wh3::add_grid(ctx->c3, gd, ctx->opt.order, grid_id, ctx->err);
  if (st) return st;
  ctx->dim = 3;
  ctx->prepared = false;
  return WH_OK;
}

wh_status wh_set_interp3(wh_ctx *ctx, const wh_interp3_desc *it) {
  if (!ctx) return WH_ERR_ARG;
  if (ctx->dim != 3 || !ctx->c3)
    return fail(ctx, WH_ERR_STATE, "add three-dimensional grids first");
  wh_status st = wh3::set_interp(ctx->c3, it, ctx->err);
  if (st) return st;
  ctx->prepared = false;
  return WH_OK;
}

wh_status wh_set_interp(wh_ctx *ctx, const wh_interp_desc *it) {
  if (!ctx || !it || it->n < 0) return fail(ctx, WH_ERR_ARG, "null interpolation data");
  if (ctx->dim == 3) return fail(ctx, WH_ERR_STATE, "use wh_set_interp3 on a 3D context");
  const int w = ctx->opt.order + 1;
  const int64_t n = it->n;
  if (n > 0 && (!it->recv_grid || !it->recv_i || !it->recv_j || !it->donor_grid ||
                !it->donor_i0 || !it->donor_j0 || !it->wx || !it->wy))
    return fail(ctx, WH_ERR_ARG, "null interpolation array");
  for (int64_t r = 0; r < n; ++r) {
    if (it->recv_grid[r] < 0 || it->recv_grid[r] >= (int)ctx->grids.size() ||
        it->donor_grid[r] < 0 || it->donor_grid[r] >= (int)ctx->grids.size())
      return fail(ctx, WH_ERR_GRID, "receiver %lld: bad grid index", (long long)r);
    if (it->recv_grid[r] == it->donor_grid[r])
      return fail(ctx, WH_ERR_GRID, "receiver %lld interpolates from its own grid", (long long)r);
    for (int a = 0; a < w; ++a)
      if (!std::isfinite(it->wx[r * w + a]) || !std::isfinite(it->wy[r * w + a]))
        return fail(ctx, WH_ERR_GRID, "receiver %lld: non-finite weight", (long long)r);
  }
  ctx->nrecv = n;
  ctx->rg.assign(it->recv_grid, it->recv_grid + n);
  ctx->ri.assign(it->recv_i, it->recv_i + n);
  ctx->rj.assign(it->recv_j, it->recv_j + n);
  ctx->dg.assign(it->donor_grid, it->donor_grid + n);
  ctx->di.assign(it->donor_i0, it->donor_i0 + n);
  ctx->dj.assign(it->donor_j0, it->donor_j0 + n);
  ctx->wx.assign(it->wx, it->wx + n * w);
  ctx->wy.assign(it->wy, it->wy + n * w);
  ctx->dirty = true;
  ctx->prepared = false;
  return WH_OK;
}

wh_status wh_set_forcing(wh_ctx *ctx, int32_t gid, const double *f) {
  if (ctx && ctx->dim == 3) {
    if (!f) return fail(ctx, WH_ERR_ARG, "null forcing");
    const wh_status st = wh3::set_forcing(ctx->c3, gid, f, ctx->err);
    if (st == WH_OK) ctx->prepared = false;
    return st;
  }
  if (!ctx || !f || gid < 0 || gid >= (int)ctx->grids.size())
    return fail(ctx, WH_ERR_ARG, "bad forcing arguments");
  HostGrid &H = ctx->grids[gid];
  const int64_t n = (int64_t)H.d.n[0] * H.d.n[1];
  // validate before storing: a rejected call leaves the context's forcing unchanged
  for (int64_t q = 0; q < n; ++q)
    if (!std::isfinite(f[q])) return fail(ctx, WH_ERR_ARG, "non-finite forcing");
  H.f.assign(f, f + n);
  ctx->dirty = true;
  ctx->prepared = false;
  return WH_OK;
}

wh_status wh_set_boundary_data(wh_ctx *ctx, int32_t gid, const double *g) {
  if (!ctx) return WH_ERR_ARG;
  if (ctx->dim == 3) {
    const wh_status st = wh3::set_boundary_data(ctx->c3, gid, g, ctx->err);
    if (st == WH_OK) ctx->prepared = false;
    return st;
  }
  if (gid < 0 || gid >= (int)ctx->grids.size())
    return fail(ctx, WH_ERR_ARG, "bad boundary data arguments");
  HostGrid &H = ctx->grids[gid];
  const int64_t n = (int64_t)H.d.n[0] * H.d.n[1];
  if (g)
    for (int64_t q = 0; q < n; ++q)
      if (!std::isfinite(g[q])) return fail(ctx, WH_ERR_ARG, "non-finite boundary data");
  if (g && ctx->opt.order == 4 && H.d.kind != WH_CARTESIAN)
    for (int sd = 0; sd < 4; ++sd)
      if (H.d.bc[sd] == WH_BC_DIRICHLET)
        return fail(ctx, WH_ERR_GRID,
                    "boundary data on a curvilinear Dirichlet side at order 4 are not supported");
  if (g && ctx->opt.order == 4)
    for (int sd = 0; sd < 4; ++sd)
      if (H.d.bc[sd] == WH_BC_DIRICHLET && H.d.n[1 - sd / 2] < 6)
        return fail(ctx, WH_ERR_GRID, "a side with boundary data needs 6 points at order 4");
  if (g)
    H.gdata.assign(g, g + n);
  else
    H.gdata.clear();
  ctx->dirty = true;
  ctx->prepared = false;
  return WH_OK;
}

// Prepare one frequency per instance: (a2) the operator coefficients and the per-instance
// frozen-coefficient stability bounds on the device, (a1) the time setup of each instance
// (Recipe OmegaTildeExplicit, alpha_d), the device step tables and the stencil weights.
static wh_status prepare_instances(wh_ctx *ctx, const double *omegas) {
  if (ctx->grids.empty()) return fail(ctx, WH_ERR_STATE, "no grids");
  for (size_t g = 0; g < ctx->grids.size(); ++g)
    for (size_t q = 0; q < ctx->grids[g].mask.size(); ++q)
      if (ctx->grids[g].mask[q] == WH_INTERP && ctx->nrecv == 0)
        return fail(ctx, WH_ERR_GRID, "interpolation points but no interpolation data");
  wh_status st;
  if ((st = ensure_stream(ctx))) return st;
  if (ctx->dirty && (st = build_layout(ctx))) return st;
  drop_graphs(ctx);
  const int order = ctx->opt.order, K = ctx->ninst;
  for (int k = 0; k < K; ++k)
    if (!(omegas[k] > 0) || !std::isfinite(omegas[k]))
      return fail(ctx, WH_ERR_ARG, "omega of instance %d must be > 0", k);
  cudaStream_t s = ctx->stream;
  CK(cudaMemsetAsync(ctx->d_smax, 0, K * sizeof(unsigned long long), s));
  for (size_t g = 0; g < ctx->hgrids.size(); ++g) {
    const DevGrid &G = ctx->hgrids[g];
    dim3 tb(32, 8), gb((G.n0 + 31) / 32, (G.n1 + 7) / 8);
    launch_coef(order, gb, tb, s, ctx->d_grids, (int)g, ctx->d_mask, ctx->d_rx, ctx->d_c2,
                ctx->d_coef, ctx->d_smax);
  }
  CK(cudaGetLastError());
  std::vector<unsigned long long> bits(K, 0);
  CK(cudaMemcpyAsync(bits.data(), ctx->d_smax, K * sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double Cp = order == 2 ? 1.0 : std::sqrt(3.0) / 2.0;
  ctx->iti.assign(K, wh_time_info{});
  ctx->maxM = 0;
  int64_t tab_len = 0;
  for (int k = 0; k < K; ++k) {
    double smax;
    std::memcpy(&smax, &bits[k], sizeof smax);
    if (!(smax > 0) || !std::isfinite(smax))
      return fail(ctx, WH_ERR_GRID, "instance %d has no discretization point", k);
    const double omega = omegas[k];
    const double dtmax = ctx->opt.cfl * Cp / std::sqrt(smax);
    int Nt = (int)std::ceil(2.0 * M_PI / (omega * dtmax));
    if (Nt < 2) Nt = 2;
    double dt = 2.0 / omega * std::sin(M_PI / Nt);
    while (dt > dtmax) {
      ++Nt;
      dt = 2.0 / omega * std::sin(M_PI / Nt);
    }
    wh_time_info &ti = ctx->iti[k];
    ti.omega = omega;
    ti.dt = dt;
    ti.Nt = Nt;
    ti.M = ctx->opt.periods * Nt;
    ti.omega_e = 2.0 * M_PI / (Nt * dt);
    ti.alpha = ctx->opt.alpha_mode ? 0.5
                                   : std::tan(ti.omega_e * dt / 2) / std::tan(ti.omega_e * dt);
    ti.dt_max = dtmax;
    ti.Tbar = ti.M * dt;
    ti.n_active = ctx->inact[k];
    ti.n_total = ctx->icend[k] - ctx->icstart[k];
    ctx->maxM = std::max(ctx->maxM, ti.M);
    tab_len += 3 * (int64_t)(ti.M + 1);
  }
  ctx->ti = ctx->iti[0];
  // device tables: per instance fc[0..M], cos[0..M], wf[0..M]
  if (ctx->tabs_cap < tab_len) {
    if ((st = dalloc(ctx, &ctx->d_tabs, (size_t)tab_len))) return st;
    if ((st = dalloc(ctx, &ctx->d_ftabs, (size_t)tab_len / 3))) return st;
    ctx->tabs_cap = tab_len;
  }
  std::vector<double> tab((size_t)tab_len);
  std::vector<float> ftab((size_t)tab_len / 3);  // fc rounded to FP32, per instance
  int64_t fo = 0;
  ctx->hinst.assign(K, InstDev{});
  int64_t o = 0;
  for (int k = 0; k < K; ++k) {
    const wh_time_info &ti = ctx->iti[k];
    const int M = ti.M;
    for (int n = 0; n <= M; ++n) {
      const double cn = std::cos(ti.omega_e * n * ti.dt);
      const double sig = (n == 0 || n == M) ? 0.5 : 1.0;
      tab[o + n] = ti.dt * ti.dt * cn;                                  // forcing factor
      tab[o + (M + 1) + n] = cn;                                        // cos(omega_e t^n)
      tab[o + 2 * (M + 1) + n] = (2.0 / M) * sig * (cn - ti.alpha / 2.0);  // filter weight
    }
    InstDev &I = ctx->hinst[k];
    I.fc = ctx->d_tabs + o;
    I.cosn = ctx->d_tabs + o + (M + 1);
    I.wf = ctx->d_tabs + o + 2 * (M + 1);
    I.dt2 = ti.dt * ti.dt;
    for (int n = 0; n <= M; ++n) ftab[fo + n] = (float)tab[o + n];
    I.fcf = ctx->d_ftabs + fo;
    I.dt2hf = (float)(0.5 * I.dt2);
    fo += M + 1;
    I.M = M;
    I.active = 1;
    o += 3 * (int64_t)(M + 1);
  }
  ctx->iactive.assign(K, 1);
  CK(cudaMemcpy(ctx->d_tabs, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_ftabs, ftab.data(), ftab.size() * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_inst, ctx->hinst.data(), K * sizeof(InstDev), cudaMemcpyHostToDevice));
  // batches: tile lists by descending M of their instance and the per-step prefix lengths
  ctx->msorted = false;
  if (K > 1) {
    auto m_of = [&](const Tile &t) { return ctx->hinst[ctx->hgrids[t.grid].inst].M; };
    auto order_by_m = [&](const std::vector<Tile> &src, Tile **dst,
                          std::vector<int32_t> &pre) -> wh_status {
      std::vector<Tile> v(src);
      std::stable_sort(v.begin(), v.end(),
                       [&](const Tile &a, const Tile &b) { return m_of(a) > m_of(b); });
      std::vector<int64_t> hist((size_t)ctx->maxM + 1, 0);
      for (const Tile &t : v) hist[(size_t)std::min(m_of(t), ctx->maxM)]++;
      pre.assign((size_t)ctx->maxM, 0);
      int64_t acc = 0;  // pre[n] = tiles whose instance has M > n
      for (int n = ctx->maxM - 1; n >= 0; --n) {
        acc += hist[(size_t)n + 1];
        pre[(size_t)n] = (int32_t)acc;
      }
      if (v.empty()) return WH_OK;
      wh_status e;
      if (!*dst && (e = dalloc(ctx, dst, v.size()))) return e;
      CK(cudaMemcpy(*dst, v.data(), v.size() * sizeof(Tile), cudaMemcpyHostToDevice));
      return WH_OK;
    };
    if ((st = order_by_m(ctx->htiles, &ctx->d_tiles_m, ctx->mpre_t)) ||
        (st = order_by_m(ctx->hftiles, &ctx->d_ftiles_m, ctx->mpre_f)) ||
        (st = order_by_m(ctx->hgtiles, &ctx->d_gtiles_m, ctx->mpre_g)))
      return st;
    // ghost-rule items and receivers by descending M; pre[L] = entries with M >= L
    auto prefix = [&](const std::vector<int> &ms, std::vector<int32_t> &pre) {
      std::vector<int64_t> hist((size_t)ctx->maxM + 2, 0);
      for (int m : ms) hist[(size_t)std::min(m, ctx->maxM)]++;
      pre.assign((size_t)ctx->maxM + 1, 0);
      int64_t acc = 0;
      for (int L = ctx->maxM; L >= 0; --L) {
        acc += hist[(size_t)L];
        pre[(size_t)L] = (int32_t)acc;
      }
    };
    {
      const int64_t nr = ctx->nrecv;
      const int ND = (order + 1) * (order + 1);
      std::vector<int64_t> perm((size_t)nr);
      for (int64_t r = 0; r < nr; ++r) perm[(size_t)r] = r;
      auto mr = [&](int64_t r) { return ctx->hinst[ctx->h_rinst[(size_t)r]].M; };
      std::stable_sort(perm.begin(), perm.end(),
                       [&](int64_t a, int64_t b) { return mr(a) > mr(b); });
      std::vector<int32_t> di((size_t)std::max<int64_t>(nr, 1) * ND, 0), ri((size_t)std::max<int64_t>(nr, 1), 0);
      std::vector<double> dwv((size_t)std::max<int64_t>(nr, 1) * ND, 0.0);
      std::vector<int64_t> rx((size_t)std::max<int64_t>(nr, 1), 0);
      std::vector<int> ms((size_t)nr);
      for (int64_t k = 0; k < nr; ++k) {
        const int64_t r = perm[(size_t)k];
        for (int d = 0; d < ND; ++d) {
          di[(size_t)(k * ND + d)] = ctx->h_didx[(size_t)(r * ND + d)];
          dwv[(size_t)(k * ND + d)] = ctx->h_dw[(size_t)(r * ND + d)];
        }
        rx[(size_t)k] = ctx->h_ridx[(size_t)r];
        ri[(size_t)k] = ctx->h_rinst[(size_t)r];
        ms[(size_t)k] = mr(r);
      }
      prefix(ms, ctx->mpre_r);
      if (nr) {
        if ((!ctx->d_didx_m && (st = dalloc(ctx, &ctx->d_didx_m, di.size()))) ||
            (!ctx->d_dw_m && (st = dalloc(ctx, &ctx->d_dw_m, dwv.size()))) ||
            (!ctx->d_ridx_m && (st = dalloc(ctx, &ctx->d_ridx_m, rx.size()))) ||
            (!ctx->d_rinst_m && (st = dalloc(ctx, &ctx->d_rinst_m, ri.size()))))
          return st;
        CK(cudaMemcpy(ctx->d_didx_m, di.data(), di.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_dw_m, dwv.data(), dwv.size() * 8, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_ridx_m, rx.data(), rx.size() * 8, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_rinst_m, ri.data(), ri.size() * 4, cudaMemcpyHostToDevice));
      }
    }
    ctx->msorted = true;
  }
  // the plain copies above and those of the layout may still be in flight; the launches
  // below run on the context's non-blocking stream, which does not wait for them
  CK(cudaStreamSynchronize(cudaStreamLegacy));
  if (!ctx->h_err) {
    CK(cudaMallocHost(&ctx->h_err, sizeof(int)));
    *ctx->h_err = 0;
  }
  if (!ctx->err_ev) CK(cudaEventCreateWithFlags(&ctx->err_ev, cudaEventDisableTiming));
  ctx->err_pending = false;
  if (ctx->persistent && ctx->iter_blocks < 1)
    return fail(ctx, WH_ERR_CUDA, "the persistent kernel cannot be resident on this device");
  // stencil weights, each grid with its instance's dt
  for (size_t g = 0; g < ctx->hgrids.size(); ++g) {
    DevGrid &G = ctx->hgrids[g];
    if (G.stencil != kConstCross) continue;
    const double dt2 = ctx->hinst[G.inst].dt2;
    const double x = dt2 / (G.h0 * G.h0), y = dt2 / (G.h1 * G.h1);
    if (order == 2) {
      G.cw[0] = 2.0 - 2.0 * x - 2.0 * y;
      G.cw[1] = x;
      G.cw[2] = 0.0;
      G.cw[3] = y;
      G.cw[4] = 0.0;
    } else {
      G.cw[0] = 2.0 - 2.5 * x - 2.5 * y;
      G.cw[1] = 16.0 / 12.0 * x;
      G.cw[2] = -1.0 / 12.0 * x;
      G.cw[3] = 16.0 / 12.0 * y;
      G.cw[4] = -1.0 / 12.0 * y;
    }
    for (int k = 0; k < 5; ++k) G.cwf[k] = (float)G.cw[k];
  }
  CK(cudaMemcpyAsync(ctx->d_grids, ctx->hgrids.data(), ctx->hgrids.size() * sizeof(DevGrid),
                     cudaMemcpyHostToDevice, s));
  for (size_t g = 0; g < ctx->hgrids.size(); ++g) {
    const DevGrid &G = ctx->hgrids[g];
    if (G.stencil == kConstCross) continue;
    dim3 tb(32, 8), gb((G.n0 + 31) / 32, (G.n1 + 7) / 8);
    for (const auto &S : ctx->set)
      if (S.present)
        launch_weight(S.fp32, order, gb, tb, s, ctx->d_grids, (int)g, ctx->d_mask, ctx->d_coef,
                      ctx->d_c2, S.Wt, ctx->hinst[G.inst].dt2);
  }
  const int nbc = (int)ctx->hbc.size();
  if (nbc && ctx->d_gb) {
    // Dirichlet data on order-4 sides: the compatibility condition's extra right side
    // -omega^2 g_b - c^2 (D_tt g)_b, D_tt the fourth-order second difference along the side
    // (centred; wrapped on a periodic side; six-point one-sided at the two ends)
    for (int k = 0; k < nbc; ++k) {
      BcItem &it = ctx->hbc[(size_t)k];
      it.fg = 0.0;
      const HostGrid &H = ctx->grids[(size_t)ctx->hbc_grid[(size_t)k]];
      if (it.type != 2 || H.gdata.empty()) continue;
      const DevGrid &G = ctx->hgrids[(size_t)ctx->hbc_grid[(size_t)k]];
      const int a = ctx->hbc_axis[(size_t)k], ta = 1 - a;
      const int64_t o = it.u[0] - G.base;
      const int j = (int)(o / G.pitch) - G.g1, i = (int)(o % G.pitch) - G.g0;
      const int nt = ta == 0 ? G.n0 : G.n1, t = ta == 0 ? i : j;
      const bool per = ta == 0 ? G.per0 : G.per1;
      auto gline = [&](int q) {
        q = per ? ((q % nt) + nt) % nt : q;
        const int ii = ta == 0 ? q : i, jj = ta == 0 ? j : q;
        return H.gdata[(size_t)jj * G.n0 + ii];
      };
      double d2 = 0.0;
      if (per || (t >= 2 && t <= nt - 3)) {
        d2 = -gline(t - 2) + 16.0 * gline(t - 1) - 30.0 * gline(t) + 16.0 * gline(t + 1) -
             gline(t + 2);
      } else {
        static const double e0[6] = {45.0, -154.0, 214.0, -156.0, 61.0, -10.0};
        static const double e1[6] = {10.0, -15.0, -4.0, 14.0, -6.0, 1.0};
        const bool lo = t < 2;
        const double *c = (lo ? t : nt - 1 - t) == 0 ? e0 : e1;
        for (int q = 0; q < 6; ++q) d2 += c[q] * gline(lo ? q : nt - 1 - q);
      }
      const double ht = ta == 0 ? G.h0 : G.h1;
      const double c2b = H.c2.empty() ? 1.0 : H.c2[(size_t)j * G.n0 + i];
      const double om = omegas[G.inst];
      it.fg = -om * om * H.gdata[(size_t)j * G.n0 + i] - c2b * d2 / (12.0 * ht * ht);
    }
    CK(cudaMemcpyAsync(ctx->d_bc, ctx->hbc.data(), (size_t)nbc * sizeof(BcItem),
                       cudaMemcpyHostToDevice, s));
  }
  if (nbc)
    launch_bc_coef(nbc, s, ctx->d_bc, ctx->d_bc_grid, ctx->d_bc_axis, ctx->d_bc_hi, ctx->d_grids,
                   ctx->d_coef, ctx->d_c2);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  if (ctx->msorted && !ctx->hbc.empty()) {
    // the ghost-rule items by descending M, taken from the device copy, whose Dirichlet
    // coefficients bc_coef_kernel has just filled in
    const size_t nbc = ctx->hbc.size();
    std::vector<BcItem> dev(nbc);
    CK(cudaMemcpy(dev.data(), ctx->d_bc, nbc * sizeof(BcItem), cudaMemcpyDeviceToHost));
    std::vector<size_t> perm(nbc);
    for (size_t k = 0; k < nbc; ++k) perm[k] = k;
    auto mb = [&](size_t k) { return ctx->hinst[ctx->hbc[k].inst].M; };
    std::stable_sort(perm.begin(), perm.end(), [&](size_t a, size_t b) { return mb(a) > mb(b); });
    std::vector<BcItem> v(nbc);
    std::vector<int64_t> hist((size_t)ctx->maxM + 2, 0);
    for (size_t k = 0; k < nbc; ++k) {
      v[k] = dev[perm[k]];
      hist[(size_t)std::min(mb(perm[k]), ctx->maxM)]++;
    }
    ctx->mpre_bc.assign((size_t)ctx->maxM + 1, 0);
    int64_t acc = 0;  // items with M >= L
    for (int L = ctx->maxM; L >= 0; --L) {
      acc += hist[(size_t)L];
      ctx->mpre_bc[(size_t)L] = (int32_t)acc;
    }
    if (!ctx->d_bc_m && (st = dalloc(ctx, &ctx->d_bc_m, nbc))) return st;
    CK(cudaMemcpyAsync(ctx->d_bc_m, v.data(), nbc * sizeof(BcItem), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  } else if (ctx->msorted) {
    ctx->mpre_bc.assign((size_t)ctx->maxM + 1, 0);
  }
  ctx->prepared = true;
  ctx->adj_ready = false;
  if (ctx->adj_graph) {  // it holds this preparation's step weights and constraint lists
    cudaGraphExecDestroy(ctx->adj_graph);
    ctx->adj_graph = nullptr;
  }
  return WH_OK;
}

// A three-dimensional context: everything below the solvers lives in wh3.
static wh_status prepare3(wh_ctx *ctx, double omega) {
  wh_status st;
  if ((st = ensure_stream(ctx))) return st;
  drop_graphs(ctx);
  ctx->prepared = false;
  wh_time_info ti{};
  int64_t nc = 0, na = 0;
  if ((st = wh3::prepare(ctx->c3, ctx->opt, omega, ctx->stream, &ti, &nc, &na, ctx->err)))
    return st;
  if (ctx->ncompact != nc) {  // solver workspace is sized by the compact length
    dfree(ctx, &ctx->d_work);
    dfree(ctx, &ctx->d_q);
    ctx->q_cap = 0;
    dfree(ctx, &ctx->d_saved);
    ctx->saved = wh_ctx::SavedSolve{};
  }
  ctx->ncompact = nc;
  ctx->nactive = na;
  ctx->ti = ti;
  ctx->iti.assign(1, ti);
  ctx->ninst = 1;
  ctx->maxM = ti.M;
  ctx->err_pending = false;
  // the layout uploads are plain copies from pageable memory, which may still be in flight
  // when they return; the context's non-blocking stream must not run ahead of them
  CK(cudaStreamSynchronize(cudaStreamLegacy));
  ctx->prepared = true;
  use_set(ctx, default_set(ctx));
  return WH_OK;
}

wh_status wh_prepare(wh_ctx *ctx, double omega, wh_time_info *info) {
  if (!ctx) return WH_ERR_ARG;
  if (!(omega > 0) || !std::isfinite(omega)) return fail(ctx, WH_ERR_ARG, "omega must be > 0");
  if (ctx->dim == 3) {
    wh_status st = prepare3(ctx, omega);
    if (st) return st;
    if (info) *info = ctx->ti;
    return WH_OK;
  }
  if (ctx->grids.empty()) return fail(ctx, WH_ERR_STATE, "no grids");
  const int K = ctx->grids.back().d.instance + 1;
  std::vector<double> om(K, omega);
  wh_status st = prepare_instances(ctx, om.data());
  if (st) return st;
  if (info) *info = ctx->ti;
  return WH_OK;
}

wh_status wh_prepare_batch(wh_ctx *ctx, const double *omegas, wh_time_info *infos) {
  if (!ctx || !omegas) return fail(ctx, WH_ERR_ARG, "null omegas");
  if (ctx->dim == 3) return wh_prepare(ctx, omegas[0], infos);
  if (ctx->grids.empty()) return fail(ctx, WH_ERR_STATE, "no grids");
  wh_status st = prepare_instances(ctx, omegas);
  if (st) return st;
  if (infos)
    for (int k = 0; k < ctx->ninst; ++k) infos[k] = ctx->iti[k];
  return WH_OK;
}

wh_status wh_iterate(wh_ctx *ctx, int32_t forcing, const double *vin, double *vout) {
  if (!ctx || !vin || !vout) return fail(ctx, WH_ERR_ARG, "null vector");
  if (!ctx->prepared) return fail(ctx, WH_ERR_STATE, "wh_prepare first");
  if (vin == vout) return fail(ctx, WH_ERR_ARG, "v_in and v_out alias");
  ctx->launches = 0;
  return iterate_device(ctx, forcing, vin, vout);
}

wh_status wh_iterate_host(wh_ctx *ctx, int32_t forcing, const double *vin, double *vout) {
  if (!ctx || !vin || !vout) return fail(ctx, WH_ERR_ARG, "null vector");
  if (!ctx->prepared) return fail(ctx, WH_ERR_STATE, "wh_prepare first");
  wh_status st;
  if (!ctx->d_work && (st = dalloc(ctx, &ctx->d_work, kWorkVectors * (size_t)ctx->ncompact))) return st;
  const size_t bytes = ctx->ncompact * sizeof(double);
  ctx->launches = 0;
  CK(cudaMemcpyAsync(ctx->d_work, vin, bytes, cudaMemcpyHostToDevice, ctx->stream));
  if ((st = iterate_device(ctx, forcing, ctx->d_work, ctx->d_work + ctx->ncompact))) return st;
  CK(cudaMemcpyAsync(vout, ctx->d_work + ctx->ncompact, bytes, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return check_timeout(ctx, true);
}

wh_status wh_dot(wh_ctx *ctx, const double *x, const double *y, int64_t n, double *out) {
  if (!ctx || !out || n < 0 || (n > 0 && (!x || !y)))
    return fail(ctx, WH_ERR_ARG, "bad wh_dot arguments");
  ctx->launches = 0;
  if (n == 0) {
    *out = 0.0;
    return WH_OK;
  }
  return multidot(ctx, x, 0, 1, y, n, out);
}

wh_status wh_widen_f32(const float *x, double *out, int64_t n, void *stream) {
  if (n < 0 || (n > 0 && (!x || !out))) return WH_ERR_ARG;
  if (n == 0) return WH_OK;
  launch_widen((cudaStream_t)stream, x, out, n);
  return cudaGetLastError() == cudaSuccess ? WH_OK : WH_ERR_CUDA;
}

wh_status wh_probe_fp64(int32_t reps, double *tflops, double *ms) {
  if (reps < 1 || !tflops) return WH_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return WH_ERR_CUDA;
  const int blocks = sms * 8, iters = 4096;  // 8 blocks of 256 threads per SM
  double *out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  wh_status st = WH_ERR_CUDA;
  double best = 0.0, best_ms = 0.0;
  if (cudaMalloc(&out, (size_t)blocks * 256 * sizeof(double)) != cudaSuccess) return WH_ERR_NOMEM;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    goto done;
  launch_dfma_probe(s, blocks, iters, out);  // warm-up
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, s);
    const int64_t fmas = launch_dfma_probe(s, blocks, iters, out);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) goto done;
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    const double tf = 2.0 * (double)fmas / (t * 1e-3) / 1e12;
    if (tf > best) {
      best = tf;
      best_ms = t;
    }
  }
  st = cudaGetLastError() == cudaSuccess ? WH_OK : WH_ERR_CUDA;
  *tflops = best;
  if (ms) *ms = best_ms;
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(out);
  return st;
}

wh_status wh_solve(wh_ctx *ctx, int32_t method, double tol, int32_t max_it, int32_t restart,
                   double *u, wh_stats *stats, double *history, int32_t history_cap) {
  if (!ctx || !u || !(tol > 0) || max_it < 1 || (method != WH_FPI && method != WH_GMRES))
    return fail(ctx, WH_ERR_ARG, "bad wh_solve arguments");
  if (!ctx->prepared) return fail(ctx, WH_ERR_STATE, "wh_prepare first");
  if (method == WH_GMRES && (restart < 1 || restart > 4000))
    return fail(ctx, WH_ERR_ARG, "restart must be in [1, 4000]");
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t n = ctx->ncompact;
  wh_status st;
  if (!ctx->d_work && (st = dalloc(ctx, &ctx->d_work, kWorkVectors * (size_t)n))) return st;
  // work vectors: [0] scratch, [1] cycle residual, [2] b, [3] outer residual, [4] correction
  double *w0 = ctx->d_work, *w1 = ctx->d_work + n, *w2 = ctx->d_work + 2 * n;
  cudaStream_t s = ctx->stream;
  ctx->launches = 0;
  SolveLog L;
  L.history = history;
  L.cap = history_cap < 0 ? 0 : history_cap;
  wh_stats S{};
  auto finish = [&](wh_status code) {
    use_set(ctx, default_set(ctx));
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    S.n_history = std::min(L.n, L.cap);
    S.products_fp64 = L.products[0];
    S.products_fp32 = L.products[1];
    S.iterations = L.products[0] + L.products[1];
    if (stats) *stats = S;
    return code;
  };
  // Deflation set (Algorithm 3): checked and its forcing pairing vector built once per solve
  const int K = ctx->defl_k;
  if (K > 0) {
    if (ctx->ninst != 1) return finish(fail(ctx, WH_ERR_STATE, "deflation needs one instance"));
    if (!ctx->defl_basis && (ctx->d_gb || (ctx->dim == 3 && wh3::has_boundary_data(ctx->c3))))
      return finish(fail(ctx, WH_ERR_STATE,
                         "Algorithm 3's inflation takes g = 0; with Dirichlet data use "
                         "wh_set_deflation_basis (exact for any data)"));
    const double om2 = ctx->ti.omega * ctx->ti.omega;
    for (double l2 : ctx->defl_lam2)
      if (!ctx->defl_basis && std::fabs(om2 - l2) <= kResonanceRel * om2)
        return finish(fail(ctx, WH_ERR_ARG,
                           "omega^2 = %.17g is within %g (relative) of a deflated eigenvalue "
                           "lambda^2 = %.17g",
                           om2, kResonanceRel, l2));
    if ((st = ensure_red(ctx, K))) return finish(st);
    if (!ctx->d_fcompact && (st = dalloc(ctx, &ctx->d_fcompact, (size_t)n))) return finish(st);
    // the forcing enters the discrete Helmholtz system on discretization rows only (the
    // generalized eigenproblem A x = lambda B x of Sec. 4.4 has B = 1 there and 0 on the
    // boundary and interpolation rows), so (f, phi_m) pairs phi_m with f at those points
    std::vector<double> fc;
    compact_forcing_disc(ctx, fc);
    if ((st = h2d(ctx, ctx->d_fcompact, fc.data(), n * sizeof(double)))) return st;
  }
  // on every return: add the Helmholtz solution's components along the deflation set,
  // u += sum_m (f, phi_m) / (omega^2 - lambda_m^2) phi_m
  auto inflate = [&]() -> wh_status {
    if (K == 0) return WH_OK;
    std::vector<double> c((size_t)K);
    wh_status e;
    if (ctx->defl_basis) {
      // exact inflation: U = v + Q c with (I - T) c = Q^T W_h(v, f) (FP64 march)
      const int keep = ctx->active;
      use_set(ctx, 0);
      e = iterate_device(ctx, 1, u, w0);
      use_set(ctx, keep);
      if (e) return e;
      L.products[0] += 1;
      if ((e = multidot(ctx, ctx->defl_phi, n, K, w0, n, c.data()))) return e;
      std::vector<double> A((size_t)K * K);
      for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) A[(size_t)i * K + j] = (i == j) - ctx->defl_T[(size_t)i * K + j];
      // Gaussian elimination with partial pivoting on the small system
      for (int col = 0; col < K; ++col) {
        int piv = col;
        for (int r = col + 1; r < K; ++r)
          if (std::fabs(A[(size_t)r * K + col]) > std::fabs(A[(size_t)piv * K + col])) piv = r;
        if (!(std::fabs(A[(size_t)piv * K + col]) > 0))
          return fail(ctx, WH_ERR_ARG, "deflation basis: I - T is singular (an eigenvalue 1)");
        if (piv != col) {
          for (int j = 0; j < K; ++j) std::swap(A[(size_t)col * K + j], A[(size_t)piv * K + j]);
          std::swap(c[col], c[piv]);
        }
        for (int r = col + 1; r < K; ++r) {
          const double f = A[(size_t)r * K + col] / A[(size_t)col * K + col];
          for (int j = col; j < K; ++j) A[(size_t)r * K + j] -= f * A[(size_t)col * K + j];
          c[r] -= f * c[col];
        }
      }
      for (int r = K - 1; r >= 0; --r) {
        double t = c[r];
        for (int j = r + 1; j < K; ++j) t -= A[(size_t)r * K + j] * c[j];
        c[r] = t / A[(size_t)r * K + r];
      }
      CK(cudaMemcpyAsync(ctx->d_red, c.data(), K * sizeof(double), cudaMemcpyHostToDevice, s));
      launch_gemv_acc(grid1d(n), s, ctx->defl_phi, n, K, ctx->d_red, u, n);
      CK(cudaGetLastError());
      CK(cudaStreamSynchronize(s));
      return WH_OK;
    }
    e = multidot(ctx, ctx->defl_phi, n, K, ctx->d_fcompact, n, c.data());
    if (e) return e;
    const double om2 = ctx->ti.omega * ctx->ti.omega;
    for (int m = 0; m < K; ++m) c[m] /= om2 - ctx->defl_lam2[m];
    CK(cudaMemcpyAsync(ctx->d_red, c.data(), K * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_gemv_acc(grid1d(n), s, ctx->defl_phi, n, K, ctx->d_red, u, n);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));  // c is read by the copy above
    return WH_OK;
  };
  // a state loaded by wh_set_state is continued; a new stop replaces the saved one
  wh_ctx::SavedSolve &SV = ctx->saved;
  const bool resume = SV.resume;
  if (resume && (SV.method != method || (method == WH_GMRES && SV.restart != restart)))
    return finish(fail(ctx, WH_ERR_STATE,
                       "the loaded state is of another solve (method %d, restart %d)", SV.method,
                       SV.restart));
  SV.resume = false;
  if (!resume) {
    SV.valid = false;
    SV.cycle = false;
  }
  if (!ctx->d_saved && (st = dalloc(ctx, &ctx->d_saved, 2 * (size_t)n))) return finish(st);
  if (resume) {
    CK(cudaMemcpyAsync(u, ctx->d_saved, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    L.products[0] = SV.products[0];
    L.products[1] = SV.products[1];
  }
  // record a stop at the product budget (before any inflation touches u): the iterate (or,
  // inside an Arnoldi cycle, the gmres_cycle already kept the cycle's start) and b
  auto save_stop = [&](int phase, double prev, double dmin, int fpi_k) -> wh_status {
    SV.valid = true;
    SV.method = method;
    SV.restart = method == WH_GMRES ? restart : 0;
    SV.phase = phase;
    SV.products[0] = L.products[0];
    SV.products[1] = L.products[1];
    SV.prev = prev;
    SV.dmin = dmin;
    SV.fpi_k = fpi_k;
    SV.residual = S.residual;
    if (!SV.cycle)
      CK(cudaMemcpyAsync(ctx->d_saved, u, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (method == WH_GMRES)
      CK(cudaMemcpyAsync(ctx->d_saved + n, w2, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    return WH_OK;
  };
  if (method == WH_FPI) {  // Algorithm 1 (Algorithm 3 with a deflation set)
    double dmin = resume ? SV.dmin : 1e300;
    for (int k = resume ? SV.fpi_k : 0; k < max_it; ++k) {
      if ((st = iterate_device(ctx, 1, u, w0))) return finish(st);
      L.products[ctx->active] += 1;
      if (K > 0 && (st = defl_project(ctx, w0))) return finish(st);  // deflate
      launch_sub(grid1d(n), s, w0, u, w1, n);
      CK(cudaMemcpyAsync(u, w0, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      double d[2];
      if ((st = multidot(ctx, w1, 0, 1, w1, n, &d[0]))) return finish(st);
      if ((st = multidot(ctx, u, 0, 1, u, n, &d[1]))) return finish(st);
      const double r = std::sqrt(d[0]) / std::max(std::sqrt(d[1]), 1e-300);
      S.residual = r;
      L.add(r);
      if (!std::isfinite(r)) return finish(fail(ctx, WH_ERR_DIVERGED, "FPI residual is %g", r));
      // the map contracts every component (|beta| <= 1), so a difference that grows past
      // kGrowth times the smallest one seen means the march itself is unstable
      const double dabs = std::sqrt(d[0]);
      if (k > 0 && dabs > kGrowth * dmin)
        return finish(fail(ctx, WH_ERR_DIVERGED,
                           "FPI: ||v_%d - v_%d|| = %g grew past %g x its smallest value %g",
                           k + 1, k, dabs, kGrowth, dmin));
      dmin = std::min(dmin, dabs);
      if (r <= tol) {
        S.converged = 1;
        return finish(inflate());
      }
    }
    if ((st = save_stop(0, 0.0, dmin, max_it))) return finish(st);
    if ((st = inflate())) return finish(st);
    return finish(fail(ctx, WH_ERR_NOT_CONVERGED, "FPI: %d iterations, residual %g", max_it,
                       S.residual));
  }
  const int m = restart;
  if ((st = ensure_q(ctx, m + 1))) return finish(st);
  if ((st = ensure_red(ctx, m + 1))) return finish(st);
  // b = W_h(0, f) with the FP64 march (residuals stay in FP64); with a deflation set the
  // system is the deflated fixed point (I - P S) v = P b, P = I - Phi Phi^T, inflated on
  // return like the fixed-point iteration's
  use_set(ctx, 0);
  double bnorm;
  if (resume) {  // b (deflated when a set is installed) and its norm come with the state
    CK(cudaMemcpyAsync(w2, ctx->d_saved + n, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    bnorm = SV.bnorm;
  } else {
    CK(cudaMemsetAsync(w0, 0, n * sizeof(double), s));
    if ((st = iterate_device(ctx, 1, w0, w2))) return finish(st);
    L.products[0] += 1;
    if (K > 0) {
      if ((st = defl_project(ctx, w2))) return finish(st);
      if ((st = defl_project(ctx, u))) return finish(st);  // the guess lives in range(P) too
    }
    double bb;
    if ((st = multidot(ctx, w2, 0, 1, w2, n, &bb))) return finish(st);
    bnorm = std::sqrt(bb);
  }
  SV.bnorm = bnorm;
  struct DeflOff {  // apply_A leaves the deflated operator on every return
    wh_ctx *c;
    ~DeflOff() { c->defl_on = false; }
  } defl_off{ctx};
  ctx->defl_on = K > 0;
  if (!(bnorm > 0)) {
    CK(cudaMemsetAsync(u, 0, n * sizeof(double), s));
    S.converged = 1;
    return finish(inflate());
  }
  double *b = w2;
  const bool fp32_phase = resume ? SV.phase == 1 : default_set(ctx) == 1;
  if (fp32_phase) {
    // FP32 march: the first digits with FP32 wave solves, the rest with FP64 ones.  Phase 1:
    // GMRES(m) cycles whose products use the FP32 march (orthogonalisation, rotations and
    // the iterate stay FP64) down to max(tol, kFp32Split), or until a cycle no longer
    // halves the residual; phase 2 below: FP64 GMRES(m) from that iterate to tol, ended by a
    // true FP64 residual.  Each Krylov space is built once; refinement, which rebuilds one
    // per correction, measured ~1.9x the wave solves of FP64 GMRES on the solve benchmark.
    const double tol1 = std::max(tol, kFp32Split);
    double prev = resume ? SV.prev : 1e300;
    use_set(ctx, 1);
    while (true) {
      double res;
      bool fin;
      const int budget = max_it - (L.products[0] + L.products[1]);
      if ((st = gmres_cycle(ctx, b, u, false, m, tol1 * bnorm, budget, 1.0 / bnorm, L, &res,
                            &fin, &SV)))
        return finish(st);
      if (!fin)
        return finish(fail(ctx, WH_ERR_DIVERGED,
                           "GMRES: residual or product norm %g is not finite or exceeds %g "
                           "(unstable march)", res, kGrowth * kOpBound));
      S.residual = res / bnorm;
      if (!SV.cycle && (res <= tol1 * bnorm || res > 0.5 * prev)) break;
      if (!SV.cycle) prev = res;
      if (L.products[0] + L.products[1] >= max_it) {
        if ((st = save_stop(1, prev, 0.0, 0))) return finish(st);
        if ((st = inflate())) return finish(st);
        return finish(fail(ctx, WH_ERR_NOT_CONVERGED, "GMRES: %d products, residual %g", max_it,
                           S.residual));
      }
    }
    use_set(ctx, 0);
  }
  // FP64 GMRES(m): restart cycles, each starting from the true residual
  while (true) {
    double res;
    bool fin;
    const int budget = max_it - (L.products[0] + L.products[1]);
    if ((st = gmres_cycle(ctx, b, u, false, m, tol * bnorm, budget, 1.0 / bnorm, L, &res, &fin,
                          &SV)))
      return finish(st);
    S.residual = res / bnorm;
    if (!fin)
      return finish(fail(ctx, WH_ERR_DIVERGED,
                         "GMRES: residual or product norm %g is not finite or exceeds %g "
                         "(unstable march)", res, kGrowth * kOpBound));
    if (!SV.cycle && res <= tol * bnorm) {
      // the cycle's last value may be the Givens estimate: confirm with a true residual
      double *rr = ctx->d_work + n;
      if ((st = apply_A(ctx, u, rr, w0, L))) return finish(st);
      launch_axpby(grid1d(n), s, 1.0, b, -1.0, rr, n);
      double r2;
      if ((st = multidot(ctx, rr, 0, 1, rr, n, &r2))) return finish(st);
      S.residual = std::sqrt(r2) / bnorm;
      L.add(S.residual);
      if (S.residual <= tol) {
        S.converged = 1;
        return finish(inflate());
      }
    }
    if (L.products[0] + L.products[1] >= max_it) {
      if ((st = save_stop(0, 0.0, 0.0, 0))) return finish(st);
      if ((st = inflate())) return finish(st);
      return finish(fail(ctx, WH_ERR_NOT_CONVERGED, "GMRES: %d products, residual %g", max_it,
                         S.residual));
    }
  }
}

wh_status wh_set_deflation(wh_ctx *ctx, int32_t k, const double *phi, const double *lambda2) {
  if (!ctx) return WH_ERR_ARG;
  if (k < 0 || k > 4000) return fail(ctx, WH_ERR_ARG, "deflation set size must be in [0, 4000]");
  if (k > 0 && (!phi || !lambda2)) return fail(ctx, WH_ERR_ARG, "null deflation arrays");
  for (int m = 0; m < k; ++m)
    if (!std::isfinite(lambda2[m])) return fail(ctx, WH_ERR_ARG, "non-finite eigenvalue");
  ctx->defl_k = k;
  ctx->defl_phi = k > 0 ? phi : nullptr;
  ctx->defl_lam2.assign(lambda2 ? lambda2 : nullptr, lambda2 ? lambda2 + k : nullptr);
  ctx->defl_basis = false;
  ctx->defl_T.clear();
  return WH_OK;
}

// Byte layout of a saved solve: this header, then (cycle only) H ((m+1) x m), cs, sn (m
// each), g (m + 1) as doubles, then the device vectors: the iterate, b (GMRES), and (cycle
// only) the Krylov basis Q[0..kk].
struct StateHeader {
  char magic[8];  // "WHSOLVE"
  uint32_t version, size;
  int32_t method, restart, phase, fpi_k, cycle, kk, products0, products1, M, pad;
  int64_t n;
  double bnorm, prev, residual, dmin, omega, dt;
};

static size_t state_bytes(const wh_ctx::SavedSolve &SV, int64_t n) {
  size_t b = sizeof(StateHeader);
  if (SV.cycle) b += sizeof(double) * ((size_t)(SV.restart + 1) * SV.restart + 3 * (size_t)SV.restart + 1);
  b += sizeof(double) * (size_t)n * (SV.method == WH_GMRES ? 2 : 1);
  if (SV.cycle) b += sizeof(double) * (size_t)n * (SV.kk + 1);
  return b;
}

wh_status wh_get_state(wh_ctx *ctx, void *buf, size_t *bytes) {
  if (!ctx || !bytes) return fail(ctx, WH_ERR_ARG, "bad wh_get_state arguments");
  const wh_ctx::SavedSolve &SV = ctx->saved;
  if (!SV.valid || SV.resume)
    return fail(ctx, WH_ERR_STATE, "no stopped solve to save (wh_solve must have ended at max_it)");
  const int64_t n = ctx->ncompact;
  const size_t need = state_bytes(SV, n);
  if (!buf) {
    *bytes = need;
    return WH_OK;
  }
  if (*bytes < need) return fail(ctx, WH_ERR_ARG, "state buffer of %zu bytes, %zu needed", *bytes, need);
  StateHeader h{};
  std::memcpy(h.magic, "WHSOLVE", 8);
  h.version = 1;
  h.size = (uint32_t)sizeof(StateHeader);
  h.method = SV.method;
  h.restart = SV.restart;
  h.phase = SV.phase;
  h.fpi_k = SV.fpi_k;
  h.cycle = SV.cycle ? 1 : 0;
  h.kk = SV.kk;
  h.products0 = SV.products[0];
  h.products1 = SV.products[1];
  h.M = ctx->ti.M;
  h.n = n;
  h.bnorm = SV.bnorm;
  h.prev = SV.prev;
  h.residual = SV.residual;
  h.dmin = SV.dmin;
  h.omega = ctx->ti.omega;
  h.dt = ctx->ti.dt;
  char *p = (char *)buf;
  std::memcpy(p, &h, sizeof h);
  p += sizeof h;
  auto put = [&](const std::vector<double> &v, size_t cnt) {
    std::memcpy(p, v.data(), cnt * sizeof(double));
    p += cnt * sizeof(double);
  };
  const int m = SV.restart;
  if (SV.cycle) {
    put(SV.H, (size_t)(m + 1) * m);
    put(SV.cs, m);
    put(SV.sn, m);
    put(SV.g, (size_t)m + 1);
  }
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(p, ctx->d_saved, n * sizeof(double), cudaMemcpyDeviceToHost));
  p += n * sizeof(double);
  if (SV.method == WH_GMRES) {
    CK(cudaMemcpy(p, ctx->d_saved + n, n * sizeof(double), cudaMemcpyDeviceToHost));
    p += n * sizeof(double);
  }
  if (SV.cycle) CK(cudaMemcpy(p, ctx->d_q, (size_t)n * (SV.kk + 1) * sizeof(double), cudaMemcpyDeviceToHost));
  *bytes = need;
  return WH_OK;
}

wh_status wh_set_state(wh_ctx *ctx, const void *buf, size_t bytes) {
  if (!ctx || !buf) return fail(ctx, WH_ERR_ARG, "bad wh_set_state arguments");
  if (!ctx->prepared) return fail(ctx, WH_ERR_STATE, "wh_prepare first");
  StateHeader h;
  if (bytes < sizeof h) return fail(ctx, WH_ERR_ARG, "state buffer too short");
  std::memcpy(&h, buf, sizeof h);
  const int64_t n = ctx->ncompact;
  if (std::memcmp(h.magic, "WHSOLVE", 8) != 0 || h.version != 1 || h.size != sizeof h)
    return fail(ctx, WH_ERR_ARG, "not a saved wh_solve state");
  if ((h.method != WH_FPI && h.method != WH_GMRES) || (h.method == WH_GMRES &&
      (h.restart < 1 || h.restart > 4000 || h.kk < 0 || h.kk > h.restart)) || h.fpi_k < 0 ||
      h.products0 < 0 || h.products1 < 0 || (h.phase != 0 && h.phase != 1))
    return fail(ctx, WH_ERR_ARG, "inconsistent saved state");
  if (h.n != n || h.M != ctx->ti.M || h.omega != ctx->ti.omega || h.dt != ctx->ti.dt)
    return fail(ctx, WH_ERR_STATE, "the saved state belongs to another problem or frequency");
  if (h.phase == 1 && ctx->opt.precision != WH_FP32)
    return fail(ctx, WH_ERR_STATE, "the saved state is an FP32-march phase; the context is FP64");
  wh_ctx::SavedSolve SV;
  SV.method = h.method;
  SV.restart = h.method == WH_GMRES ? h.restart : 0;
  SV.phase = h.phase;
  SV.fpi_k = h.fpi_k;
  SV.cycle = h.cycle != 0;
  SV.kk = h.kk;
  SV.products[0] = h.products0;
  SV.products[1] = h.products1;
  SV.bnorm = h.bnorm;
  SV.prev = h.prev;
  SV.residual = h.residual;
  SV.dmin = h.dmin;
  if (bytes < state_bytes(SV, n)) return fail(ctx, WH_ERR_ARG, "state buffer too short");
  const char *p = (const char *)buf + sizeof h;
  auto get = [&](std::vector<double> &v, size_t cnt) {
    v.resize(cnt);
    std::memcpy(v.data(), p, cnt * sizeof(double));
    p += cnt * sizeof(double);
  };
  const int m = SV.restart;
  if (SV.cycle) {
    get(SV.H, (size_t)(m + 1) * m);
    get(SV.cs, m);
    get(SV.sn, m);
    get(SV.g, (size_t)m + 1);
  }
  wh_status st;
  if (!ctx->d_saved && (st = dalloc(ctx, &ctx->d_saved, 2 * (size_t)n))) return st;
  if (SV.method == WH_GMRES && (st = ensure_q(ctx, m + 1))) return st;
  CK(cudaStreamSynchronize(ctx->stream));
  if ((st = h2d(ctx, ctx->d_saved, p, n * sizeof(double)))) return st;
  p += n * sizeof(double);
  if (SV.method == WH_GMRES) {
    if ((st = h2d(ctx, ctx->d_saved + n, p, n * sizeof(double)))) return st;
    p += n * sizeof(double);
  }
  if (SV.cycle && (st = h2d(ctx, ctx->d_q, p, (size_t)n * (SV.kk + 1) * sizeof(double))))
    return st;
  SV.valid = true;
  SV.resume = true;
  ctx->saved = std::move(SV);
  return WH_OK;
}

wh_status wh_set_deflation_basis(wh_ctx *ctx, int32_t k, const double *Q, const double *T) {
  if (!ctx) return WH_ERR_ARG;
  if (k < 1 || k > 4000) return fail(ctx, WH_ERR_ARG, "deflation basis size must be in [1, 4000]");
  if (!Q || !T) return fail(ctx, WH_ERR_ARG, "null deflation arrays");
  std::vector<double> A((size_t)k * k);
  for (int64_t i = 0; i < (int64_t)k * k; ++i) {
    if (!std::isfinite(T[i])) return fail(ctx, WH_ERR_ARG, "non-finite Rayleigh matrix");
    A[i] = T[i];
  }
  ctx->defl_k = k;
  ctx->defl_phi = Q;
  ctx->defl_lam2.assign((size_t)k, 0.0);
  ctx->defl_basis = true;
  ctx->defl_T = std::move(A);
  return WH_OK;
}

wh_status wh_eigs(wh_ctx *ctx, int32_t k, int32_t m, double tol, int32_t max_products,
                  int32_t passes, uint64_t seed, double *Q, double *T, double *beta,
                  double *lambda2, wh_stats *stats) {
  if (!ctx || !Q || !beta || k < 1 || !(tol > 0) || max_products < 1 || passes < 1 ||
      passes > 2 || m < 0 || m > 2048)
    return fail(ctx, WH_ERR_ARG, "bad wh_eigs arguments");
  if (!ctx->prepared) return fail(ctx, WH_ERR_STATE, "wh_prepare first");
  if (ctx->ninst != 1) return fail(ctx, WH_ERR_STATE, "wh_eigs needs one instance");
  // default basis: wide enough for the clustered spectra of S near 1 (|beta| of many modes
  // within 1e-4 of 1 at high frequency)
  if (m == 0) m = std::min(2048, std::max(3 * k, k + 60));
  if (m < k + 2) return fail(ctx, WH_ERR_ARG, "basis size m must be at least k + 2");
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t n = ctx->ncompact;
  cudaStream_t s = ctx->stream;
  ctx->launches = 0;
  wh_status st;
  // the FP64 march throughout; the deflation set is ignored while computing a new one
  const int keep_set = ctx->active;
  use_set(ctx, 0);
  struct Restore {
    wh_ctx *c;
    int set;
    ~Restore() { use_set(c, set); }
  } restore{ctx, keep_set};
  // workspace: basis V (m + 1), scratch W (max(m, 2k)), locked/merged L (2k), eigvecs Y (k)
  const int nw = std::max(m, 2 * k);
  double *V = nullptr, *Wk = nullptr, *Lk = nullptr, *Y = nullptr;
  struct Bufs {
    wh_ctx *c;
    double **a, **b, **d, **e;
    ~Bufs() { dfree(c, a); dfree(c, b); dfree(c, d); dfree(c, e); }
  } bufs{ctx, &V, &Wk, &Lk, &Y};
  if ((st = dalloc(ctx, &V, (size_t)(m + 1) * n)) || (st = dalloc(ctx, &Wk, (size_t)nw * n)) ||
      (st = dalloc(ctx, &Lk, (size_t)2 * k * n)) || (st = dalloc(ctx, &Y, (size_t)k * n)))
    return st;
  if (!ctx->d_work && (st = dalloc(ctx, &ctx->d_work, kWorkVectors * (size_t)n))) return st;
  int products = 0;
  EigPass P1, P2;
  if ((st = eig_pass(ctx, k, m, tol, max_products, seed, nullptr, 0, V, Wk, Lk, P1, products)))
    return st;
  int kb = P1.k;  // basis vectors in Lk: Schur vectors of pass 1, then pass 2
  std::vector<double> TB = P1.T;
  bool conv = P1.converged;
  double maxres = P1.maxres;
  // the second pass only when the first converged (its span is then S-invariant, which the
  // block-triangular coupling below assumes) and a whole basis still fits in the budget
  if (passes == 2 && P1.converged && max_products - products >= m) {
    // a second Krylov sequence on P S P finds the copies of repeated eigenvalues the first
    // one only meets through rounding; the union stays invariant (S Q2 = Q2 T2 + Q1 X)
    if ((st = eig_pass(ctx, k, m, tol, max_products, seed ^ 0x5DEECE66Dull, Lk, kb, V, Wk,
                       Lk + (int64_t)kb * n, P2, products)))
      return st;
    if (!P2.converged) goto merged;  // keep the first pass's invariant subspace
    {
    const int k2 = P2.k, kt = kb + k2;
    // X = Q1^T S Q2 (k2 products)
    std::vector<double> X((size_t)kb * k2), col((size_t)kb);
    for (int j = 0; j < k2; ++j) {
      if ((st = iterate_device(ctx, 0, Lk + (int64_t)(kb + j) * n, Wk))) return st;
      ++products;
      if ((st = multidot(ctx, Lk, n, kb, Wk, n, col.data()))) return st;
      for (int i = 0; i < kb; ++i) X[(size_t)i * k2 + j] = col[i];
    }
    std::vector<double> TT((size_t)kt * kt, 0.0);
    for (int i = 0; i < kb; ++i)
      for (int j = 0; j < kb; ++j) TT[(size_t)i * kt + j] = P1.T[(size_t)i * kb + j];
    for (int i = 0; i < kb; ++i)
      for (int j = 0; j < k2; ++j) TT[(size_t)i * kt + kb + j] = X[(size_t)i * k2 + j];
    for (int i = 0; i < k2; ++i)
      for (int j = 0; j < k2; ++j) TT[(size_t)(kb + i) * kt + kb + j] = P2.T[(size_t)i * k2 + j];
    TB = TT;
    kb = kt;
    maxres = std::max(maxres, P2.maxres);
    }
  }
merged:
  // the k eigenvalues of largest modulus of T_B, their eigenvectors in the basis, and an
  // orthonormal basis of their span (Q) with its Rayleigh matrix
  SmallEig E;
  std::vector<double> Z;
  const int kk = std::min(k, kb);
  int pk = real_basis(kb, TB, kk, E, Z, true);
  if (pk < 0) return fail(ctx, WH_ERR_CUDA, "wh_eigs: the small eigenproblem did not converge");
  std::vector<double> Zy(Z.begin(), Z.begin() + (size_t)kb * pk);  // eigenvectors (lambda^2)
  std::vector<std::complex<double>> wsel;
  int pq = invariant_basis(kb, TB.data(), kk, Z, wsel);
  for (int w = kk - 1; pq > k && w >= 1; --w) pq = invariant_basis(kb, TB.data(), w, Z, wsel);
  if (pq < 0) return fail(ctx, WH_ERR_CUDA, "wh_eigs: the small eigenproblem did not converge");
  std::vector<double> Tout = project(kb, TB, pq, Z);
  double *dZ = nullptr;
  struct FreeZ {
    wh_ctx *c;
    double **p;
    ~FreeZ() { dfree(c, p); }
  } fz{ctx, &dZ};
  if ((st = dalloc(ctx, &dZ, (size_t)kb * std::max(pq, pk)))) return st;
  // both coefficient sets are uploaded on the launching stream (a plain copy would not be
  // ordered after the first product and could overwrite its operand while it runs)
  if ((st = h2d(ctx, dZ, Z.data(), (size_t)kb * pq * sizeof(double)))) return st;
  launch_gemm_tall(s, Lk, n, kb, dZ, pq, Q, n, n);
  CK(cudaGetLastError());
  if ((st = h2d(ctx, dZ, Zy.data(), (size_t)kb * pk * sizeof(double)))) return st;
  launch_gemm_tall(s, Lk, n, kb, dZ, pk, Y, n, n);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  // outputs (k entries; missing ones, when the basis came out smaller, are zero)
  for (int i = 0; i < k; ++i) beta[i] = 0.0;
  int t = 0;
  for (int q = 0; q < kb && t < kk; ++q) {
    const std::complex<double> th = E.w[E.order[q]];
    if (std::fabs(th.imag()) > 1e-8 * std::abs(th) && th.imag() < 0) continue;
    beta[t++] = th.real();
    if (t < kk && std::fabs(th.imag()) > 1e-8 * std::abs(th)) beta[t++] = th.real();
  }
  if (T) {
    for (int64_t i = 0; i < (int64_t)k * k; ++i) T[i] = 0.0;
    for (int i = 0; i < pq && i < k; ++i)
      for (int j = 0; j < pq && j < k; ++j) T[(size_t)i * k + j] = Tout[(size_t)i * pq + j];
  }
  if (lambda2) {
    double *w0 = ctx->d_work, *w1 = ctx->d_work + n;
    for (int i = 0; i < k; ++i) lambda2[i] = 0.0;
    for (int i = 0; i < pk && i < k; ++i)
      if ((st = rayleigh_lam2(ctx, Y + (int64_t)i * n, w0, w1, &lambda2[i]))) return st;
  }
  if (stats) {
    wh_stats S{};
    S.iterations = products;
    S.products_fp64 = products;
    S.converged = conv ? 1 : 0;
    S.residual = maxres;
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *stats = S;
  }
  if (pq < k) return fail(ctx, WH_ERR_NOT_CONVERGED, "wh_eigs: only %d basis vectors", pq);
  if (!conv)
    return fail(ctx, WH_ERR_NOT_CONVERGED, "wh_eigs: %d products, largest residual %g",
                products, maxres);
  return WH_OK;
}

wh_status wh_dense_invariant(int32_t m, const double *A, int32_t want, double *Q, int32_t *p) {
  if (m < 1 || m > 4096 || !A || !Q || !p || want < 1 || want > m) return WH_ERR_ARG;
  std::vector<double> Z;
  std::vector<std::complex<double>> w;
  const int q = invariant_basis(m, A, want, Z, w);
  if (q < 0) return WH_ERR_NOT_CONVERGED;
  std::copy(Z.begin(), Z.end(), Q);
  *p = q;
  return WH_OK;
}

wh_status wh_dense_eig(int32_t m, const double *A, double *w, double *V) {
  if (m < 1 || m > 4096 || !A || !w) return WH_ERR_ARG;
  std::vector<std::complex<double>> ew, EV;
  if (!dense_eig(m, A, ew, EV)) return WH_ERR_NOT_CONVERGED;
  for (int i = 0; i < m; ++i) {
    w[2 * i] = ew[i].real();
    w[2 * i + 1] = ew[i].imag();
  }
  if (V)
    for (int64_t q = 0; q < (int64_t)m * m; ++q) {
      V[2 * q] = EV[q].real();
      V[2 * q + 1] = EV[q].imag();
    }
  return WH_OK;
}

wh_status wh_solve_batch(wh_ctx *ctx, double tol, int32_t max_it, int32_t restart, double *u,
                         wh_stats *stats) {
  if (!ctx || !u || !(tol > 0) || max_it < 1 || restart < 1 || restart > 4000)
    return fail(ctx, WH_ERR_ARG, "bad wh_solve_batch arguments");
  if (ctx->dim == 3) return fail(ctx, WH_ERR_STATE, "3D contexts hold one instance: wh_solve");
  if (!ctx->prepared) return fail(ctx, WH_ERR_STATE, "wh_prepare first");
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t n = ctx->ncompact;
  const int K = ctx->ninst, m = restart;
  cudaStream_t s = ctx->stream;
  wh_status st;
  if (!ctx->d_work && (st = dalloc(ctx, &ctx->d_work, kWorkVectors * (size_t)n))) return st;
  if ((st = ensure_q(ctx, m + 1))) return st;
  if ((st = ensure_red(ctx, m + 1))) return st;
  ctx->launches = 0;
  std::vector<InstGmres> I(K);
  for (int k = 0; k < K; ++k) {
    I[k].off = ctx->icstart[k];
    I[k].len = ctx->icend[k] - ctx->icstart[k];
  }
  double *w0 = ctx->d_work, *b = ctx->d_work + 2 * n, *r = ctx->d_work + 3 * n;
  std::vector<int8_t> all(K, 1);
  auto finish = [&](wh_status code) {
    std::vector<int8_t> on(K, 1);
    set_active(ctx, on);
    use_set(ctx, default_set(ctx));
    const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats)
      for (int k = 0; k < K; ++k) {
        wh_stats &S = stats[k];
        S = wh_stats{};
        S.products_fp64 = I[k].products;
        S.products_fp32 = I[k].products32;
        S.iterations = I[k].products + I[k].products32;
        S.converged = I[k].converged;
        S.residual = I[k].bnorm > 0 ? I[k].res / I[k].bnorm : 0.0;
        S.seconds = sec;
      }
    return code;
  };
  // b = W_h(0, f) with the FP64 march, all instances
  use_set(ctx, 0);
  CK(cudaMemsetAsync(w0, 0, n * sizeof(double), s));
  if ((st = set_active(ctx, all)) || (st = iterate_device(ctx, 1, w0, b))) return finish(st);
  for (int k = 0; k < K; ++k) {
    I[k].products += 1;
    double bb;
    if ((st = multidot(ctx, b + I[k].off, 0, 1, b + I[k].off, I[k].len, &bb))) return finish(st);
    I[k].bnorm = std::sqrt(bb);
    if (!(I[k].bnorm > 0)) {
      I[k].converged = true;
      CK(cudaMemsetAsync(u + I[k].off, 0, I[k].len * sizeof(double), s));
    }
  }
  int budget = max_it - 1;
  auto all_done = [&]() {
    for (auto &G : I)
      if (!G.converged) return false;
    return true;
  };
  if (default_set(ctx) == 1) {
    // FP32 march, phase 1 (as in wh_solve): FP32 wave solves down to max(tol, kFp32Split)
    // per instance, or until an instance's cycle no longer halves its residual
    const double tol1 = std::max(tol, kFp32Split);
    std::vector<int8_t> p1(K, 0);
    std::vector<double> prev(K, 1e300);
    for (int k = 0; k < K; ++k) p1[k] = !I[k].converged;
    use_set(ctx, 1);
    auto any = [&]() {
      for (int8_t x : p1)
        if (x) return true;
      return false;
    };
    while (any() && budget > 0) {
      for (int k = 0; k < K; ++k) {
        I[k].in_cycle = p1[k] != 0;
        I[k].tol_abs = tol1 * I[k].bnorm;
      }
      if ((st = gmres_cycle_batch(ctx, b, u, false, m, budget, I))) return finish(st);
      for (int k = 0; k < K; ++k) {
        if (!p1[k]) continue;
        if (!I[k].finite) return finish(fail(ctx, WH_ERR_DIVERGED, "batched GMRES: non-finite"));
        if (I[k].res <= tol1 * I[k].bnorm || I[k].res > 0.5 * prev[k]) p1[k] = 0;
        prev[k] = I[k].res;
      }
    }
    use_set(ctx, 0);
  }
  // FP64 GMRES(m) cycles to tol, each instance confirmed by a true FP64 residual
  while (!all_done() && budget > 0) {
    for (auto &G : I) {
      G.in_cycle = !G.converged;
      G.tol_abs = tol * G.bnorm;
    }
    if ((st = gmres_cycle_batch(ctx, b, u, false, m, budget, I))) return finish(st);
    for (auto &G : I)
      if (!G.finite) return finish(fail(ctx, WH_ERR_DIVERGED, "batched GMRES: non-finite"));
    std::vector<int8_t> act(K, 0);
    for (int k = 0; k < K; ++k) act[k] = !I[k].converged;
    if ((st = apply_A_batch(ctx, u, r, w0, I, act))) return finish(st);
    --budget;
    launch_axpby(grid1d(n), s, 1.0, b, -1.0, r, n);
    for (int k = 0; k < K; ++k) {
      if (!act[k]) continue;
      double rr;
      if ((st = multidot(ctx, r + I[k].off, 0, 1, r + I[k].off, I[k].len, &rr)))
        return finish(st);
      I[k].res = std::sqrt(rr);
      if (I[k].res <= tol * I[k].bnorm) I[k].converged = true;
    }
  }
  if (all_done()) return finish(WH_OK);
  return finish(fail(ctx, WH_ERR_NOT_CONVERGED, "batched GMRES: budget of %d wave solves used",
                     max_it));
}

static wh_status adj_check(wh_ctx *ctx) {
  if (ctx->dim == 3)
    return fail(ctx, WH_ERR_STATE, "differentiation is not available on 3D contexts");
  if (!ctx->prepared) return fail(ctx, WH_ERR_STATE, "wh_prepare first");
  if (ctx->ninst != 1) return fail(ctx, WH_ERR_ARG, "differentiation needs a single instance");
  if (ctx->d_gb)
    return fail(ctx, WH_ERR_STATE, "differentiation needs zero Dirichlet data (g = 0)");
  return WH_OK;
}

wh_status wh_apply_adjoint(wh_ctx *ctx, const double *w_in, double *w_out) {
  if (!ctx || !w_in || !w_out || w_in == w_out) return fail(ctx, WH_ERR_ARG, "bad vectors");
  wh_status st = adj_check(ctx);
  if (st) return st;
  use_set(ctx, 0);
  st = apply_adjoint(ctx, w_in, w_out);
  use_set(ctx, default_set(ctx));
  return st;
}

wh_status wh_adjoint(wh_ctx *ctx, const double *u, const double *g, double tol, int32_t max_it,
                     int32_t restart, double *lam, double *grad_c2, double *grad_f,
                     wh_stats *stats) {
  if (!ctx || !u || !g || !lam || !grad_c2 || !grad_f || !(tol > 0) || max_it < 1 ||
      restart < 1 || restart > 4000)
    return fail(ctx, WH_ERR_ARG, "bad wh_adjoint arguments");
  wh_status st = adj_check(ctx);
  if (st) return st;
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t n = ctx->ncompact, total = ctx->total;
  const int ng = (int)ctx->hgrids.size();
  cudaStream_t s = ctx->stream;
  use_set(ctx, 0);
  if ((st = adj_setup(ctx))) return st;
  if (!ctx->d_work && (st = dalloc(ctx, &ctx->d_work, kWorkVectors * (size_t)n))) return st;
  if ((st = ensure_q(ctx, restart + 1))) return st;
  if ((st = ensure_red(ctx, restart + 1))) return st;
  SolveLog L;
  wh_stats S{};
  auto finish = [&](wh_status code) {
    ctx->adjoint_mode = false;
    use_set(ctx, default_set(ctx));
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    S.products_fp64 = L.products[0];
    S.iterations = L.products[0];
    if (stats) *stats = S;
    return code;
  };
  // (I - S^T) lam = g by GMRES; lam starts at 0
  ctx->adjoint_mode = true;
  CK(cudaMemsetAsync(lam, 0, n * sizeof(double), s));
  double gg;
  if ((st = multidot(ctx, g, 0, 1, g, n, &gg))) return finish(st);
  const double gnorm = std::sqrt(gg);
  if (gnorm > 0) {
    while (true) {
      double res;
      bool fin;
      const int budget = max_it - L.products[0];
      if ((st = gmres_cycle(ctx, g, lam, false, restart, tol * gnorm, budget, 1.0 / gnorm, L,
                            &res, &fin)))
        return finish(st);
      S.residual = res / gnorm;
      if (!fin) return finish(fail(ctx, WH_ERR_DIVERGED, "adjoint GMRES residual not finite"));
      if (S.residual <= tol) {
        S.converged = 1;
        break;
      }
      if (L.products[0] >= max_it) break;  // gradients of the last lam, then NOT_CONVERGED
    }
  } else {
    S.converged = 1;
  }
  ctx->adjoint_mode = false;
  // gradient sweep: d(lam . W_h(u, f))/d theta
  double *lam_ext = ctx->d_adj, *gc2 = ctx->d_adj + 5 * total, *gf = ctx->d_adj + 6 * total;
  launch_compact_to_ext(s, ctx->d_grids, ng, ctx->d_mask, lam, lam_ext, total);
  CK(cudaMemsetAsync(gc2, 0, total * sizeof(double), s));
  CK(cudaMemsetAsync(gf, 0, total * sizeof(double), s));
  double *z0;
  if ((st = adj_sweep(ctx, lam_ext, &z0, u, gc2, gf))) return finish(st);
  // the sweep accumulates c^2 dJ/dc^2
  launch_ext_to_compact(s, ctx->d_grids, ng, ctx->d_mask, gc2, grad_c2, n, 0, ctx->d_c2);
  launch_ext_to_compact(s, ctx->d_grids, ng, ctx->d_mask, gf, grad_f, n, 0);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  if (!S.converged)
    return finish(fail(ctx, WH_ERR_NOT_CONVERGED, "adjoint GMRES: %d products, residual %g",
                       max_it, S.residual));
  return finish(WH_OK);
}

wh_status wh_set_coefficient(wh_ctx *ctx, int32_t gid, const double *c2) {
  if (ctx && ctx->dim == 3)
    return fail(ctx, WH_ERR_STATE, "3D contexts take c(x)^2 in wh_add_grid3");
  if (!ctx || gid < 0 || gid >= (int)ctx->grids.size())
    return fail(ctx, WH_ERR_ARG, "bad wh_set_coefficient arguments");
  HostGrid &H = ctx->grids[gid];
  const int64_t n = (int64_t)H.d.n[0] * H.d.n[1];
  if (!c2) {
    H.c2.clear();
  } else {
    H.c2.assign(c2, c2 + n);
    for (double v : H.c2)
      if (!(v > 0) || !std::isfinite(v)) return fail(ctx, WH_ERR_ARG, "c^2 must be positive");
  }
  ctx->dirty = true;
  ctx->prepared = false;
  return WH_OK;
}

wh_status wh_set_tuning(wh_ctx *ctx, const wh_tuning *t) {
  if (!ctx || !t) return fail(ctx, WH_ERR_ARG, "bad wh_set_tuning arguments");
  if (ctx->dim == 3) {
    if (t->launch_mode != -1 || t->fold_gather != -1 || t->tile_tickets != -1 ||
        t->tma != -1 || t->pdl != -1)
      return fail(ctx, WH_ERR_STATE,
                  "3D contexts take only temporal_depth and unit_depth (other fields -1)");
    return wh3::set_blocking(ctx->c3, t->temporal_depth, t->unit_depth, ctx->err);
  }
  if (t->temporal_depth < -1 || t->temporal_depth > 1 || t->unit_depth < -1)
    return fail(ctx, WH_ERR_ARG, "temporal blocking is a three-dimensional FP32 form");
  auto tri = [](int32_t v) { return v >= -1 && v <= 1; };
  if (!tri(t->fold_gather) || !tri(t->tile_tickets) || !tri(t->tma) || !tri(t->pdl) ||
      (t->launch_mode != -1 && t->launch_mode != WH_LAUNCH_GRAPH &&
       t->launch_mode != WH_LAUNCH_PERSISTENT))
    return fail(ctx, WH_ERR_ARG, "tuning fields must be -1, 0 or 1 (launch_mode: -1 or a mode)");
  if (t->launch_mode == WH_LAUNCH_PERSISTENT && ctx->prepared && ctx->iter_blocks < 1)
    return fail(ctx, WH_ERR_CUDA, "the persistent kernel cannot be resident on this device");
  ctx->tune_fold = t->fold_gather;
  ctx->tune_tickets = t->tile_tickets;
  ctx->tune_tma = t->tma;
  ctx->tune_pdl = t->pdl;
  if (t->launch_mode != -1) ctx->persistent = t->launch_mode == WH_LAUNCH_PERSISTENT;
  drop_graphs(ctx);
  return WH_OK;
}

wh_status wh_get_tuning(const wh_ctx *ctx, wh_tuning *out) {
  if (!ctx || !out) return WH_ERR_ARG;
  *out = wh_tuning{};
  out->launch_mode = out->fold_gather = out->tile_tickets = out->tma = out->pdl = -1;
  out->temporal_depth = 1;
  out->unit_depth = 0;
  if (!ctx->prepared) return WH_ERR_STATE;
  if (ctx->dim == 3) {
    int K = 1, uz = 0;
    int64_t pts = 0, nu = 0;
    wh3::blocking(ctx->c3, &K, &uz, &pts, &nu);
    out->temporal_depth = ctx->opt.precision == WH_FP32 ? K : 1;
    out->unit_depth = uz;
    out->blocked_points = ctx->opt.precision == WH_FP32 && K > 1 ? pts : 0;
    return WH_OK;
  }
  out->launch_mode = ctx->persistent ? WH_LAUNCH_PERSISTENT : WH_LAUNCH_GRAPH;
  out->fold_gather = folds_gather(ctx) ? 1 : 0;
  out->tile_tickets = tile_tickets(ctx) ? 1 : 0;
  out->tma = uses_tma(ctx) ? 1 : 0;
  out->pdl = ctx->tune_pdl != 0 ? 1 : 0;
  return WH_OK;
}

// Three-dimensional autotuner: the FP32 march's temporal depth and unit depth.
static wh_status autotune3(wh_ctx *ctx, int32_t reps, wh_tuning *out) {
  wh_status st = WH_OK;
  const int64_t n = ctx->ncompact;
  if (!ctx->d_work && (st = dalloc(ctx, &ctx->d_work, kWorkVectors * (size_t)n))) return st;
  double *vin = ctx->d_work, *vout = ctx->d_work + n;
  cudaStream_t s = ctx->stream;
  CK(cudaMemsetAsync(vin, 0, n * sizeof(double), s));
  std::vector<std::pair<int, int>> cands;
  if (ctx->opt.precision == WH_FP32) {
    cands.push_back({1, 64});
    for (int K = 2; K <= 4; ++K)
      for (int uz : {32, 64, 128}) cands.push_back({K, uz});
  } else {
    cands.push_back({1, 64});
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = 1e300;
  int ib = -1;
  for (size_t k = 0; k < cands.size() && !st; ++k) {
    if ((st = wh3::set_blocking(ctx->c3, cands[k].first, cands[k].second, ctx->err))) break;
    if ((st = iterate_device(ctx, 1, vin, vout))) break;  // untimed (builds the graph)
    CK(cudaEventRecord(e0, s));
    for (int r = 0; r < reps && !st; ++r) st = iterate_device(ctx, 1, vin, vout);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    if (st) break;
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms / reps < best) {
      best = ms / reps;
      ib = (int)k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st || ib < 0) {
    wh3::set_blocking(ctx->c3, -1, -1, ctx->err);
    return st ? st : fail(ctx, WH_ERR_CUDA, "no layout could be timed");
  }
  if ((st = wh3::set_blocking(ctx->c3, cands[ib].first, cands[ib].second, ctx->err))) return st;
  if (out) {
    wh_get_tuning(ctx, out);
    out->ms_per_iteration = best;
    out->candidates = (int32_t)cands.size();
  }
  return WH_OK;
}

wh_status wh_autotune(wh_ctx *ctx, int32_t reps, wh_tuning *out) {
  if (!ctx || reps < 1 || reps > 1000) return fail(ctx, WH_ERR_ARG, "bad wh_autotune arguments");
  if (!ctx->prepared) return fail(ctx, WH_ERR_STATE, "wh_prepare first");
  if (ctx->dim == 3) return autotune3(ctx, reps, out);
  wh_status st;
  const int64_t n = ctx->ncompact;
  if (!ctx->d_work && (st = dalloc(ctx, &ctx->d_work, kWorkVectors * (size_t)n))) return st;
  double *vin = ctx->d_work, *vout = ctx->d_work + n;
  cudaStream_t s = ctx->stream;
  CK(cudaMemsetAsync(vin, 0, n * sizeof(double), s));
  struct Cand {
    bool persistent;
    int fold, tickets, tma, pdl;
  };
  std::vector<Cand> cands;
  const bool has_tma = ctx->set[ctx->active].tma;
  for (int pdl = 1; pdl >= 0; --pdl)
    for (int tma = has_tma ? 1 : 0; tma >= 0; --tma) {
      if (tma) {
        if (ctx->nunits > 0) cands.push_back({false, 1, 0, 1, pdl});
        cands.push_back({false, 0, 0, 1, pdl});
        continue;
      }
      if (ctx->nunits > 0) cands.push_back({false, 1, 0, 0, pdl});
      cands.push_back({false, 0, 1, 0, pdl});
      cands.push_back({false, 0, 0, 0, pdl});
    }
  if (ctx->iter_blocks >= 1) cands.push_back({true, 0, 0, has_tma ? 1 : 0, 0});
  const int sf = ctx->tune_fold, stk = ctx->tune_tickets, stm = ctx->tune_tma;
  const int spd = ctx->tune_pdl;
  const bool sp = ctx->persistent;
  auto apply = [&](const Cand &c) {
    ctx->tune_fold = c.fold;
    ctx->tune_tickets = c.tickets;
    ctx->tune_tma = c.tma;
    ctx->tune_pdl = c.pdl;
    ctx->persistent = c.persistent;
    drop_graphs(ctx);
  };
  auto restore = [&](wh_status code) {
    ctx->tune_fold = sf;
    ctx->tune_tickets = stk;
    ctx->tune_tma = stm;
    ctx->tune_pdl = spd;
    ctx->persistent = sp;
    drop_graphs(ctx);
    return code;
  };
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = 1e300;
  int ib = -1;
  for (size_t k = 0; k < cands.size(); ++k) {
    apply(cands[k]);
    if ((st = iterate_device(ctx, 1, vin, vout))) break;  // untimed (builds the graph)
    CK(cudaEventRecord(e0, s));
    for (int r = 0; r < reps && !st; ++r) st = iterate_device(ctx, 1, vin, vout);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    if (st || (st = check_timeout(ctx, true))) break;
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms / reps < best) {
      best = ms / reps;
      ib = (int)k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st || ib < 0) return restore(st ? st : fail(ctx, WH_ERR_CUDA, "no layout could be timed"));
  apply(cands[ib]);
  if (out) {
    out->launch_mode = cands[ib].persistent ? WH_LAUNCH_PERSISTENT : WH_LAUNCH_GRAPH;
    out->fold_gather = cands[ib].fold;
    out->tile_tickets = cands[ib].tickets;
    out->tma = cands[ib].tma;
    out->pdl = cands[ib].pdl;
    out->ms_per_iteration = best;
    out->candidates = (int32_t)cands.size();
    out->temporal_depth = 1;
    out->unit_depth = 0;
    out->blocked_points = 0;
  }
  return WH_OK;
}

wh_status wh_profile_kernels(wh_ctx *ctx, int32_t reps, double *ms, int32_t *counts) {
  if (!ctx || !ms || !counts || reps < 1 || reps > 10000)
    return fail(ctx, WH_ERR_ARG, "bad wh_profile_kernels arguments");
  if (!ctx->prepared) return fail(ctx, WH_ERR_STATE, "wh_prepare first");
  if (ctx->dim == 3) {
    for (int k = 0; k < 4; ++k) {
      ms[k] = 0.0;
      counts[k] = 0;
    }
    return wh3::profile(ctx->c3, ctx->active == 1, ctx->stream, reps, ms, counts, ctx->err);
  }
  const int order = ctx->opt.order;
  const bool f32 = is_fp32(ctx);
  cudaStream_t s = ctx->stream;
  const int nbc = (int)ctx->hbc.size();
  const int bc_blocks = (nbc + 255) / 256;
  const int lanes = order == 4 ? 8 : 4;
  const int bg_blocks = bc_blocks + (int)((ctx->nrecv * lanes + 255) / 256);
  const int ntiles = (int)ctx->htiles.size();
  const int nblocks = std::min(ntiles, ctx->march_blocks);
  const int blk = 256;
  const int ng = (int)ctx->hgrids.size();
  const bool fold = folds_gather(ctx);
  const GatherArgs ga = gather_args(ctx);
  GatherArgs ga_tiles{};  // tickets only, as in the iteration
  ga_tiles.ctl = ctx->d_err;
  // four bursts of `reps` back-to-back launches, each captured in a graph
  auto burst = [&](int kind) {
    for (int r = 0; r < reps; ++r) {
      void *cur = (r & 1) ? ctx->d_Wb : ctx->d_Wa, *oth = (r & 1) ? ctx->d_Wa : ctx->d_Wb;
      if (kind == 0 && fold) {
        // the folded launch, as in the iteration: steps 1, 2, ... so that the tiles' step
        // flags increase (cleared at the start and whenever the steps wrap)
        const int nn = 1 + r % std::max(ctx->maxM - 2, 1);
        if (nn == 1)
          (void)cudaMemsetAsync(ctx->d_tile_done, 0, ctx->htiles.size() * sizeof(int32_t), s);
        march_step(ctx, nn, cur, oth, 1.0, &ga);
      } else if (kind == 0) {
        march_step(ctx, 1 + (r & 1), cur, oth, 1.0, tile_tickets(ctx) ? &ga_tiles : nullptr);
      }
      else if (kind == 1 && bg_blocks)
        launch_bc_gather(f32, order, bg_blocks, s, ctx->d_bc, nbc, bc_blocks, ctx->d_didx,
                         ctx->d_dw, ctx->d_ridx, ctx->d_rinst, (int)ctx->nrecv, oth, ctx->d_F,
                         ctx->d_inst, 1, 1.0);
      else if (kind == 2)
        launch_init(f32, (unsigned)((ctx->total + blk - 1) / blk), s, ctx->d_grids, ng,
                    ctx->d_mask, ctx->d_work, ctx->d_Wa, ctx->d_V, ctx->total, ctx->d_inst, 1.0);
      else if (kind == 3)
        launch_finish(f32, (unsigned)((ctx->ncompact + blk - 1) / blk), s, ctx->d_grids, ng,
                      ctx->d_mask, ctx->d_V, ctx->d_Wa, ctx->d_Wb, ctx->d_inst,
                      ctx->d_work + ctx->ncompact, ctx->ncompact);
    }
  };
  wh_status st;
  if (!ctx->d_work && (st = dalloc(ctx, &ctx->d_work, kWorkVectors * (size_t)ctx->ncompact))) return st;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int per_iter[4] = {ctx->maxM, bg_blocks ? (fold ? 1 : ctx->maxM + 1) : 0, 1, 1};
  for (int kind = 0; kind < 4; ++kind) {
    ms[kind] = 0.0;
    counts[kind] = per_iter[kind];
    if (per_iter[kind] == 0) continue;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    burst(kind);
    CK(cudaStreamEndCapture(s, &g));
    cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(ctx, WH_ERR_CUDA, "profile graph: %s", cudaGetErrorString(e));
    CK(cudaGraphLaunch(ge, s));  // warm-up
    CK(cudaEventRecord(e0, s));
    CK(cudaGraphLaunch(ge, s));
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, e0, e1));
    ms[kind] = (double)t / reps;
    cudaGraphExecDestroy(ge);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->launches = 8 * (int64_t)reps;
  return WH_OK;
}

wh_status wh_get_time_info(const wh_ctx *ctx, wh_time_info *info) {
  if (!ctx || !info) return WH_ERR_ARG;
  if (!ctx->prepared) return WH_ERR_STATE;
  *info = ctx->ti;
  return WH_OK;
}

int64_t wh_last_launch_count(const wh_ctx *ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"
