// wh_api3.cu -- host side of the three-dimensional path of libwaveholtz (second order; fourth
// order on Cartesian grids).
//
// Validates and uploads a 3D overset grid description (component grids with masks, metrics
// and c(x)^2; explicit (p + 1)^3 interpolation), prepares one frequency (coefficients and
// the CFL bound on the device, Recipe OmegaTildeExplicit, alpha_d of Eq. alphad, stencil
// weights, per-step tables) and issues one WaveHoltz iteration as init + a CUDA graph of
// 2M + 1 kernels + output.  The solvers of wh_api.cu (fixed-point iteration, GMRES, the
// two-phase FP32 solve) drive it through iterate().
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "wh3_internal.h"

namespace wh3 {
namespace {

struct HostGrid3 {
  wh_grid3_desc d{};
  std::vector<int8_t> mask;  // compact (n2, n1, n0)
  std::vector<double> rx;    // 9 extended planes
  std::vector<double> c2;    // compact, empty for c = 1
  std::vector<double> f;     // compact
  std::vector<double> gdata; // compact Dirichlet boundary data, empty when none
  int g[3] = {1, 1, 1};
  int e[3] = {0, 0, 0};
};

}  // namespace

struct Ctx3 {
  int order = 2;  // 2, or 4 (Cartesian grids only); fixed by the context's options
  std::vector<HostGrid3> grids;
  int64_t nrecv = 0;
  std::vector<int32_t> rg, ri, rj, rk, dg, di, dj, dk;
  std::vector<double> wx, wy, wz;
  bool dirty = true, f_dirty = true, fp32_ready = false;
  std::vector<Grid3Dev> hg;
  std::vector<Tile3> tiles;
  int64_t total = 0, ncompact = 0, nactive = 0, max_ext = 0, max_compact = 0, nghost = 0;
  int64_t w_total = 0, coef_total = 0;
  std::vector<void *> allocs;
  Grid3Dev *d_grids = nullptr;
  Tile3 *d_tiles = nullptr;
  int8_t *d_mask = nullptr;
  double *d_Wa = nullptr, *d_Wb = nullptr, *d_F = nullptr, *d_V = nullptr, *d_c2 = nullptr;
  double *d_rx = nullptr, *d_coef = nullptr, *d_Wt = nullptr;
  float *d_Wa32 = nullptr, *d_Wb32 = nullptr, *d_F32 = nullptr, *d_Wt32 = nullptr;
  int64_t *d_ridx = nullptr;
  // Dirichlet points with boundary data: state indices and values
  int64_t ndir = 0;
  int64_t *d_dir_idx = nullptr;
  double *d_dir_g = nullptr;
  double omega_e = 0.0, dt = 0.0;  // the prepared time setup (host copies)
  int32_t *d_gbase = nullptr, *d_goff = nullptr, *d_gdst = nullptr, *d_gsrc = nullptr;
  double *d_gw = nullptr;
  double *d_tabs = nullptr;
  float *d_ftabs = nullptr;
  int64_t tabs_cap = 0;
  unsigned long long *d_smax = nullptr;
  int M = 0;
  double dt2 = 0.0;
  Tab3 tab{};
  cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [fp32][forcing]
  // fourth order: the ghost rules of the boundary points of Dirichlet and Neumann faces
  int64_t ng4 = 0;
  Ghost4 *d_g4 = nullptr;
  // Neumann ghost copies (grid, i, j, k of destination and source), kept for the blocking plan
  std::vector<int32_t> nghost_dst, nghost_src;  // 4 ints per copy
  // temporal blocking of the FP32 march: depth K (1 = off), unit depth along axis 2, the
  // plan they were built for, the units and the single-step (coupled) tiles, and the ring
  // of K + 2 FP32 state levels
  int tdepth = 0, unit_depth = 0;  // requested (0 = the library's choice)
  int plan_K = 1, plan_uz = 0;
  std::vector<Unit3> units;
  std::vector<Tile3> ctiles;
  Unit3 *d_units = nullptr;
  Tile3 *d_ctiles = nullptr;
  float *d_ring = nullptr;
  float *d_FM32 = nullptr;  // FP32 forcing at discretization points, NaN elsewhere
  int ring_L = 0;
  int64_t blocked_points = 0;  // points in blocked units
};

namespace {

wh_status fail3(std::string &err, wh_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  err = buf;
  return s;
}

#define CK3(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail3(err, WH_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

template <typename T>
wh_status alloc3(Ctx3 *c, T **p, size_t n, std::string &err) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
  if (e != cudaSuccess)
    return fail3(err, WH_ERR_NOMEM, "cudaMalloc of %zu bytes failed: %s", n * sizeof(T),
                 cudaGetErrorString(e));
  c->allocs.push_back((void *)*p);
  // finish the legacy-stream zero fill before any launch on a non-blocking stream
  e = cudaMemset(*p, 0, n * sizeof(T));
  if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
  if (e != cudaSuccess) return fail3(err, WH_ERR_CUDA, "cudaMemset: %s", cudaGetErrorString(e));
  return WH_OK;
}

// Release one buffer from alloc3 (after the device has finished with it).
template <typename T>
void free3(Ctx3 *c, T **p) {
  if (!*p) return;
  cudaDeviceSynchronize();
  for (size_t k = 0; k < c->allocs.size(); ++k)
    if (c->allocs[k] == (void *)*p) {
      c->allocs.erase(c->allocs.begin() + k);
      cudaFree((void *)*p);
      break;
    }
  *p = nullptr;
}

void drop_graphs3(Ctx3 *c) {
  for (auto &row : c->gexec)
    for (auto &g : row)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
}

void free_all(Ctx3 *c) {
  drop_graphs3(c);
  for (void *p : c->allocs) cudaFree(p);
  c->allocs.clear();
  c->d_grids = nullptr;
  c->d_tiles = nullptr;
  c->d_mask = nullptr;
  c->d_Wa = c->d_Wb = c->d_F = c->d_V = c->d_c2 = c->d_rx = c->d_coef = c->d_Wt = nullptr;
  c->d_Wa32 = c->d_Wb32 = c->d_F32 = c->d_Wt32 = nullptr;
  c->d_ridx = nullptr;
  c->d_gbase = c->d_goff = c->d_gdst = c->d_gsrc = nullptr;
  c->d_gw = nullptr;
  c->ng4 = 0;
  c->d_g4 = nullptr;
  c->d_tabs = nullptr;
  c->d_ftabs = nullptr;
  c->tabs_cap = 0;
  c->d_smax = nullptr;
  c->fp32_ready = false;
  c->d_units = nullptr;
  c->ndir = 0;
  c->d_dir_idx = nullptr;
  c->d_dir_g = nullptr;
  c->d_ctiles = nullptr;
  c->d_ring = nullptr;
  c->d_FM32 = nullptr;
  c->ring_L = 0;
  c->plan_K = 1;
  c->plan_uz = 0;
  c->units.clear();
  c->ctiles.clear();
}

inline bool periodic(const HostGrid3 &G, int a) { return G.d.bc[2 * a] == WH_BC_PERIODIC; }

// compact index of (i, j, k)
inline int64_t cidx(const HostGrid3 &G, int i, int j, int k) {
  return ((int64_t)k * G.d.n[1] + j) * G.d.n[0] + i;
}

// extended index (relative to the grid's base) of (i, j, k), wrapping periodic axes;
// -1 outside the extended range
inline int64_t eidx(const HostGrid3 &G, int i, int j, int k) {
  int ix[3] = {i, j, k};
  for (int a = 0; a < 3; ++a) {
    if (periodic(G, a)) ix[a] = ((ix[a] % G.d.n[a]) + G.d.n[a]) % G.d.n[a];
    if (ix[a] < -G.g[a] || ix[a] >= G.d.n[a] + G.g[a]) return -1;
  }
  return ((int64_t)(ix[2] + G.g[2]) * G.e[1] + (ix[1] + G.g[1])) * G.e[0] + (ix[0] + G.g[0]);
}

// mask at (i, j, k) with wrap; -1 outside the grid's points (ghosts included)
inline int mask_at(const HostGrid3 &G, int i, int j, int k) {
  int ix[3] = {i, j, k};
  for (int a = 0; a < 3; ++a) {
    if (periodic(G, a)) ix[a] = ((ix[a] % G.d.n[a]) + G.d.n[a]) % G.d.n[a];
    if (ix[a] < 0 || ix[a] >= G.d.n[a]) return -1;
  }
  return G.mask[cidx(G, ix[0], ix[1], ix[2])];
}

int pair_bit(int a, int b) { return 1 << (std::min(a, b) + std::max(a, b) - 1); }

// Structural checks of one grid's discretization points: a point on a non-periodic side
// must lie on a Neumann side, with a discretization or Dirichlet point inward; every grid
// point its stencil reads (the 7-point cross, plus the edges of non-orthogonal pairs) must
// be in use.
wh_status check_grid(const HostGrid3 &G, std::string &err) {
  const int n0 = G.d.n[0], n1 = G.d.n[1], n2 = G.d.n[2];
  const bool curv = G.d.kind == WH_CURVILINEAR;
  for (int k = 0; k < n2; ++k)
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n0; ++i) {
        if (G.mask[cidx(G, i, j, k)] != WH_DISC) continue;
        const int ix[3] = {i, j, k};
        for (int a = 0; a < 3; ++a) {
          if (periodic(G, a)) continue;
          for (int hi = 0; hi < 2; ++hi) {
            if (ix[a] != (hi ? G.d.n[a] - 1 : 0)) continue;
            if (G.d.bc[2 * a + hi] != WH_BC_NEUMANN)
              return fail3(err, WH_ERR_GRID,
                           "discretization point (%d,%d,%d) lies on a side without a Neumann "
                           "condition", i, j, k);
            int in[3] = {i, j, k};
            in[a] += hi ? -1 : 1;
            const int m = mask_at(G, in[0], in[1], in[2]);
            if (m != WH_DISC && m != WH_DIRICHLET)
              return fail3(err, WH_ERR_GRID,
                           "the inward neighbour of Neumann boundary point (%d,%d,%d) is not a "
                           "discretization or Dirichlet point", i, j, k);
          }
        }
        for (int a = 0; a < 3; ++a)
          for (int s = -1; s <= 1; s += 2) {
            int d[3] = {0, 0, 0};
            d[a] = s;
            const int m = mask_at(G, i + d[0], j + d[1], k + d[2]);
            if (m == WH_UNUSED)
              return fail3(err, WH_ERR_GRID,
                           "the stencil of discretization point (%d,%d,%d) reads an unused point",
                           i, j, k);
          }
        if (curv)
          for (int a = 0; a < 3; ++a)
            for (int b = a + 1; b < 3; ++b) {
              if (G.d.ortho & pair_bit(a, b)) continue;
              for (int sa = -1; sa <= 1; sa += 2)
                for (int sb = -1; sb <= 1; sb += 2) {
                  int d[3] = {0, 0, 0};
                  d[a] = sa;
                  d[b] = sb;
                  const int m = mask_at(G, i + d[0], j + d[1], k + d[2]);
                  if (m == WH_UNUSED)
                    return fail3(err, WH_ERR_GRID,
                                 "the stencil of discretization point (%d,%d,%d) reads an "
                                 "unused point", i, j, k);
                }
            }
      }
  return WH_OK;
}

// Structural checks at fourth order (Cartesian grids).  A discretization point on a
// non-periodic side must lie on a Neumann side; every grid point its 13-point stencil reads
// must be in use, and every ghost it reads must be one that a rule fills: the boundary point
// of that grid line is a discretization point of a Neumann face or a Dirichlet point of a
// Dirichlet face.  The rules read the boundary point and three points inward, which may not
// be receivers (the kernel that applies the rules rewrites receivers at the same time).
wh_status check_grid4(const HostGrid3 &G, std::string &err) {
  const int n0 = G.d.n[0], n1 = G.d.n[1], n2 = G.d.n[2];
  for (int k = 0; k < n2; ++k)
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n0; ++i) {
        if (G.mask[cidx(G, i, j, k)] != WH_DISC) continue;
        const int ix[3] = {i, j, k};
        for (int a = 0; a < 3; ++a) {
          const int na = G.d.n[a];
          if (!periodic(G, a))
            for (int hi = 0; hi < 2; ++hi)
              if (ix[a] == (hi ? na - 1 : 0) && G.d.bc[2 * a + hi] != WH_BC_NEUMANN)
                return fail3(err, WH_ERR_GRID,
                             "discretization point (%d,%d,%d) lies on a side without a Neumann "
                             "condition", i, j, k);
          for (int d = -2; d <= 2; ++d) {
            if (d == 0) continue;
            int p[3] = {i, j, k};
            p[a] += d;
            if (periodic(G, a) || (p[a] >= 0 && p[a] < na)) {
              if (mask_at(G, p[0], p[1], p[2]) == WH_UNUSED)
                return fail3(err, WH_ERR_GRID,
                             "the stencil of discretization point (%d,%d,%d) reads an unused "
                             "point", i, j, k);
              continue;
            }
            const int hi = p[a] >= na ? 1 : 0, code = G.d.bc[2 * a + hi];
            p[a] = hi ? na - 1 : 0;
            const int mb = mask_at(G, p[0], p[1], p[2]);
            if (!((code == WH_BC_NEUMANN && mb == WH_DISC) ||
                  (code == WH_BC_DIRICHLET && mb == WH_DIRICHLET)))
              return fail3(err, WH_ERR_GRID,
                           "the stencil of discretization point (%d,%d,%d) reads a ghost point "
                           "that no boundary rule fills", i, j, k);
          }
        }
      }
  for (int s = 0; s < 6; ++s) {
    const int code = G.d.bc[s];
    if (code != WH_BC_NEUMANN && code != WH_BC_DIRICHLET) continue;
    const int a = s / 2, hi = s % 2, t1 = (a + 1) % 3, t2 = (a + 2) % 3;
    for (int v = 0; v < G.d.n[t2]; ++v)
      for (int u = 0; u < G.d.n[t1]; ++u) {
        int p[3];
        p[t1] = u;
        p[t2] = v;
        p[a] = hi ? G.d.n[a] - 1 : 0;
        const int mb = mask_at(G, p[0], p[1], p[2]);
        if (mb != (code == WH_BC_NEUMANN ? WH_DISC : WH_DIRICHLET)) continue;
        for (int kk = 1; kk <= 3; ++kk) {
          int q[3] = {p[0], p[1], p[2]};
          q[a] += hi ? -kk : kk;
          if (mask_at(G, q[0], q[1], q[2]) == WH_INTERP)
            return fail3(err, WH_ERR_GRID,
                         "the fourth-order ghost rule of boundary point (%d,%d,%d) reads an "
                         "interpolation point", p[0], p[1], p[2]);
        }
      }
  }
  return WH_OK;
}

// Device layout: extended arrays of all grids in one state array (each starting on a
// 32-element boundary), tiles, masks, metrics, c^2, forcing, interpolation lists, Neumann
// ghost lists.
wh_status build_layout(Ctx3 *c, std::string &err) {
  free_all(c);
  const int ng = (int)c->grids.size();
  c->hg.assign(ng, Grid3Dev{});
  c->tiles.clear();
  int64_t base = 0, cbase = 0, wbase = 0, kbase = 0;
  c->nactive = 0;
  c->max_ext = c->max_compact = 0;
  for (int g = 0; g < ng; ++g) {
    HostGrid3 &H = c->grids[g];
    Grid3Dev &D = c->hg[g];
    D.n0 = H.d.n[0];
    D.n1 = H.d.n[1];
    D.n2 = H.d.n[2];
    D.g0 = H.g[0];
    D.g1 = H.g[1];
    D.g2 = H.g[2];
    D.e0 = H.e[0];
    D.e1 = H.e[1];
    D.e2 = H.e[2];
    D.per = (periodic(H, 0) ? 1 : 0) | (periodic(H, 1) ? 2 : 0) | (periodic(H, 2) ? 4 : 0);
    D.kind = H.d.kind;
    D.ortho = H.d.kind == WH_CARTESIAN ? 7 : H.d.ortho;
    if (c->order == 4) {  // Cartesian grids only
      D.stencil = H.c2.empty() ? kConst13 : kPoint13;
      D.nw = H.c2.empty() ? 0 : kNw13;
    } else if (H.d.kind == WH_CARTESIAN && H.c2.empty()) {
      D.stencil = kConst7;
      D.nw = 0;
    } else if (D.ortho == 7) {
      D.stencil = kPoint7;
      D.nw = kNw7;
    } else {
      D.stencil = kPoint19;
      D.nw = kNw19;
    }
    D.ext = (int64_t)D.e0 * D.e1 * D.e2;
    D.base = base;
    D.cbase = cbase;
    D.wbase = wbase;
    D.kbase = H.d.kind == WH_CURVILINEAR ? kbase : -1;
    D.rbase = D.kbase;  // metrics use the same layout as the coefficients (9 planes)
    for (int a = 0; a < 3; ++a) D.h[a] = H.d.h[a];
    base += (D.ext + 31) / 32 * 32;
    const int64_t np = (int64_t)D.n0 * D.n1 * D.n2;
    cbase += np;
    wbase += (int64_t)D.nw * D.ext;
    if (H.d.kind == WH_CURVILINEAR) kbase += (int64_t)kNcoef * D.ext;
    c->max_ext = std::max(c->max_ext, D.ext);
    c->max_compact = std::max(c->max_compact, np);
    for (int8_t m : H.mask) c->nactive += m != WH_UNUSED;
    for (int k0 = 0; k0 < D.n2; k0 += kTZ)
      for (int j0 = 0; j0 < D.n1; j0 += kTY)
        for (int i0 = 0; i0 < D.n0; i0 += kTX) c->tiles.push_back(Tile3{g, i0, j0, k0});
  }
  c->total = base;
  c->ncompact = cbase;
  c->w_total = wbase;
  c->coef_total = kbase;
  if (c->total >= (int64_t)INT32_MAX)
    return fail3(err, WH_ERR_GRID, "%lld extended points exceed 32-bit donor indices",
                 (long long)c->total);
  wh_status st;
  if ((st = alloc3(c, &c->d_grids, ng, err)) || (st = alloc3(c, &c->d_tiles, c->tiles.size(), err)) ||
      (st = alloc3(c, &c->d_mask, c->total, err)) || (st = alloc3(c, &c->d_Wa, c->total, err)) ||
      (st = alloc3(c, &c->d_Wb, c->total, err)) || (st = alloc3(c, &c->d_F, c->total, err)) ||
      (st = alloc3(c, &c->d_V, c->total, err)) || (st = alloc3(c, &c->d_c2, c->total, err)) ||
      (st = alloc3(c, &c->d_rx, c->coef_total, err)) ||
      (st = alloc3(c, &c->d_coef, c->coef_total, err)) ||
      (st = alloc3(c, &c->d_Wt, c->w_total, err)) || (st = alloc3(c, &c->d_smax, 1, err)))
    return st;
  CK3(cudaMemcpy(c->d_tiles, c->tiles.data(), c->tiles.size() * sizeof(Tile3),
                 cudaMemcpyHostToDevice));
  // per grid: mask and c^2 over the extended extent, metrics
  for (int g = 0; g < ng; ++g) {
    const HostGrid3 &H = c->grids[g];
    const Grid3Dev &D = c->hg[g];
    std::vector<int8_t> m(D.ext, (int8_t)WH_UNUSED);
    std::vector<double> c2(D.ext, 1.0);
    for (int k = 0; k < D.n2; ++k)
      for (int j = 0; j < D.n1; ++j)
        for (int i = 0; i < D.n0; ++i) {
          const int64_t q = eidx(H, i, j, k), p = cidx(H, i, j, k);
          m[q] = H.mask[p];
          if (!H.c2.empty()) c2[q] = H.c2[p];
        }
    CK3(cudaMemcpy(c->d_mask + D.base, m.data(), D.ext, cudaMemcpyHostToDevice));
    CK3(cudaMemcpy(c->d_c2 + D.base, c2.data(), D.ext * sizeof(double), cudaMemcpyHostToDevice));
    if (H.d.kind == WH_CURVILINEAR)
      CK3(cudaMemcpy(c->d_rx + D.rbase, H.rx.data(), 9 * D.ext * sizeof(double),
                     cudaMemcpyHostToDevice));
  }
  // interpolation: receiver index; donor corner index, per-axis offsets (wrapped on
  // periodic axes) and per-axis weights, as planes of R entries
  const int64_t R = c->nrecv;
  const int Wd = c->order + 1;  // donor stencil width
  std::vector<int64_t> ridx(R > 0 ? R : 1);
  std::vector<int32_t> gbase(R > 0 ? R : 1), goff(R > 0 ? R * 3 * Wd : 1);
  std::vector<double> gw(R > 0 ? R * 3 * Wd : 1);
  for (int64_t r = 0; r < R; ++r) {
    const HostGrid3 &RG = c->grids[c->rg[r]];
    ridx[r] = c->hg[c->rg[r]].base + eidx(RG, c->ri[r], c->rj[r], c->rk[r]);
    const HostGrid3 &DG = c->grids[c->dg[r]];
    const int64_t db = c->hg[c->dg[r]].base;
    const int c0[3] = {c->di[r], c->dj[r], c->dk[r]};
    const int64_t corner = eidx(DG, c0[0], c0[1], c0[2]);
    gbase[r] = (int32_t)(db + corner);
    for (int a = 0; a < 3; ++a)
      for (int t = 0; t < Wd; ++t) {
        int d[3] = {c0[0], c0[1], c0[2]};
        d[a] += t;
        goff[(Wd * a + t) * R + r] = (int32_t)(eidx(DG, d[0], d[1], d[2]) - corner);
      }
    for (int t = 0; t < Wd; ++t) {
      gw[t * R + r] = c->wx[r * Wd + t];
      gw[(Wd + t) * R + r] = c->wy[r * Wd + t];
      gw[(2 * Wd + t) * R + r] = c->wz[r * Wd + t];
    }
  }
  // Neumann ghosts next to discretization points
  std::vector<int32_t> gdst, gsrc;
  c->nghost_dst.clear();
  c->nghost_src.clear();
  for (int g = 0; g < ng && c->order == 2; ++g) {
    const HostGrid3 &H = c->grids[g];
    const int64_t b0 = c->hg[g].base;
    for (int s = 0; s < 6; ++s) {
      if (H.d.bc[s] != WH_BC_NEUMANN) continue;
      const int a = s / 2, hi = s % 2, t1 = (a + 1) % 3, t2 = (a + 2) % 3;
      for (int v = 0; v < H.d.n[t2]; ++v)
        for (int u = 0; u < H.d.n[t1]; ++u) {
          int ib[3], ig[3], in[3];
          ib[t1] = ig[t1] = in[t1] = u;
          ib[t2] = ig[t2] = in[t2] = v;
          ib[a] = hi ? H.d.n[a] - 1 : 0;
          ig[a] = hi ? H.d.n[a] : -1;
          in[a] = hi ? H.d.n[a] - 2 : 1;
          if (H.mask[cidx(H, ib[0], ib[1], ib[2])] != WH_DISC) continue;
          gdst.push_back((int32_t)(b0 + eidx(H, ig[0], ig[1], ig[2])));
          gsrc.push_back((int32_t)(b0 + eidx(H, in[0], in[1], in[2])));
          c->nghost_dst.insert(c->nghost_dst.end(), {g, ig[0], ig[1], ig[2]});
          c->nghost_src.insert(c->nghost_src.end(), {g, in[0], in[1], in[2]});
        }
    }
  }
  c->nghost = (int64_t)gdst.size();
  if (gdst.empty()) {
    gdst.push_back(0);
    gsrc.push_back(0);
  }
  if ((st = alloc3(c, &c->d_ridx, ridx.size(), err)) ||
      (st = alloc3(c, &c->d_gbase, gbase.size(), err)) ||
      (st = alloc3(c, &c->d_goff, goff.size(), err)) || (st = alloc3(c, &c->d_gw, gw.size(), err)) ||
      (st = alloc3(c, &c->d_gdst, gdst.size(), err)) ||
      (st = alloc3(c, &c->d_gsrc, gsrc.size(), err)))
    return st;
  CK3(cudaMemcpy(c->d_ridx, ridx.data(), ridx.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  CK3(cudaMemcpy(c->d_gbase, gbase.data(), gbase.size() * sizeof(int32_t),
                 cudaMemcpyHostToDevice));
  CK3(cudaMemcpy(c->d_goff, goff.data(), goff.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK3(cudaMemcpy(c->d_gw, gw.data(), gw.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK3(cudaMemcpy(c->d_gdst, gdst.data(), gdst.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  CK3(cudaMemcpy(c->d_gsrc, gsrc.data(), gsrc.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  if (c->order == 4) {
    // the fourth-order ghost rules: one item per boundary point of a Neumann face that is a
    // discretization point and per Dirichlet point of a Dirichlet face
    std::vector<Ghost4> items;
    for (int g = 0; g < ng; ++g) {
      const HostGrid3 &H = c->grids[g];
      const Grid3Dev &D = c->hg[g];
      const int64_t sa[3] = {1, (int64_t)D.e0, (int64_t)D.e0 * D.e1};
      for (int s = 0; s < 6; ++s) {
        const int code = H.d.bc[s];
        if (code != WH_BC_NEUMANN && code != WH_BC_DIRICHLET) continue;
        const int a = s / 2, hi = s % 2, t1 = (a + 1) % 3, t2 = (a + 2) % 3;
        for (int v = 0; v < H.d.n[t2]; ++v)
          for (int u = 0; u < H.d.n[t1]; ++u) {
            int p[3];
            p[t1] = u;
            p[t2] = v;
            p[a] = hi ? H.d.n[a] - 1 : 0;
            const int64_t pc = cidx(H, p[0], p[1], p[2]);
            if (H.mask[pc] != (code == WH_BC_NEUMANN ? WH_DISC : WH_DIRICHLET)) continue;
            Ghost4 it;
            it.q0 = D.base + eidx(H, p[0], p[1], p[2]);
            it.s = hi ? -sa[a] : sa[a];
            const double c2b = H.c2.empty() ? 1.0 : H.c2[pc];
            it.a2 = code == WH_BC_DIRICHLET ? c2b / (12.0 * H.d.h[a] * H.d.h[a]) : 0.0;
            items.push_back(it);
          }
      }
    }
    c->ng4 = (int64_t)items.size();
    if ((st = alloc3(c, &c->d_g4, std::max<size_t>(items.size(), 1), err))) return st;
    if (!items.empty())
      CK3(cudaMemcpy(c->d_g4, items.data(), items.size() * sizeof(Ghost4),
                     cudaMemcpyHostToDevice));
  }
  {
    // Dirichlet points of the grids with boundary data
    std::vector<int64_t> di;
    std::vector<double> dv;
    for (int g = 0; g < ng; ++g) {
      const HostGrid3 &H = c->grids[g];
      if (H.gdata.empty()) continue;
      const Grid3Dev &D = c->hg[g];
      for (int k = 0; k < D.n2; ++k)
        for (int j = 0; j < D.n1; ++j)
          for (int i = 0; i < D.n0; ++i)
            if (H.mask[cidx(H, i, j, k)] == WH_DIRICHLET) {
              di.push_back(D.base + eidx(H, i, j, k));
              dv.push_back(H.gdata[cidx(H, i, j, k)]);
            }
    }
    c->ndir = (int64_t)di.size();
    if (c->ndir) {
      if ((st = alloc3(c, &c->d_dir_idx, di.size(), err)) ||
          (st = alloc3(c, &c->d_dir_g, dv.size(), err)))
        return st;
      CK3(cudaMemcpy(c->d_dir_idx, di.data(), di.size() * sizeof(int64_t),
                     cudaMemcpyHostToDevice));
      CK3(cudaMemcpy(c->d_dir_g, dv.data(), dv.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
  }
  c->dirty = false;
  c->f_dirty = true;
  return WH_OK;
}

wh_status upload_forcing(Ctx3 *c, std::string &err) {
  for (size_t g = 0; g < c->grids.size(); ++g) {
    const HostGrid3 &H = c->grids[g];
    const Grid3Dev &D = c->hg[g];
    std::vector<double> f(D.ext, 0.0);
    if (!H.f.empty())
      for (int k = 0; k < D.n2; ++k)
        for (int j = 0; j < D.n1; ++j)
          for (int i = 0; i < D.n0; ++i) f[eidx(H, i, j, k)] = H.f[cidx(H, i, j, k)];
    CK3(cudaMemcpy(c->d_F + D.base, f.data(), D.ext * sizeof(double), cudaMemcpyHostToDevice));
  }
  c->f_dirty = false;
  c->fp32_ready = false;
  return WH_OK;
}

// Temporal blocking plan for depth K and unit depth uz (FP32 march).  Eligible grids
// (constant weights, no periodic axis) are cut into units of kTX x kUY x uz points; a unit
// is coupled (marched one step at a time, as its march tiles) when its box dilated by K - 1
// points holds a point whose value is not the march's own: a receiver (rewritten by the
// interpolation every step) or a ghost that a Neumann rule rewrites.  Every other point a
// K-step block reads is marched by the block itself or constant (Dirichlet values, unused
// points).  A blocked unit exports every intermediate level when something outside it
// reads them: a coupled neighbour (the 26 around it), a donor of the interpolation or a
// Neumann ghost source inside it.  Units without a discretization point are dropped.
wh_status plan_blocking(Ctx3 *c, int K, int uz, std::string &err) {
  c->units.clear();
  c->ctiles.clear();
  c->blocked_points = 0;
  c->plan_K = K;
  c->plan_uz = uz;
  const int ng = (int)c->grids.size();
  for (int g = 0; g < ng; ++g) {
    const HostGrid3 &H = c->grids[g];
    const Grid3Dev &D = c->hg[g];
    const int n0 = D.n0, n1 = D.n1, n2 = D.n2;
    auto add_tiles = [&](int i0, int i1, int j0, int j1, int k0, int k1) {
      for (int k = k0; k < k1; k += kTZ)
        for (int j = j0; j < j1; j += kTY)
          for (int i = i0; i < i1; i += kTX) c->ctiles.push_back(Tile3{g, i, j, k});
    };
    // the blocked kernel indexes the ring with 32-bit integers
    const bool fits = (int64_t)(K + 2) * c->total < (int64_t)INT32_MAX;
    if (K < 2 || !fits || D.stencil != kConst7 || D.per != 0) {
      add_tiles(0, n0, 0, n1, 0, n2);
      continue;
    }
    const int nux = (n0 + kTX - 1) / kTX, nuy = (n1 + kUY - 1) / kUY, nuz = (n2 + uz - 1) / uz;
    const size_t nu = (size_t)nux * nuy * nuz;
    std::vector<uint8_t> coupled(nu, 0), exporter(nu, 0), hasdisc(nu, 0);
    auto uid = [&](int ux, int uy, int uzi) { return ((size_t)uzi * nuy + uy) * nux + ux; };
    // mark every unit whose (K-1)-dilated box contains grid point (i, j, k)
    auto mark_near = [&](int i, int j, int k) {
      const int r = K - 1;
      const int ax0 = std::max(0, (i - r) >= 0 ? (i - r) / kTX : 0);
      const int ax1 = std::min(nux - 1, (i + r) / kTX);
      const int ay0 = std::max(0, (j - r) >= 0 ? (j - r) / kUY : 0);
      const int ay1 = std::min(nuy - 1, (j + r) / kUY);
      const int az0 = std::max(0, (k - r) >= 0 ? (k - r) / uz : 0);
      const int az1 = std::min(nuz - 1, (k + r) / uz);
      for (int a = az0; a <= az1; ++a)
        for (int b = ay0; b <= ay1; ++b)
          for (int d = ax0; d <= ax1; ++d) coupled[uid(d, b, a)] = 1;
    };
    auto unit_of = [&](int i, int j, int k) -> int64_t {
      if (i < 0 || j < 0 || k < 0 || i >= n0 || j >= n1 || k >= n2) return -1;
      return (int64_t)uid(i / kTX, j / kUY, k / uz);
    };
    for (int64_t r = 0; r < c->nrecv; ++r)
      if (c->rg[r] == g) mark_near(c->ri[r], c->rj[r], c->rk[r]);
    if (!H.gdata.empty())  // Dirichlet points with data change in time: single steps there
      for (int k = 0; k < n2; ++k)
        for (int j = 0; j < n1; ++j)
          for (int i = 0; i < n0; ++i)
            if (H.mask[cidx(H, i, j, k)] == WH_DIRICHLET) mark_near(i, j, k);
    for (size_t t = 0; t < c->nghost_dst.size(); t += 4)
      if (c->nghost_dst[t] == g)
        mark_near(c->nghost_dst[t + 1], c->nghost_dst[t + 2], c->nghost_dst[t + 3]);
    for (int64_t r = 0; r < c->nrecv; ++r)
      if (c->dg[r] == g)
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            for (int d = 0; d < 3; ++d) {
              const int64_t q = unit_of(c->di[r] + d, c->dj[r] + b, c->dk[r] + a);
              if (q >= 0) exporter[q] = 1;
            }
    for (size_t t = 0; t < c->nghost_src.size(); t += 4)
      if (c->nghost_src[t] == g) {
        const int64_t q =
            unit_of(c->nghost_src[t + 1], c->nghost_src[t + 2], c->nghost_src[t + 3]);
        if (q >= 0) exporter[q] = 1;
      }
    for (int k = 0; k < n2; ++k)
      for (int j = 0; j < n1; ++j)
        for (int i = 0; i < n0; ++i)
          if (H.mask[cidx(H, i, j, k)] == WH_DISC) hasdisc[uid(i / kTX, j / kUY, k / uz)] = 1;
    for (int a = 0; a < nuz; ++a)
      for (int b = 0; b < nuy; ++b)
        for (int d = 0; d < nux; ++d) {
          const size_t q = uid(d, b, a);
          const int i0 = d * kTX, j0 = b * kUY, k0 = a * uz;
          const int i1 = std::min(n0, i0 + kTX), j1 = std::min(n1, j0 + kUY),
                    k1 = std::min(n2, k0 + uz);
          if (coupled[q]) {
            add_tiles(i0, i1, j0, j1, k0, k1);
            continue;
          }
          if (!hasdisc[q]) continue;
          bool ex = exporter[q] != 0;
          for (int za = std::max(0, a - 1); za <= std::min(nuz - 1, a + 1) && !ex; ++za)
            for (int yb = std::max(0, b - 1); yb <= std::min(nuy - 1, b + 1) && !ex; ++yb)
              for (int xd = std::max(0, d - 1); xd <= std::min(nux - 1, d + 1) && !ex; ++xd)
                if (coupled[uid(xd, yb, za)]) ex = true;
          c->units.push_back(Unit3{g, i0, j0, k0, k1 - k0, ex ? 1 : 0});
          c->blocked_points += (int64_t)(i1 - i0) * (j1 - j0) * (k1 - k0);
        }
  }
  // units in plane-chunk-major order (already: k outermost per grid); upload
  wh_status st;
  free3(c, &c->d_units);  // the previous plan's lists
  free3(c, &c->d_ctiles);
  if ((st = alloc3(c, &c->d_units, std::max<size_t>(c->units.size(), 1), err)) ||
      (st = alloc3(c, &c->d_ctiles, std::max<size_t>(c->ctiles.size(), 1), err)))
    return st;
  if (!c->units.empty())
    CK3(cudaMemcpy(c->d_units, c->units.data(), c->units.size() * sizeof(Unit3),
                   cudaMemcpyHostToDevice));
  if (!c->ctiles.empty())
    CK3(cudaMemcpy(c->d_ctiles, c->ctiles.data(), c->ctiles.size() * sizeof(Tile3),
                   cudaMemcpyHostToDevice));
  if (K > 1 && !c->units.empty() && c->ring_L < K + 2) {
    // the ring: K + 2 levels (n - 1 .. n + K live during a block)
    free3(c, &c->d_ring);
    c->ring_L = 0;
    if ((st = alloc3(c, &c->d_ring, (size_t)(K + 2) * c->total, err))) return st;
    c->ring_L = K + 2;
  }
  if (K > 1 && !c->units.empty() && !c->d_FM32) {
    if ((st = alloc3(c, &c->d_FM32, c->total, err))) return st;
    launch_forcing_mask(nullptr, c->d_F32, c->d_mask, c->d_FM32, c->total);
  }
  // the unit and tile lists are plain copies from pageable memory: complete them (and the
  // mask) before a launch on the context's non-blocking stream reads them
  CK3(cudaDeviceSynchronize());
  return WH_OK;
}

bool blocked(const Ctx3 *c, bool fp32) {
  return fp32 && c->order == 2 && c->plan_K > 1 && !c->units.empty();
}

// The library's choice: depth 3 with 64-plane units when at least kAutoBlockedShare of the
// points advance in blocked units, else single steps.  Measured: on a 512^3 cube (all
// points blocked) depth 3 runs 1.27x the single-step march; on the sphere-in-box, where 86%
// are blocked, the coupled region's single steps (the curvilinear shell and patches, the
// background around the hole) cost more than blocking saves.
constexpr int kDefaultDepth = 3, kDefaultUnitDepth = 64;
constexpr double kAutoBlockedShare = 0.95;

// Build the blocking plan the requested (or default) depth calls for, if it changed.
wh_status ensure_plan(Ctx3 *c, std::string &err) {
  const int K = c->tdepth > 0 ? c->tdepth : kDefaultDepth;
  const int uz = c->unit_depth > 0 ? c->unit_depth : kDefaultUnitDepth;
  if (K == c->plan_K && uz == c->plan_uz) return WH_OK;
  drop_graphs3(c);
  wh_status st = plan_blocking(c, K, uz, err);
  if (st || c->tdepth > 0) return st;
  if ((double)c->blocked_points < kAutoBlockedShare * (double)c->ncompact)
    st = plan_blocking(c, 1, uz, err);
  return st;
}

// State pointer of level l in the FP32 ring.
inline float *ring_level(Ctx3 *c, int l) { return c->d_ring + (int64_t)(l % c->ring_L) * c->total; }

// Launches of one iteration after init (without init and output).
int64_t step_launches(const Ctx3 *c, bool fp32) {
  const int64_t dir = c->ndir ? (int64_t)c->M + 1 : 0;  // Dirichlet data, one per level
  if (!blocked(c, fp32)) return 1 + 2 * (int64_t)c->M + dir;
  const int K = c->plan_K;
  const int64_t sup = c->M > 1 ? (c->M - 1) / K : 0;
  const int64_t rest = (int64_t)c->M - 1 - sup * K;
  const int64_t cm = c->ctiles.empty() ? 0 : 1;  // coupled march launches per single step
  return 1 + 2 + sup * (1 + K * (cm + 1)) + 2 * rest + dir;
}

// The body of one iteration after init: level-0 ghost rules + interpolation, then M steps.
// Temporally blocked FP32 march: after the first step, blocks of K steps (the blocked units'
// kernel, then K single steps of the coupled tiles, each followed by the ghost rules and
// interpolation of its level), then single steps for the remainder.
void launch_steps(Ctx3 *c, bool fp32, int forcing, cudaStream_t s) {
  if (blocked(c, fp32)) {
    const double fs = forcing ? 1.0 : 0.0;
    const int K = c->plan_K;
    auto gather = [&](int level) {
      if (c->ndir)
        launch_dirichlet3(true, s, c->ndir, c->d_dir_idx, c->d_dir_g, ring_level(c, level),
                          c->d_V, fs * std::cos(c->omega_e * level * c->dt), c->tab.wf, level);
      launch_gather3(true, s, c->nrecv, c->nghost, c->d_ridx, c->d_gbase, c->d_goff, c->d_gw,
                     c->d_gdst, c->d_gsrc, ring_level(c, level), c->d_V, c->tab.wf, level);
    };
    auto single = [&](int nt, const Tile3 *tiles, int n) {
      launch_march3(true, s, nt, c->d_grids, tiles, c->d_mask, ring_level(c, n),
                    n > 0 ? ring_level(c, n - 1) : nullptr, ring_level(c, n + 1), c->d_F32,
                    c->d_Wt32, c->d_V, c->tab, n, fs);
    };
    gather(0);
    single((int)c->tiles.size(), c->d_tiles, 0);
    gather(1);
    int n = 1;
    for (; n + K <= c->M; n += K) {
      launch_march3_block(K, s, (int)c->units.size(), c->d_grids, c->d_units, c->d_FM32,
                          c->d_ring, c->total, c->ring_L, c->d_V, c->tab, n, fs);
      for (int t = 0; t < K; ++t) {
        single((int)c->ctiles.size(), c->d_ctiles, n + t);
        gather(n + t + 1);
      }
    }
    for (; n < c->M; ++n) {
      single((int)c->tiles.size(), c->d_tiles, n);
      gather(n + 1);
    }
    return;
  }
  void *Wa = fp32 ? (void *)c->d_Wa32 : (void *)c->d_Wa;
  void *Wb = fp32 ? (void *)c->d_Wb32 : (void *)c->d_Wb;
  const void *F = fp32 ? (const void *)c->d_F32 : (const void *)c->d_F;
  const void *Wt = fp32 ? (const void *)c->d_Wt32 : (const void *)c->d_Wt;
  const double fs = forcing ? 1.0 : 0.0;
  auto gather = [&](void *W, int level) {
    const double fcl = fs * std::cos(c->omega_e * level * c->dt);
    if (c->order == 4) {
      launch_gather3o4(fp32, s, c->nrecv, c->ng4, c->d_ridx, c->d_gbase, c->d_goff, c->d_gw,
                       c->d_g4, c->d_F, fcl, W, c->d_V, c->tab.wf, level);
      return;
    }
    if (c->ndir)  // Dirichlet data first: receivers may take them as donors
      launch_dirichlet3(fp32, s, c->ndir, c->d_dir_idx, c->d_dir_g, W, c->d_V, fcl, c->tab.wf,
                        level);
    launch_gather3(fp32, s, c->nrecv, c->nghost, c->d_ridx, c->d_gbase, c->d_goff, c->d_gw,
                   c->d_gdst, c->d_gsrc, W, c->d_V, c->tab.wf, level);
  };
  gather(Wa, 0);
  for (int n = 0; n < c->M; ++n) {
    void *cur = (n & 1) ? Wb : Wa;
    void *oth = (n & 1) ? Wa : Wb;
    if (c->order == 4)
      launch_march3o4(fp32, s, (int)c->tiles.size(), c->d_grids, c->d_tiles, c->d_mask, cur,
                      oth, oth, F, Wt, c->d_V, c->tab, n, fs);
    else
      launch_march3(fp32, s, (int)c->tiles.size(), c->d_grids, c->d_tiles, c->d_mask, cur, oth,
                    oth, F, Wt, c->d_V, c->tab, n, fs);
    gather(oth, n + 1);
  }
}

wh_status build_graph3(Ctx3 *c, bool fp32, int forcing, cudaStream_t s, std::string &err) {
  cudaGraph_t graph = nullptr;
  CK3(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  launch_steps(c, fp32, forcing, s);
  cudaError_t e = cudaStreamEndCapture(s, &graph);
  if (e != cudaSuccess) return fail3(err, WH_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->gexec[fp32][forcing], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess)
    return fail3(err, WH_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return WH_OK;
}

}  // namespace

Ctx3 *create() { return new (std::nothrow) Ctx3(); }

void destroy(Ctx3 *c) {
  if (!c) return;
  free_all(c);
  delete c;
}

int ngrids(const Ctx3 *c) { return c ? (int)c->grids.size() : 0; }

void compact_mask(const Ctx3 *c, std::vector<int8_t> &m) {
  m.clear();
  for (const auto &H : c->grids) m.insert(m.end(), H.mask.begin(), H.mask.end());
}

void compact_forcing(const Ctx3 *c, std::vector<double> &f) {
  f.clear();
  for (const auto &H : c->grids) {
    if (H.f.empty())
      f.insert(f.end(), H.mask.size(), 0.0);
    else
      f.insert(f.end(), H.f.begin(), H.f.end());
  }
}

wh_status first_step(Ctx3 *c, const double *y, double *wy, double *w1, cudaStream_t s,
                     std::string &err) {
  if (!c->d_Wa || c->dirty) return fail3(err, WH_ERR_STATE, "wh_prepare first");
  const int ng = (int)c->grids.size();
  launch_init3(false, s, c->d_grids, ng, c->max_ext, c->d_mask, y, c->d_Wa, c->d_V, c->tab.wf);
  // the ghost rules of level 0 only (no receivers)
  if (c->order == 4) {
    launch_gather3o4(false, s, 0, c->ng4, c->d_ridx, c->d_gbase, c->d_goff, c->d_gw, c->d_g4,
                     c->d_F, 0.0, c->d_Wa, c->d_V, c->tab.wf, 0);
    launch_march3o4(false, s, (int)c->tiles.size(), c->d_grids, c->d_tiles, c->d_mask, c->d_Wa,
                    c->d_Wb, c->d_Wb, c->d_F, c->d_Wt, c->d_V, c->tab, 0, 0.0);
  } else {
    launch_gather3(false, s, 0, c->nghost, c->d_ridx, c->d_gbase, c->d_goff, c->d_gw,
                   c->d_gdst, c->d_gsrc, c->d_Wa, c->d_V, c->tab.wf, 0);
    launch_march3(false, s, (int)c->tiles.size(), c->d_grids, c->d_tiles, c->d_mask, c->d_Wa,
                  c->d_Wb, c->d_Wb, c->d_F, c->d_Wt, c->d_V, c->tab, 0, 0.0);
  }
  launch_disc3(s, c->d_grids, ng, c->max_compact, c->d_mask, c->d_Wa, wy);
  launch_disc3(s, c->d_grids, ng, c->max_compact, c->d_mask, c->d_Wb, w1);
  CK3(cudaGetLastError());
  return WH_OK;
}

wh_status add_grid(Ctx3 *c, const wh_grid3_desc *d, int order, int32_t *id, std::string &err) {
  if (!d || !d->mask) return fail3(err, WH_ERR_ARG, "null grid description or mask");
  if (order != 2 && order != 4)
    return fail3(err, WH_ERR_ARG, "three-dimensional grids need order 2 or 4");
  if (order == 4 && d->kind != WH_CARTESIAN)
    return fail3(err, WH_ERR_ARG, "fourth order in three dimensions: Cartesian grids only");
  if (d->instance != 0)
    return fail3(err, WH_ERR_ARG, "three-dimensional contexts hold one instance");
  if (d->kind != WH_CARTESIAN && d->kind != WH_CURVILINEAR)
    return fail3(err, WH_ERR_ARG, "bad grid kind %d", d->kind);
  if (d->kind == WH_CURVILINEAR && !d->rx)
    return fail3(err, WH_ERR_ARG, "curvilinear grid without metrics");
  if (d->ortho < 0 || d->ortho > 7) return fail3(err, WH_ERR_ARG, "ortho must be in [0, 7]");
  if (c->grids.size() >= 64) return fail3(err, WH_ERR_ARG, "at most 64 grids");
  for (int s = 0; s < 6; ++s)
    if (d->bc[s] < WH_BC_NONE || d->bc[s] > WH_BC_PERIODIC)
      return fail3(err, WH_ERR_ARG, "bad boundary code on side %d", s);
  HostGrid3 H;
  H.d = *d;
  for (int a = 0; a < 3; ++a) {
    const bool p0 = d->bc[2 * a] == WH_BC_PERIODIC, p1 = d->bc[2 * a + 1] == WH_BC_PERIODIC;
    if (p0 != p1) return fail3(err, WH_ERR_ARG, "periodic sides must come in pairs");
    if (d->n[a] < (p0 ? 3 : 5))
      return fail3(err, WH_ERR_ARG, "axis %d: %d points (need >= %d)", a, d->n[a], p0 ? 3 : 5);
    if (!(d->h[a] > 0) || !std::isfinite(d->h[a]))
      return fail3(err, WH_ERR_ARG, "spacing of axis %d must be > 0", a);
    H.g[a] = p0 ? 0 : order / 2;
    H.e[a] = d->n[a] + 2 * H.g[a];
  }
  if (order == 4)
    // the fourth-order Neumann rule is unstable at corners with another physical face
    for (int s = 0; s < 6; ++s)
      for (int s2 = 0; s2 < 6; ++s2)
        if (s / 2 != s2 / 2 && d->bc[s] == WH_BC_NEUMANN &&
            (d->bc[s2] == WH_BC_NEUMANN || d->bc[s2] == WH_BC_DIRICHLET))
          return fail3(err, WH_ERR_ARG,
                       "fourth order: a Neumann face may only meet periodic or interpolation "
                       "faces");
  if (d->kind == WH_CURVILINEAR)
    for (int s = 0; s < 6; ++s) {
      if (d->bc[s] != WH_BC_NEUMANN) continue;
      const int a = s / 2;
      for (int b = 0; b < 3; ++b)
        if (b != a && !(d->ortho & pair_bit(a, b)))
          return fail3(err, WH_ERR_ARG,
                       "a Neumann side's normal axis must be orthogonal to the other two");
    }
  const int64_t np = (int64_t)d->n[0] * d->n[1] * d->n[2];
  const int64_t ext = (int64_t)H.e[0] * H.e[1] * H.e[2];
  H.mask.assign(d->mask, d->mask + np);
  for (int8_t m : H.mask)
    if (m < WH_UNUSED || m > WH_DIRICHLET) return fail3(err, WH_ERR_ARG, "bad mask value %d", m);
  if (d->kind == WH_CURVILINEAR) H.rx.assign(d->rx, d->rx + 9 * ext);
  if (d->c2) {
    H.c2.assign(d->c2, d->c2 + np);
    for (double v : H.c2)
      if (!(v > 0) || !std::isfinite(v)) return fail3(err, WH_ERR_ARG, "c^2 must be > 0");
  }
  wh_status st = order == 4 ? check_grid4(H, err) : check_grid(H, err);
  if (st) return st;
  c->order = order;
  c->grids.push_back(std::move(H));
  c->dirty = true;
  if (id) *id = (int32_t)c->grids.size() - 1;
  return WH_OK;
}

wh_status set_interp(Ctx3 *c, const wh_interp3_desc *d, std::string &err) {
  if (!d || d->n < 0) return fail3(err, WH_ERR_ARG, "bad interpolation description");
  const int64_t n = d->n;
  if (n > 0 && (!d->recv_grid || !d->recv_i || !d->recv_j || !d->recv_k || !d->donor_grid ||
                !d->donor_i0 || !d->donor_j0 || !d->donor_k0 || !d->wx || !d->wy || !d->wz))
    return fail3(err, WH_ERR_ARG, "null interpolation array");
  const int ng = (int)c->grids.size();
  const int W = c->order + 1;  // donor stencil width
  std::vector<std::vector<int8_t>> seen(ng);
  for (int g = 0; g < ng; ++g) seen[g].assign(c->grids[g].mask.size(), 0);
  for (int64_t r = 0; r < n; ++r) {
    const int g = d->recv_grid[r], dgid = d->donor_grid[r];
    if (g < 0 || g >= ng || dgid < 0 || dgid >= ng)
      return fail3(err, WH_ERR_GRID, "receiver %lld: bad grid index", (long long)r);
    const HostGrid3 &RG = c->grids[g];
    const int i = d->recv_i[r], j = d->recv_j[r], k = d->recv_k[r];
    if (i < 0 || i >= RG.d.n[0] || j < 0 || j >= RG.d.n[1] || k < 0 || k >= RG.d.n[2])
      return fail3(err, WH_ERR_GRID, "receiver %lld outside its grid", (long long)r);
    const int64_t p = cidx(RG, i, j, k);
    if (RG.mask[p] != WH_INTERP)
      return fail3(err, WH_ERR_GRID, "receiver %lld is not an interpolation point", (long long)r);
    if (seen[g][p]++)
      return fail3(err, WH_ERR_GRID, "receiver %lld listed twice", (long long)r);
    const HostGrid3 &DG = c->grids[dgid];
    const int c0[3] = {d->donor_i0[r], d->donor_j0[r], d->donor_k0[r]};
    for (int a = 0; a < 3; ++a)
      if (!periodic(DG, a) && (c0[a] < 0 || c0[a] + W - 1 >= DG.d.n[a]))
        return fail3(err, WH_ERR_GRID, "receiver %lld: donor stencil outside its grid",
                     (long long)r);
    for (int cc = 0; cc < W; ++cc)
      for (int b = 0; b < W; ++b)
        for (int a = 0; a < W; ++a) {
          const int m = mask_at(DG, c0[0] + a, c0[1] + b, c0[2] + cc);
          if (m != WH_DISC && m != WH_DIRICHLET)
            return fail3(err, WH_ERR_GRID,
                         "receiver %lld: a donor is not a discretization or Dirichlet point "
                         "(explicit interpolation)", (long long)r);
        }
    for (int a = 0; a < W; ++a)
      if (!std::isfinite(d->wx[r * W + a]) || !std::isfinite(d->wy[r * W + a]) ||
          !std::isfinite(d->wz[r * W + a]))
        return fail3(err, WH_ERR_ARG, "receiver %lld: weight not finite", (long long)r);
  }
  for (int g = 0; g < ng; ++g)
    for (size_t p = 0; p < seen[g].size(); ++p)
      if (c->grids[g].mask[p] == WH_INTERP && !seen[g][p])
        return fail3(err, WH_ERR_GRID, "grid %d: an interpolation point has no donor stencil", g);
  auto cp = [n](std::vector<int32_t> &v, const int32_t *s) { v.assign(s, s + n); };
  cp(c->rg, d->recv_grid);
  cp(c->ri, d->recv_i);
  cp(c->rj, d->recv_j);
  cp(c->rk, d->recv_k);
  cp(c->dg, d->donor_grid);
  cp(c->di, d->donor_i0);
  cp(c->dj, d->donor_j0);
  cp(c->dk, d->donor_k0);
  c->wx.assign(d->wx, d->wx + W * n);
  c->wy.assign(d->wy, d->wy + W * n);
  c->wz.assign(d->wz, d->wz + W * n);
  c->nrecv = n;
  c->dirty = true;
  return WH_OK;
}

wh_status set_forcing(Ctx3 *c, int32_t gid, const double *f, std::string &err) {
  if (gid < 0 || gid >= (int)c->grids.size() || !f)
    return fail3(err, WH_ERR_ARG, "bad grid index or null forcing");
  HostGrid3 &H = c->grids[gid];
  // validate before storing: a rejected call leaves the forcing unchanged
  for (size_t q = 0; q < H.mask.size(); ++q)
    if (!std::isfinite(f[q])) return fail3(err, WH_ERR_ARG, "non-finite forcing");
  H.f.assign(f, f + H.mask.size());
  c->f_dirty = true;
  return WH_OK;
}

wh_status set_boundary_data(Ctx3 *c, int32_t gid, const double *g, std::string &err) {
  if (gid < 0 || gid >= (int)c->grids.size())
    return fail3(err, WH_ERR_ARG, "bad boundary data arguments");
  HostGrid3 &H = c->grids[gid];
  if (g && c->order != 2)
    return fail3(err, WH_ERR_ARG, "boundary data need order 2 in three dimensions");
  if (g)
    for (size_t q = 0; q < H.mask.size(); ++q)
      if (!std::isfinite(g[q])) return fail3(err, WH_ERR_ARG, "non-finite boundary data");
  if (g)
    H.gdata.assign(g, g + H.mask.size());
  else
    H.gdata.clear();
  c->dirty = true;  // the lists of Dirichlet points and the blocking plan change
  return WH_OK;
}

bool has_boundary_data(const Ctx3 *c) {
  for (const auto &H : c->grids)
    if (!H.gdata.empty()) return true;
  return false;
}

wh_status prepare(Ctx3 *c, const wh_options &opt, double omega, cudaStream_t s,
                  wh_time_info *ti, int64_t *ncompact, int64_t *nactive, std::string &err) {
  if (c->grids.empty()) return fail3(err, WH_ERR_STATE, "no grids");
  for (const auto &H : c->grids)
    for (int8_t m : H.mask)
      if (m == WH_INTERP && c->nrecv == 0)
        return fail3(err, WH_ERR_GRID, "interpolation points but no interpolation data");
  // earlier iterations on the stream may still read the arrays rewritten below
  CK3(cudaStreamSynchronize(s));
  wh_status st;
  if (c->dirty && (st = build_layout(c, err))) return st;
  if (c->f_dirty && (st = upload_forcing(c, err))) return st;
  drop_graphs3(c);
  const int ng = (int)c->grids.size();
  CK3(cudaMemcpy(c->d_grids, c->hg.data(), ng * sizeof(Grid3Dev), cudaMemcpyHostToDevice));
  // plain copies from pageable memory may still be in flight when they return, and the
  // launches below go to a non-blocking stream: let the layout and forcing uploads land
  CK3(cudaStreamSynchronize(cudaStreamLegacy));
  CK3(cudaMemsetAsync(c->d_smax, 0, sizeof(unsigned long long), s));
  for (int g = 0; g < ng; ++g)
    launch_coef3(s, c->d_grids, g, c->hg[g], c->d_mask, c->d_rx, c->d_c2, c->d_coef, c->d_smax);
  CK3(cudaGetLastError());
  unsigned long long bits = 0;
  CK3(cudaMemcpyAsync(&bits, c->d_smax, sizeof bits, cudaMemcpyDeviceToHost, s));
  CK3(cudaStreamSynchronize(s));
  double smax;
  std::memcpy(&smax, &bits, sizeof smax);
  if (!(smax > 0) || !std::isfinite(smax))
    return fail3(err, WH_ERR_GRID, "no discretization point");
  // Eq. dtForCartesian (C = 1 at second order, sqrt(3)/2 at fourth), Recipe
  // OmegaTildeExplicit, Eq. alphad
  const double dtmax = opt.cfl * (c->order == 4 ? std::sqrt(3.0) / 2.0 : 1.0) / std::sqrt(smax);
  int Nt = (int)std::ceil(2.0 * M_PI / (omega * dtmax));
  if (Nt < 2) Nt = 2;
  double dt = 2.0 / omega * std::sin(M_PI / Nt);
  while (dt > dtmax) {
    ++Nt;
    dt = 2.0 / omega * std::sin(M_PI / Nt);
  }
  wh_time_info T{};
  T.omega = omega;
  T.dt = dt;
  T.Nt = Nt;
  T.M = opt.periods * Nt;
  T.omega_e = 2.0 * M_PI / (Nt * dt);
  T.alpha = opt.alpha_mode ? 0.5 : std::tan(T.omega_e * dt / 2) / std::tan(T.omega_e * dt);
  T.dt_max = dtmax;
  T.Tbar = T.M * dt;
  T.n_active = c->nactive;
  T.n_total = c->ncompact;
  const int M = T.M;
  c->M = M;
  c->omega_e = T.omega_e;
  c->dt = dt;
  c->dt2 = dt * dt;
  // tables: fc[0..M], wf[0..M]; fc rounded to FP32
  const int64_t len = 2 * (int64_t)(M + 1);
  if (c->tabs_cap < len) {
    if ((st = alloc3(c, &c->d_tabs, len, err)) || (st = alloc3(c, &c->d_ftabs, M + 1, err)))
      return st;
    c->tabs_cap = len;
  }
  std::vector<double> tab(len);
  std::vector<float> ftab(M + 1);
  for (int n = 0; n <= M; ++n) {
    const double cn = std::cos(T.omega_e * n * dt);
    const double sig = (n == 0 || n == M) ? 0.5 : 1.0;
    tab[n] = dt * dt * cn;
    tab[(M + 1) + n] = (2.0 / M) * sig * (cn - T.alpha / 2.0);
    ftab[n] = (float)tab[n];
  }
  CK3(cudaMemcpy(c->d_tabs, tab.data(), len * sizeof(double), cudaMemcpyHostToDevice));
  CK3(cudaMemcpy(c->d_ftabs, ftab.data(), (M + 1) * sizeof(float), cudaMemcpyHostToDevice));
  c->tab.fc = c->d_tabs;
  c->tab.wf = c->d_tabs + (M + 1);
  c->tab.fcf = c->d_ftabs;
  c->tab.dt2h = 0.5 * dt * dt;
  c->tab.dt2hf = (float)(0.5 * dt * dt);
  // constant weights (Cartesian, c = 1): centre 2 - 2 dt^2 sum 1/h^2, neighbours dt^2/h^2
  // fourth order (kConst13): centre 2 - (30/12) dt^2 sum 1/h^2, per axis the +-1 neighbours
  // (16/12) dt^2/h^2 and the +-2 neighbours -(1/12) dt^2/h^2
  for (auto &D : c->hg) {
    if (D.stencil != kConst7 && D.stencil != kConst13) continue;
    double x[3];
    for (int a = 0; a < 3; ++a) x[a] = c->dt2 / (D.h[a] * D.h[a]);
    if (D.stencil == kConst7) {
      D.cw[0] = 2.0 - 2.0 * (x[0] + x[1] + x[2]);
      for (int a = 0; a < 3; ++a) D.cw[1 + a] = x[a];
    } else {
      D.cw[0] = 2.0 - 2.5 * (x[0] + x[1] + x[2]);
      for (int a = 0; a < 3; ++a) {
        D.cw[1 + 2 * a] = x[a] * (16.0 / 12.0);
        D.cw[2 + 2 * a] = -x[a] / 12.0;
      }
    }
    for (int a = 0; a < 7; ++a) D.cwf[a] = (float)D.cw[a];
  }
  CK3(cudaMemcpy(c->d_grids, c->hg.data(), ng * sizeof(Grid3Dev), cudaMemcpyHostToDevice));
  CK3(cudaStreamSynchronize(cudaStreamLegacy));
  const bool fp32 = opt.precision == WH_FP32;
  if (fp32 && !c->d_Wa32) {
    if ((st = alloc3(c, &c->d_Wa32, c->total, err)) || (st = alloc3(c, &c->d_Wb32, c->total, err)) ||
        (st = alloc3(c, &c->d_F32, c->total, err)) || (st = alloc3(c, &c->d_Wt32, c->w_total, err)))
      return st;
  }
  for (int g = 0; g < ng; ++g) {
    if (c->hg[g].stencil == kConst7 || c->hg[g].stencil == kConst13) continue;
    if (c->hg[g].stencil == kPoint13) {
      launch_weight3o4(false, s, c->d_grids, g, c->hg[g], c->d_mask, c->d_c2, c->d_Wt, c->dt2);
      if (fp32)
        launch_weight3o4(true, s, c->d_grids, g, c->hg[g], c->d_mask, c->d_c2, c->d_Wt32,
                         c->dt2);
      continue;
    }
    launch_weight3(false, s, c->d_grids, g, c->hg[g], c->d_mask, c->d_coef, c->d_c2, c->d_Wt,
                   c->dt2);
    if (fp32)
      launch_weight3(true, s, c->d_grids, g, c->hg[g], c->d_mask, c->d_coef, c->d_c2,
                     c->d_Wt32, c->dt2);
  }
  if (fp32 && !c->fp32_ready) {
    launch_to_precision(true, s, c->d_F, c->d_F32, c->total);
    if (c->d_FM32) launch_forcing_mask(s, c->d_F32, c->d_mask, c->d_FM32, c->total);
    c->fp32_ready = true;
  }
  if (fp32 && (st = ensure_plan(c, err))) return st;
  CK3(cudaGetLastError());
  CK3(cudaStreamSynchronize(s));
  if (ti) *ti = T;
  if (ncompact) *ncompact = c->ncompact;
  if (nactive) *nactive = c->nactive;
  return WH_OK;
}

wh_status iterate(Ctx3 *c, bool fp32, int forcing, const double *vin, double *vout,
                  cudaStream_t s, int64_t *launches, std::string &err) {
  forcing = forcing ? 1 : 0;
  if (fp32 && !c->d_Wa32)
    return fail3(err, WH_ERR_STATE, "the FP32 march was not prepared");
  if (!c->gexec[fp32][forcing]) {
    wh_status st = build_graph3(c, fp32, forcing, s, err);
    if (st) return st;
  }
  const int ng = (int)c->grids.size();
  void *W0 = blocked(c, fp32) ? (void *)ring_level(c, 0)
                              : (fp32 ? (void *)c->d_Wa32 : (void *)c->d_Wa);
  launch_init3(fp32, s, c->d_grids, ng, c->max_ext, c->d_mask, vin, W0, c->d_V, c->tab.wf);
  CK3(cudaGetLastError());
  CK3(cudaGraphLaunch(c->gexec[fp32][forcing], s));
  launch_finish3(s, c->d_grids, ng, c->max_compact, c->d_V, vout);
  CK3(cudaGetLastError());
  if (launches) *launches += 2 + step_launches(c, fp32);
  return WH_OK;
}

wh_status set_blocking(Ctx3 *c, int K, int uz, std::string &err) {
  if (K != -1 && (K < 1 || K > 4))
    return fail3(err, WH_ERR_ARG, "temporal_depth must be -1 or in [1, 4]");
  if (uz != -1 && (uz < 8 || uz > 256 || uz % 8))
    return fail3(err, WH_ERR_ARG, "unit_depth must be -1 or a multiple of 8 in [8, 256]");
  c->tdepth = K < 0 ? 0 : K;
  c->unit_depth = uz < 0 ? 0 : uz;
  if (c->d_Wa32 && !c->dirty) return ensure_plan(c, err);  // FP32 march prepared
  return WH_OK;
}

void blocking(const Ctx3 *c, int *K, int *uz, int64_t *points, int64_t *units) {
  if (K) *K = c->plan_K;
  if (uz) *uz = c->plan_uz;
  if (points) *points = c->blocked_points;
  if (units) *units = (int64_t)c->units.size();
}

wh_status profile(Ctx3 *c, bool fp32, cudaStream_t s, int reps, double *ms, int32_t *counts,
                  std::string &err) {
  if (reps < 1) reps = 1;
  if (fp32 && !c->d_Wa32) return fail3(err, WH_ERR_STATE, "the FP32 march was not prepared");
  cudaEvent_t ev[2];
  for (auto &e : ev) CK3(cudaEventCreate(&e));
  // kinds: [0] single-step march, [1] ghost rules + interpolation, [2] K-step blocked march
  double tot[3] = {0, 0, 0};
  int64_t cnt[3] = {0, 0, 0};
  float t;
  wh_status st = WH_OK;
  auto timed = [&](int kind, auto &&launch) {
    if (st) return;
    cudaEventRecord(ev[0], s);
    launch();
    cudaEventRecord(ev[1], s);
    if (cudaEventSynchronize(ev[1]) != cudaSuccess ||
        cudaEventElapsedTime(&t, ev[0], ev[1]) != cudaSuccess) {
      st = fail3(err, WH_ERR_CUDA, "profile: %s", cudaGetErrorString(cudaGetLastError()));
      return;
    }
    tot[kind] += t;
    cnt[kind] += 1;
  };
  if (blocked(c, fp32)) {
    const int K = c->plan_K;
    auto gather = [&](int level) {
      timed(1, [&] {
        launch_gather3(true, s, c->nrecv, c->nghost, c->d_ridx, c->d_gbase, c->d_goff, c->d_gw,
                       c->d_gdst, c->d_gsrc, ring_level(c, level), c->d_V, c->tab.wf, level);
      });
    };
    auto single = [&](int nt, const Tile3 *tiles, int n) {
      if (nt < 1) return;
      timed(0, [&] {
        launch_march3(true, s, nt, c->d_grids, tiles, c->d_mask, ring_level(c, n),
                      n > 0 ? ring_level(c, n - 1) : nullptr, ring_level(c, n + 1), c->d_F32,
                      c->d_Wt32, c->d_V, c->tab, n, 0.0);
      });
    };
    for (int r = 0; r < reps; ++r) {
      gather(0);
      single((int)c->tiles.size(), c->d_tiles, 0);
      gather(1);
      int n = 1;
      for (; n + K <= c->M; n += K) {
        timed(2, [&] {
          launch_march3_block(K, s, (int)c->units.size(), c->d_grids, c->d_units, c->d_FM32,
                              c->d_ring, c->total, c->ring_L, c->d_V, c->tab, n, 0.0);
        });
        for (int q = 0; q < K; ++q) {
          single((int)c->ctiles.size(), c->d_ctiles, n + q);
          gather(n + q + 1);
        }
      }
      for (; n < c->M; ++n) {
        single((int)c->tiles.size(), c->d_tiles, n);
        gather(n + 1);
      }
    }
  } else {
    void *Wa = fp32 ? (void *)c->d_Wa32 : (void *)c->d_Wa;
    void *Wb = fp32 ? (void *)c->d_Wb32 : (void *)c->d_Wb;
    const void *F = fp32 ? (const void *)c->d_F32 : (const void *)c->d_F;
    const void *Wt = fp32 ? (const void *)c->d_Wt32 : (const void *)c->d_Wt;
    for (int r = 0; r < reps; ++r) {
      for (int n = 0; n < c->M; ++n) {
        void *cur = (n & 1) ? Wb : Wa;
        void *oth = (n & 1) ? Wa : Wb;
        timed(0, [&] {
          if (c->order == 4)
            launch_march3o4(fp32, s, (int)c->tiles.size(), c->d_grids, c->d_tiles, c->d_mask,
                            cur, oth, oth, F, Wt, c->d_V, c->tab, n, 0.0);
          else
            launch_march3(fp32, s, (int)c->tiles.size(), c->d_grids, c->d_tiles, c->d_mask,
                          cur, oth, oth, F, Wt, c->d_V, c->tab, n, 0.0);
        });
        timed(1, [&] {
          if (c->order == 4)
            launch_gather3o4(fp32, s, c->nrecv, c->ng4, c->d_ridx, c->d_gbase, c->d_goff,
                             c->d_gw, c->d_g4, c->d_F, 0.0, oth, c->d_V, c->tab.wf, n + 1);
          else
            launch_gather3(fp32, s, c->nrecv, c->nghost, c->d_ridx, c->d_gbase, c->d_goff,
                           c->d_gw, c->d_gdst, c->d_gsrc, oth, c->d_V, c->tab.wf, n + 1);
        });
      }
    }
  }
  for (auto &e : ev) cudaEventDestroy(e);
  if (st) return st;
  CK3(cudaGetLastError());
  for (int k = 0; k < 3; ++k) {
    if (ms) ms[k] = cnt[k] ? tot[k] / (double)cnt[k] : 0.0;  // per launch
    if (counts) counts[k] = (int32_t)(cnt[k] / reps);        // per iteration
  }
  return WH_OK;
}

}  // namespace wh3
