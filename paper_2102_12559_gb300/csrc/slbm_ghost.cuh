// slbm_ghost.cuh -- ghost-ring images of boundary cells (post-step kernel).
//
// Ghost rule (the same as the setup ghost kernel's): a periodic axis wraps; a
// non-periodic y side takes precedence at corners; OUTFLOW ghosts copy the
// nearest interior cell; INLET ghosts are the lattice equilibrium at the
// prescribed velocity and the density of the first interior cell; DIRICHLET
// ghosts are constant; DIFFUSE ghosts are a diffuse-reflection wall
// (diffuse_value).
#pragma once

#include "../../include/slbm.h"
#include "slbm_eq.cuh"

namespace slbm {

constexpr int kBandMax = 3;  // largest stencil reach (order 5)

// Ghost cell g of the ring (0 <= g < 2 G (nx + 2G) + 2 G ny) -> (gx, gy)
// (32-bit arithmetic: the ring is far smaller than 2^31 cells).
__device__ __forceinline__ void ghost_coords(int G, int nx, int ny, int g, int& gx, int& gy) {
  const int W = nx + 2 * G;
  const int nstrip = G * W;
  if (g < nstrip) {
    gy = -G + g / W; gx = -G + g % W;
  } else if (g < 2 * nstrip) {
    const int j = g - nstrip;
    gy = ny + j / W; gx = -G + j % W;
  } else if (g < 2 * nstrip + G * ny) {
    const int j = g - 2 * nstrip;
    gy = j / G; gx = -G + j % G;
  } else {
    const int j = g - 2 * nstrip - G * ny;
    gy = j / G; gx = nx + j % G;
  }
}

// Source of ghost (gx, gy) under the ghost rule: kind 0 = copy of interior
// (sx, sy); 1 = INLET equilibrium (density of interior (sx, sy), velocity
// bc[side][idx]); 2 = DIRICHLET (constant, written at setup); 3 = DIFFUSE
// wall against interior (sx, sy) with wall velocity bc[side][idx] (the axis
// along the wall is periodic, so (sx, sy) is interior).
__device__ __forceinline__ int ghost_source(int nx, int ny, int px, int py, const BcDev& bc,
                                            int gx, int gy, int& sx, int& sy, int& side,
                                            int& idx) {
  sx = px ? (gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx)) : gx;
  sy = py ? (gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy)) : gy;
  if (sy < 0 || sy >= ny) {  // non-periodic y side (wins at corners)
    side = sy < 0 ? SLBM_SIDE_YMIN : SLBM_SIDE_YMAX;
    const int xi = min(max(sx, 0), nx - 1), yi = sy < 0 ? 0 : ny - 1;
    const int kind = bc.kind[side];
    if (kind == SLBM_BC_OUTFLOW) {
      sy = yi;
    } else {
      sx = xi; sy = yi; idx = xi;
      return kind == SLBM_BC_INLET ? 1 : (kind == SLBM_BC_DIFFUSE ? 3 : 2);
    }
  }
  if (sx < 0 || sx >= nx) {  // non-periodic x side
    side = sx < 0 ? SLBM_SIDE_XMIN : SLBM_SIDE_XMAX;
    const int xi = sx < 0 ? 0 : nx - 1;
    const int kind = bc.kind[side];
    if (kind == SLBM_BC_OUTFLOW) {
      sx = xi;
    } else {
      sx = xi; idx = sy;
      return kind == SLBM_BC_INLET ? 1 : (kind == SLBM_BC_DIFFUSE ? 3 : 2);
    }
  }
  return 0;
}

// Ghost cell g: a ring cell (g < ring, ghost_coords / ghost_source) or an
// internal wall ghost (g = ring + e, BcDev::wall[e]: always a DIFFUSE wall,
// idx = -e - 1 selects its velocity in ghost_ux / ghost_uy).
__device__ __forceinline__ int ghost_cell(int G, int nx, int ny, int px, int py, const BcDev& bc,
                                          int g, int& gx, int& gy, int& sx, int& sy, int& side,
                                          int& idx) {
  const int ring = 2 * G * (nx + 2 * G) + 2 * G * ny;
  if (g >= ring) {
    const int4 w = bc.wall[g - ring];
    gx = w.x;
    gy = w.y;
    sx = w.z;
    sy = w.y;
    side = w.w;
    idx = -(g - ring) - 1;
    return 3;
  }
  ghost_coords(G, nx, ny, g, gx, gy);
  return ghost_source(nx, ny, px, py, bc, gx, gy, sx, sy, side, idx);
}

// Prescribed velocity of an INLET / DIFFUSE ghost (side, idx from ghost_cell).
__device__ __forceinline__ double ghost_ux(const BcDev& bc, int side, int idx) {
  return idx < 0 ? bc.wall_u[2 * (-idx - 1)] : bc.ux[side][idx];
}
__device__ __forceinline__ double ghost_uy(const BcDev& bc, int side, int idx) {
  return idx < 0 ? bc.wall_u[2 * (-idx - 1) + 1] : bc.uy[side][idx];
}

// Diffuse-reflection wall ghost, population i of lattice L (N nodes per axis),
// on deviations.  The wall of `side` has its normal along x (XMIN / XMAX) or y
// (YMIN / YMAX), fluid on the side of sign n.  Populations entering the fluid
// (c.n > 0) are the lattice equilibrium at the wall velocity (uwx, uwy), scaled
// to rho_w so the mass they carry into the fluid equals the mass the interior
// cell (deviations s at `sbase` in L's planes f) sends into the wall; the
// others copy that cell.  With e_j = f^L_j(1, u_w) - W_j and the symmetric
// sum A = sum_{c.n>0} (c.n) W_j = sum_{c.n<0} |c.n| W_j:
//   rho_w - 1 = (sum_{c.n<0} |c.n| s_j - sum_{c.n>0} (c.n) e_j) / (A + sum_{c.n>0} (c.n) e_j).
template <int N, class S, class R>
__device__ __forceinline__ R diffuse_value(const LatTab<R>& L, const S* f, long long plane,
                                           int sbase, int side, R uwx, R uwy, int i) {
  const bool axis_y = side >= SLBM_SIDE_YMIN;
  const R nsign = (side == SLBM_SIDE_XMIN || side == SLBM_SIDE_YMIN) ? R(1) : R(-1);
  R dx[N], dy[N];
  dphi<R>(L, N, uwx, dx);
  dphi<R>(L, N, uwy, dy);
  R s_out = R(0), e_in = R(0), a = R(0), s_i = R(0), e_i = R(0), cn_i = R(0), w_i = R(0);
#pragma unroll
  for (int jy = 0; jy < N; ++jy)
#pragma unroll
    for (int jx = 0; jx < N; ++jx) {
      const int j = jx + N * jy;
      const R cn = (axis_y ? L.c[jy] : L.c[jx]) * nsign;
      const R w = L.w1[jx] * L.w1[jy];
      const R e = L.w1[jx] * dy[jy] + dx[jx] * L.w1[jy] + dx[jx] * dy[jy];
      const R sj = from_s<R>(ldcg_s(f + (size_t)j * plane + sbase), L.sc[j]);
      if (cn < R(0)) s_out -= cn * sj;
      if (cn > R(0)) {
        e_in += cn * e;
        a += cn * w;
      }
      if (j == i) {
        s_i = sj;
        e_i = e;
        cn_i = cn;
        w_i = w;
      }
    }
  if (!(cn_i > R(0))) return s_i;
  const R drw = (s_out - e_in) / (a + e_in);
  return drw * (w_i + e_i) + e_i;
}

// INLET ghost value of population i of lattice k: the lattice equilibrium
// at density deviation dr and velocity (ux, uy), on deviations (one product
// term of the equilibrium evaluated, no per-node arrays).
template <int NL, int NH, class R>
__device__ __forceinline__ R inlet_value(const Params<R>& p, int k, int i, R dr, R ux, R uy) {
  const LatTab<R>& L = p.lat[k];
  const int n = k ? NH : NL;
  const int ix = i % n, iy = i / n;
  R hx[kMaxN], hy[kMaxN];
  gauss_dev<R>(ux, hx);
  gauss_dev<R>(uy, hy);
  R dxi = R(0), dyi = R(0);
#pragma unroll
  for (int m = 1; m < kMaxN; ++m)
    if (m < n) {
      dxi += L.vinv[ix][m] * hx[m];
      dyi += L.vinv[iy][m] * hy[m];
    }
  const R px = L.w1[ix] + dxi, py = L.w1[iy] + dyi;
  return dr * px * py + L.w1[ix] * dyi + dxi * L.w1[iy] + dxi * dyi;
}

// The N x N populations of lattice L at element `base` of its planes f, in
// the arithmetic type (load_t), and back to storage (store_t).
template <int N, class S, class R>
__device__ __forceinline__ void load_t(const LatTab<R>& L, const S* f, long long plane, int base,
                                       R (*s)[kMaxN]) {
#pragma unroll
  for (int iy = 0; iy < N; ++iy)
#pragma unroll
    for (int ix = 0; ix < N; ++ix)
      s[iy][ix] = from_s<R>(f[(size_t)(ix + N * iy) * plane + base], L.sc[ix + N * iy]);
}

template <int N, class S, class R>
__device__ __forceinline__ void store_t(const LatTab<R>& L, S* f, long long plane, int base,
                                        const R (*s)[kMaxN]) {
#pragma unroll
  for (int iy = 0; iy < N; ++iy)
#pragma unroll
    for (int ix = 0; ix < N; ++ix)
      f[(size_t)(ix + N * iy) * plane + base] = to_s<S, R>(s[iy][ix], L.isc[ix + N * iy]);
}

// Ghost coordinates along one axis that are copies of interior coordinate v
// (periodic images, OUTFLOW extrapolation), v itself first.  Returns count.
__device__ __forceinline__ int copy_images(int v, int n, int G, int periodic, int kind_lo,
                                           int kind_hi, int* out) {
  int c = 0;
  out[c++] = v;
  if (periodic) {
    if (v < G) out[c++] = v + n;
    if (v >= n - G) out[c++] = v - n;
  } else {
    if (v == 0 && kind_lo == SLBM_BC_OUTFLOW)
      for (int g = 1; g <= G; ++g) out[c++] = -g;
    if (v == n - 1 && kind_hi == SLBM_BC_OUTFLOW)
      for (int g = 0; g < G; ++g) out[c++] = n + g;
  }
  return c;
}

template <int NL, int NH, class S, class R>
__device__ void write_eq_t(const Params<R>& p, S* f0, S* f1, int base, R dr, R ux, R uy) {
  R e[kMaxN][kMaxN];
  eq_dev<R>(p.lat[0], NL, dr, ux, uy, e);
  store_t<NL, S, R>(p.lat[0], f0, p.plane, base, e);
  eq_dev<R>(p.lat[1], NH, dr, ux, uy, e);
  store_t<NH, S, R>(p.lat[1], f1, p.plane, base, e);
}

// INLET ghosts fed by interior cell (x, y) (density deviation dr): the
// equilibrium of both lattices at the side's prescribed velocity.
template <int NL, int NH, class S, class R>
__device__ void inlet_ghosts(const Params<R>& p, S* f0, S* f1, const BcDev& bc, int x, int y,
                             R dr) {
  const int G = p.G;
  const bool inx0 = !p.periodic_x && x == 0 && bc.kind[SLBM_SIDE_XMIN] == SLBM_BC_INLET;
  const bool inx1 = !p.periodic_x && x == p.nx - 1 && bc.kind[SLBM_SIDE_XMAX] == SLBM_BC_INLET;
  const bool iny0 = !p.periodic_y && y == 0 && bc.kind[SLBM_SIDE_YMIN] == SLBM_BC_INLET;
  const bool iny1 = !p.periodic_y && y == p.ny - 1 && bc.kind[SLBM_SIDE_YMAX] == SLBM_BC_INLET;
  if (inx0 || inx1) {  // x side: this row and its copy-type y images
    int ys[2 * kBandMax + 2];
    const int nyc = copy_images(y, p.ny, G, p.periodic_y, bc.kind[SLBM_SIDE_YMIN],
                                bc.kind[SLBM_SIDE_YMAX], ys);
    const int side = inx0 ? SLBM_SIDE_XMIN : SLBM_SIDE_XMAX;
    const R ux = (R)bc.ux[side][y], uy = (R)bc.uy[side][y];
    for (int a = 0; a < nyc; ++a)
      for (int g = 1; g <= G; ++g) {
        const int gx = inx0 ? -g : p.nx - 1 + g;
        write_eq_t<NL, NH, S, R>(p, f0, f1, (ys[a] + G) * p.pitch + (gx + kOX), dr, ux, uy);
      }
  }
  if (iny0 || iny1) {  // y side wins at corners: columns = copy images and clamped corners
    const int side = iny0 ? SLBM_SIDE_YMIN : SLBM_SIDE_YMAX;
    const R ux = (R)bc.ux[side][x], uy = (R)bc.uy[side][x];
    int cols[2 * kBandMax + 2];
    int nc = 0;
    cols[nc++] = x;
    if (p.periodic_x) {
      if (x < G) cols[nc++] = x + p.nx;
      if (x >= p.nx - G) cols[nc++] = x - p.nx;
    } else {
      if (x == 0)
        for (int g = 1; g <= G; ++g) cols[nc++] = -g;
      if (x == p.nx - 1)
        for (int g = 0; g < G; ++g) cols[nc++] = p.nx + g;
    }
    for (int b = 0; b < nc; ++b)
      for (int g = 1; g <= G; ++g) {
        const int gy = iny0 ? -g : p.ny - 1 + g;
        write_eq_t<NL, NH, S, R>(p, f0, f1, (gy + G) * p.pitch + (cols[b] + kOX), dr, ux, uy);
      }
  }
}

// Element offsets of the copy-type ghost images of interior cell (x, y)
// (periodic images, OUTFLOW copies; the cell itself excluded).  Returns the
// count (at most 15).
template <class R>
__device__ __forceinline__ int copy_image_bases(const Params<R>& p, const BcDev& bc, int x, int y,
                                                int* out) {
  int xs[2 * kBandMax + 2], ys[2 * kBandMax + 2];
  const int nxc = copy_images(x, p.nx, p.G, p.periodic_x, bc.kind[SLBM_SIDE_XMIN],
                              bc.kind[SLBM_SIDE_XMAX], xs);
  const int nyc = copy_images(y, p.ny, p.G, p.periodic_y, bc.kind[SLBM_SIDE_YMIN],
                              bc.kind[SLBM_SIDE_YMAX], ys);
  int n = 0;
  for (int a = 0; a < nyc; ++a)
    for (int b = 0; b < nxc; ++b)
      if (a || b) out[n++] = (ys[a] + p.G) * p.pitch + (xs[b] + kOX);
  return n;
}

// Every ghost image of boundary cell (x, y) whose own lattice is `flag`: all
// planes of both lattices to its copy images, then its INLET ghosts.
template <int NL, int NH, class S, class R>
__device__ void boundary_images(const Params<R>& p, S* f0, S* f1, const BcDev& bc, int x, int y,
                                int flag) {
  constexpr int QL = NL * NL, QH = NH * NH;
  const int src = (y + p.G) * p.pitch + (x + kOX);
  int img[16];
  const int n = copy_image_bases(p, bc, x, y, img);
  if (n) {
    // all loads first: stores through f0 / f1 may alias later loads for the
    // compiler, which would otherwise serialise one L2 round trip per plane
    S v0[QL], v1[QH];
#pragma unroll
    for (int i = 0; i < QL; ++i) v0[i] = f0[(size_t)i * p.plane + src];
#pragma unroll
    for (int i = 0; i < QH; ++i) v1[i] = f1[(size_t)i * p.plane + src];
    for (int m = 0; m < n; ++m) {
#pragma unroll
      for (int i = 0; i < QL; ++i) f0[(size_t)i * p.plane + img[m]] = v0[i];
#pragma unroll
      for (int i = 0; i < QH; ++i) f1[(size_t)i * p.plane + img[m]] = v1[i];
    }
  }
  const bool inlet = (!p.periodic_x && ((x == 0 && bc.kind[SLBM_SIDE_XMIN] == SLBM_BC_INLET) ||
                                        (x == p.nx - 1 && bc.kind[SLBM_SIDE_XMAX] == SLBM_BC_INLET))) ||
                     (!p.periodic_y && ((y == 0 && bc.kind[SLBM_SIDE_YMIN] == SLBM_BC_INLET) ||
                                        (y == p.ny - 1 && bc.kind[SLBM_SIDE_YMAX] == SLBM_BC_INLET)));
  if (!inlet) return;
  double r = 0.0;
  if (flag) {
#pragma unroll
    for (int i = 0; i < QH; ++i) r += (double)f1[(size_t)i * p.plane + src];
  } else {
#pragma unroll
    for (int i = 0; i < QL; ++i) r += (double)f0[(size_t)i * p.plane + src];
  }
  inlet_ghosts<NL, NH, S, R>(p, f0, f1, bc, x, y, (R)r);
}

}  // namespace slbm
