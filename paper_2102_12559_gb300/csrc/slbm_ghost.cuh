// slbm_ghost.cuh -- ghost-ring images of boundary cells (post-step kernel).
//
// Ghost rule (the same as the setup ghost kernel's): a periodic axis wraps; a
// non-periodic y side takes precedence at corners; OUTFLOW ghosts copy the
// nearest interior cell; INLET ghosts are the lattice equilibrium at the
// prescribed velocity and the density of the first interior cell; DIRICHLET
// ghosts are constant.
#pragma once

#include "../../include/slbm.h"
#include "slbm_eq.cuh"

namespace slbm {

constexpr int kBandMax = 3;  // largest stencil reach (order 5)

template <int N, class S, class R>
__device__ __forceinline__ void load_t(const S* f, long long plane, int base, R (*s)[kMaxN]) {
#pragma unroll
  for (int iy = 0; iy < N; ++iy)
#pragma unroll
    for (int ix = 0; ix < N; ++ix) s[iy][ix] = static_cast<R>(f[(size_t)(ix + N * iy) * plane + base]);
}

template <int N, class S, class R>
__device__ __forceinline__ void store_t(S* f, long long plane, int base, const R (*s)[kMaxN]) {
#pragma unroll
  for (int iy = 0; iy < N; ++iy)
#pragma unroll
    for (int ix = 0; ix < N; ++ix) f[(size_t)(ix + N * iy) * plane + base] = static_cast<S>(s[iy][ix]);
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
  store_t<NL, S, R>(f0, p.plane, base, e);
  eq_dev<R>(p.lat[1], NH, dr, ux, uy, e);
  store_t<NH, S, R>(f1, p.plane, base, e);
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
