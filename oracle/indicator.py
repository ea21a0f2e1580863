"""Reference features and forward pass of the learned refinement indicator.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle``): plain FP64 numpy from
the oracle's state, one cell at a time, restating the definitions; it shares
nothing with the CUDA path.

Features of a cell, from its own lattice (the lattice-frame model of Sec. II):
rho - 1, u, T - 1 with the kinetic T = (sum |c|^2 f / rho - |u|^2) / 2, the
non-equilibrium stress sum c_a c_b (f - f^L) (xx, xy, yy) with f^L the lattice
equilibrium of eq. (feqL0) at the cell's rho, u, the non-equilibrium energy
flux 1/2 sum c_a |c|^2 (f - f^L), central differences of rho, u_x, u_y along x
and y (periodic wrap, else the edge cell repeated), and |u|; each times the
fixed scale below.
"""
from __future__ import annotations

import numpy as np

from . import eq_lattice, lattice

SCALE = np.array([10, 3, 3, 10, 100, 100, 100, 100, 100, 100, 100, 100, 100, 100, 100, 3],
                 dtype=np.float64)


def features(o) -> np.ndarray:
    """(ny, nx, 16) features of the oracle state `o`."""
    ny, nx = o.ny, o.nx
    fl = o.get_flags()
    pops = [o.get_pops(0), o.get_pops(1)]
    lat = [lattice(o.n[0]), lattice(o.n[1])]
    rho, ux, uy, _ = o.moments()
    px, py = o.periodic if hasattr(o, "periodic") else (True, True)
    out = np.zeros((ny, nx, 16))
    for y in range(ny):
        for x in range(nx):
            k = int(fl[y, x])
            cx, cy, _W = lat[k]
            f = pops[k][y, x]
            r = f.sum()
            u, v = (cx * f).sum() / r, (cy * f).sum() / r
            T = ((cx * cx + cy * cy) * f).sum() / r / 2 - (u * u + v * v) / 2
            ne = f - eq_lattice(o.n[k], r, u, v)
            c2 = cx * cx + cy * cy

            def nb(a, dx, dy):
                xx, yy = x + dx, y + dy
                xx = xx % nx if px else min(max(xx, 0), nx - 1)
                yy = yy % ny if py else min(max(yy, 0), ny - 1)
                return a[yy, xx]

            out[y, x] = [r - 1, u, v, T - 1,
                         (cx * cx * ne).sum(), (cx * cy * ne).sum(), (cy * cy * ne).sum(),
                         0.5 * (cx * c2 * ne).sum(), 0.5 * (cy * c2 * ne).sum(),
                         0.5 * (nb(rho, 1, 0) - nb(rho, -1, 0)), 0.5 * (nb(rho, 0, 1) - nb(rho, 0, -1)),
                         0.5 * (nb(ux, 1, 0) - nb(ux, -1, 0)), 0.5 * (nb(ux, 0, 1) - nb(ux, 0, -1)),
                         0.5 * (nb(uy, 1, 0) - nb(uy, -1, 0)), 0.5 * (nb(uy, 0, 1) - nb(uy, 0, -1)),
                         np.hypot(u, v)]
    return out * SCALE


def forward_fp16(w: dict, x: np.ndarray) -> np.ndarray:
    """Logits with the precision the indicator's inference uses: inputs,
    W1, W2 and the first hidden layer rounded to FP16, everything else
    accumulated exactly (FP64 here)."""
    h16 = lambda a: np.asarray(a, dtype=np.float16).astype(np.float64)
    x16 = h16(x)
    h1 = np.maximum(x16 @ h16(w["w1"]) + np.asarray(w["b1"], np.float32), 0.0)
    h2 = np.maximum(h16(h1) @ h16(w["w2"]) + np.asarray(w["b2"], np.float32), 0.0)
    return h2 @ np.asarray(w["w3"], np.float32) + np.float32(w["b3"])
