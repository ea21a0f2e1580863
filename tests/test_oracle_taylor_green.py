"""End-to-end accuracy pin of the oracle's multi-scale step: Taylor-Green
decay (App. A).

The paper reports that the hybrid scheme -- a disc of the high-order lattice
inside the standard one -- keeps the second-order convergence of the
single-lattice scheme on the decaying Taylor-Green vortex.  Here a D2Q25 disc
of radius N/4 sits in a D2Q9 field, cubic Lagrange streaming, on N = 12, 24,
48 periodic grids in diffusive scaling (tau fixed, so the lattice viscosity
nu = (tau - 1/2) dt is fixed; U0 proportional to 1/N; the run lasts until
2 nu k^2 t = 1/2, i.e. N^2-proportional steps).  The measured quantity is the
amplitude of the Taylor-Green mode (the velocity projected onto the initial
field's shape) against the analytic decay exp(-2 nu k^2 t).  The equilibrium
start also excites standing sound waves of twice the wavenumber, orthogonal
to the mode; they are excluded by the projection.

The observed order log2(e(N) / e(2N)) must be 2 +- 0.3 at both refinements.
An interpolation of lower order breaks it (linear Lagrange leaves a
resolution-independent error of ~0.66 here), as does a wrong relaxation rate
(the decay rate would not converge to 2 nu k^2).
"""
import numpy as np

import oracle as O
from paper_2102_12559_gb300 import workloads as WL


def _mode_error(N, tau):
    dt = O.Oracle(8, 8, 3, 5, tau=0.6).dt
    nu = (tau - 0.5) * dt
    k = 2 * np.pi / N
    steps = int(round(0.25 / (nu * k * k * dt)))
    rho, ux, uy = WL.taylor_green(N, U0=0.64 / N)
    o = O.Oracle(N, N, 3, 5, tau=tau, order=3)
    o.init_equilibrium(rho, ux, uy)
    x = np.arange(N)
    X, Y = np.meshgrid(x, x)
    disc = (((X - N / 2 + 0.5) ** 2 + (Y - N / 2 + 0.5) ** 2) < (N / 4) ** 2).astype(np.uint8)
    o.set_flags(disc)
    o.step(steps)
    _, u, v, _ = o.moments()
    amp = np.sum(u * ux + v * uy) / np.sum(ux * ux + uy * uy)
    return abs(amp / np.exp(-2 * nu * k * k * steps * dt) - 1.0)


def test_hybrid_taylor_green_second_order():
    errs = [_mode_error(N, 0.8) for N in (12, 24, 48)]
    orders = [np.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert all(1.7 <= p <= 2.3 for p in orders), (errs, orders)
    assert errs[-1] < 1e-2, errs
