"""Per-cell lattice loss: what the low-order lattice loses in one step.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle``): a composition of the
oracle's own step, lift and projection (Sec. III.B-D), in FP64; it shares
nothing with the CUDA path.

From a state in which every cell is high-order (f_Q at time t), two steps are
taken from the same start:
  a = one step of the all-high-order state            -> f_Q(t + 1)
  b = one step of the projected state project(f_Q(t)), all low-order,
      lifted back                                     -> lift(f_q(t + 1))
and the loss of cell x is the Euclidean norm over the high-order lattice's
populations, relative to the density,
  loss(x) = || a(x) - b(x) ||_2 / rho_a(x).
It holds both effects the low-order lattice misses: the moments of order 3
and 4 per axis of the non-equilibrium, which the projection drops (Knudsen
layers, Sec. IV.C), and the aliased fluxes of its equilibrium at high Mach
number (its third moment per axis equals three times the first, Sec. IV.A).
The oracle's state ends at a, as after one high-order step.
"""
from __future__ import annotations

import numpy as np


def lattice_loss(o) -> np.ndarray:
    """(ny, nx) loss of every cell of the oracle `o` (all flags 1 on entry)."""
    fl = o.get_flags()
    if not (fl == 1).all():
        raise ValueError("the lattice loss starts from an all-high-order state")
    fq_t = o.get_pops(1).copy()
    o.step(1)
    a = o.get_pops(1).copy()
    o.set_pops(1, fq_t)
    o.set_flags(np.zeros_like(fl))       # projection of every cell
    o.step(1)
    o.set_flags(np.ones_like(fl))        # lifting of every cell
    b = o.get_pops(1)
    o.set_pops(1, a)
    rho = a.sum(axis=2)
    return np.sqrt(((a - b) ** 2).sum(axis=2)) / rho
