"""GB300-native multi-scale semi-Lagrangian lattice Boltzmann step
(Kallikounis, Dorschner & Karlin, arXiv:2102.12559).

The compute path is the C-ABI library ``libslbm.so`` (CUDA, sm_103a) built
from ``csrc/``; ``slbm`` is its thin ctypes binding.  Importing the package
does not load the library: ``from paper_2102_12559_gb300 import slbm`` does.
"""
