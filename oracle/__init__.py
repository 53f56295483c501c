"""CPU FP64 oracle for the Fourier-Galerkin homogenization hot path.

TEST INFRASTRUCTURE ONLY. The oracle is a plain, slow, NumPy FP64 restatement of the method of
Mishra, Vondrejc & Zeman (arXiv:1508.02045): the DFT of eq. (DFT) written as dense matrices,
the projection of eqs. (proj)/(discrete_proj), the GaNi and Ga linear systems of eq. (linsys),
the double-grid coefficients of eq. (Ga_exact_integration), the prolongation and energies of
eq. (ev_bounds), and Algorithms 1-4. It shares no code with the CUDA library, and the product
path never imports it: only tests/, the smoke check and the benchmark's CPU-baseline leg do.

The linear-elasticity form (symmetric strain fields, the compatibility projection onto
symmetric gradients, stiffness tensors in Mandel notation) is in oracle/elastic.py.

Parity status: every function here is pinned by a test in tests/test_oracle_*.py against
something other than itself (library FFT, closed forms, dense Galerkin solves in a real
trigonometric basis, the values printed in Section 4).
"""
from .hom import *  # noqa: F401,F403
from .hom import __all__ as _hom_all
from . import elastic  # noqa: F401  (linear elasticity: oracle/elastic.py)

__all__ = list(_hom_all) + ["elastic"]
