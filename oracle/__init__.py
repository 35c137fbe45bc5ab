"""Plain FP64 CPU oracle for the many-k H|psi>, Davidson and Sternheimer path.

TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check of ``__graft_entry__`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA path (no kernels, no tables, no index
maps) and uses no FFT library: every Fourier sum is written out as a direct sum.

Modules
  hamiltonian  -- kinetic, local (dense convolution and direct Fourier sums),
                  nonlocal projector terms; dense H(k); H|psi>  (paper Sec. 2.2, Sec. 4)
  davidson     -- the block Davidson iteration of Sec. 2.1 and the dense reference
  sternheimer  -- right-hand side, operator, dense solve and the PCG of Sec. 2.4 (Eq. linear_system)

Every function names the passage of the paper it follows.  Floating point is FP64.
"""
from . import hamiltonian, davidson, sternheimer  # noqa: F401
