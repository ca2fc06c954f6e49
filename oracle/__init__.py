"""FP64 CPU oracle for the stochastic multigrid SELM method (Atzberger, arXiv:1003.2680).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow reference that the
CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py`` may import it.  The
product package never imports it and shares no code with it.

Every function follows a passage of the paper (section, equation or
algorithm) and runs the method's steps in the paper's order, in float64.
Library primitives (sparse matrix products, Cholesky, triangular solves) serve
as single steps; nothing is blocked, fused or reordered beyond what the cited
definition states.

Modules
-------
philox      counter-based normal variates (Philox4x32-10 + Box-Muller)
grid        MAC lattices, 1-D factors, trilinear prolongation, Galerkin levels
gibbs       stochastic Gauss-Seidel (heat-bath) sweeps, Section 3.1
multigrid   V-cycle (Algorithm 3), FAC iteration (Algorithm 1), coarsest step
coupling    Peskin 4-point interpolation Gamma and spreading Gamma^T (Section 2.1)
projection  MAC divergence / gradient and the discrete projection (Section 4)
selm        mobility, thermal field, Euler-Maruyama step (Algorithm 4)
composite   composite (refined-patch) grid, Algorithms 1-2
decorrelation  lag correlations of the multigrid and Gauss-Seidel samplers (Section 5)
composite_mac  divergence, gradient and projection on the composite MAC grid (Section 4)

Parity status: every function is pinned by a ``-m "not gpu"`` test (closed
forms, exact invariance identities, dense direct references); none is
"parity unpinned".
"""

from . import philox, grid, gibbs, multigrid, coupling, projection, selm  # noqa: F401
from . import composite, composite_mac, decorrelation  # noqa: F401
