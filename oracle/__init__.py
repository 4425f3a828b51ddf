"""FP64 CPU oracle for the matrix-free DG acoustic wave solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA library never calls it, and it shares no code with the CUDA path.

It computes the same discrete scheme as the GPU path in the plainest way:
dense element matrices built by direct quadrature (every basis function
evaluated at every quadrature point, no sum factorisation), dense Cholesky
inversion of the mass matrices (no basis-change trick), face integrals with
both traces evaluated from all coefficients of each element (no face-node
shortcut), and a Taylor-Cauchy-Kowalevski predictor built from dense
collocation-derivative, projection and prolongation matrices.

Parity status per function is stated in each module's header.
"""
from .basis import (gauss_1d, gauss_lobatto_1d, lagrange_1d,  # noqa: F401
                    lagrange_deriv_1d, tensor_points)
from .dg import (Oracle, LSRK54_A, LSRK54_B, LSRK45_KCL_A, LSRK45_KCL_B,  # noqa: F401
                 LSRK59_KCL_A, LSRK59_KCL_B)
from .dg2d import Oracle2D  # noqa: F401
