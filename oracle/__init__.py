"""CPU oracle for the iterative HPS Helmholtz solver (test infrastructure only).

This package is the slow, plain FP64-complex restatement of the discrete
method of arXiv:2112.02211 ("An iterative solver for the HPS discretization
applied to three dimensional Helmholtz problems").  It exists to check the
CUDA path: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  The product path never calls it and it
shares no code with the CUDA library (it computes its own nodes,
differentiation matrices, leaf maps and face coupling from the paper).

Modules
-------
discretization  Chebyshev/Gauss tables, the leaf collocation system (Sec. 2.1,
                eq. (leaf)), leaf ItI maps and the Gauss change of basis.
face_system     The face (impedance-data) system I + Pi R, its RHS, dense and
                iterative solves, and the cluster block-Jacobi preconditioner
                with locally homogenized leaf maps (Sec. 4).
full_system     The paper's global system of Sec. 3 (eq. (2x2), Fig. 4) for
                tiny grids: the cross-check that the face system is the same
                discrete problem.
kron            Lemma 1 and Algorithms 1 and 3 (Kronecker applies).
full_iterative  The paper's iterative path on the global system: matrix-free
                apply (Algorithms 1-2) and the per-leaf homogenized block-Jacobi
                preconditioner of eq. (block_pc) (Algorithms 3-4).

Parity pins live in ``tests/test_oracle_*.py``.
"""

from .discretization import *  # noqa: F401,F403
from .face_system import *  # noqa: F401,F403
from .full_system import *  # noqa: F401,F403
from .kron import *  # noqa: F401,F403
from .full_iterative import *  # noqa: F401,F403
