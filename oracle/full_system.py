"""The paper's global HPS system (Sec. 3.1, eq. (2x2), Fig. 4) for tiny grids.

Unknowns are all nodes of every leaf (n = n_i + n_b per leaf, N = N_l n).
Block row of leaf alpha:

* interior rows: A_c^alpha(I_i, :) u^alpha = s^alpha;
* face k of alpha with a neighbour beta across it:
      F^alpha(I_k, :) u^alpha + G^beta(I_opp(k), :) u^beta = 0
  (the interface condition f^alpha = -g^beta of eq. (inter); the coupling
  blocks G^tau_{+-x,+-y,+-z} of eq. (outgoingimpedance));
* face k on the boundary of (0,1)^3:  F^alpha(I_k, :) u^alpha = t.

This module is the cross-check that the face system solved elsewhere is the
same discrete problem: the incoming data F u_b of the solution here, moved to
Gauss points, equals the face-system solution.  Boundary data t is supplied at
the Chebyshev face nodes (P^{-1} applied to Gauss-point data keeps both
systems identical).
"""

import numpy as np

from .discretization import (
    leaf_matrix, leaf_incoming_op, leaf_outgoing_op, face_interp,
)

__all__ = ["full_system_matrix", "full_system_solve"]


def full_system_matrix(grid, eta, cdiag_all):
    """Dense N x N global matrix of Sec. 3.1 (tiny grids only)."""
    L = grid.layout
    n, ni = L.n, L.ni
    q2 = grid.q * grid.q
    N = grid.nleaves * n
    A = np.zeros((N, N), dtype=np.complex128)
    G = leaf_outgoing_op(grid.p, grid.h, eta)
    for leaf in range(grid.nleaves):
        Aleaf = leaf_matrix(grid.p, grid.h, eta, cdiag_all[leaf])
        A[leaf * n:(leaf + 1) * n, leaf * n:(leaf + 1) * n] = Aleaf
        for face in range(6):
            nbr = grid.neighbor(leaf, face)
            if nbr < 0:
                continue
            rows = slice(leaf * n + ni + face * q2, leaf * n + ni + (face + 1) * q2)
            src = (face ^ 1) * q2
            A[rows, nbr * n:(nbr + 1) * n] = G[src:src + q2, :]
    return A


def full_system_solve(grid, eta, cdiag_all, s_int, t_face_gauss):
    """Solve the global system; return (u, f) with f the Gauss-basis incoming data.

    s_int: (N_l, n_i) body load at interior nodes (or None);
    t_face_gauss: (N_l, 6, q^2) boundary data at Gauss points (or None), moved
    to Chebyshev face nodes by P^{-1}.
    """
    L = grid.layout
    n, ni = L.n, L.ni
    q2 = grid.q * grid.q
    Pf = face_interp(grid.p)
    A = full_system_matrix(grid, eta, cdiag_all)
    rhs = np.zeros(grid.nleaves * n, dtype=np.complex128)
    for leaf in range(grid.nleaves):
        if s_int is not None:
            rhs[leaf * n:leaf * n + ni] = s_int[leaf]
        for face in range(6):
            if grid.neighbor(leaf, face) < 0 and t_face_gauss is not None:
                r0 = leaf * n + ni + face * q2
                rhs[r0:r0 + q2] = np.linalg.solve(Pf, t_face_gauss[leaf, face])
    u = np.linalg.solve(A, rhs)
    F = leaf_incoming_op(grid.p, grid.h, eta)
    f = np.zeros((grid.nleaves, 6, q2), dtype=np.complex128)
    for leaf in range(grid.nleaves):
        fc = F @ u[leaf * n:(leaf + 1) * n]
        for face in range(6):
            f[leaf, face] = Pf @ fc[face * q2:(face + 1) * q2]
    return u.reshape(grid.nleaves, n), f.reshape(-1)
