"""The paper's own iterative path on the global system (Sec. 3-4) for moderate grids
(oracle; test infrastructure only).

* full_apply: A u for the global system of Sec. 3.1 without forming A.  Per
  leaf the leaf matrix of eq. (leaf) (interior rows: the Kronecker form of
  eq. (leafmat) / Algorithm 1 with the line ends on the face nodes; face rows
  F = N + i eta I), plus, on every face with a neighbour beta, beta's outgoing
  rows G^beta = N - i eta I on the opposite face (Algorithm 2, eq. (inter)).
* full_rhs: [s at interior nodes; t at the Chebyshev face nodes of faces on the
  boundary of (0,1)^3; 0 on shared faces].
* FullBlockJacobi: the block-Jacobi preconditioner of Sec. 4 on the global
  system, one block per leaf: the homogenized leaf matrix A~ (C replaced by
  lambda^tau, Sec. 4.1), applied by the Schur route of eq. (block_pc):
      z_b = S~^{-1} (r_b - F_bi A~_ii^{-1} r_i),  z_i = A~_ii^{-1} (r_i - A_ib z_b),
  S~ = F_bb - F_bi A~_ii^{-1} A_ib, with A~_ii^{-1} applied by Algorithm 3
  (Algorithm 4).
* full_to_face: the incoming impedance data P F u_b at the Gauss points, the
  unknowns of the face system, from a global solution.

Vectors are [leaf][n] with the leaf's local order of LeafLayout (interior
nodes x fastest, then the six faces' n1 x n1 nodes).
"""

import numpy as np

from .discretization import face_interp, homogenized_lambda, leaf_incoming_op, leaf_matrix, leaf_outgoing_op
from .face_system import cdiag_from_b
from .kron import alg3_apply_Aii_homog_inv

__all__ = ["full_apply", "full_rhs", "FullBlockJacobi", "full_to_face", "full_lambdas"]


def full_apply(grid, eta, cdiag_all, u):
    """A u of the global system (eq. (2x2)), leaf by leaf."""
    L = grid.layout
    n, ni = L.n, L.ni
    q2 = grid.q * grid.q
    G = leaf_outgoing_op(grid.p, grid.h, eta)
    u = np.asarray(u, dtype=np.complex128).reshape(grid.nleaves, n)
    y = np.zeros_like(u)
    for leaf in range(grid.nleaves):
        y[leaf] = leaf_matrix(grid.p, grid.h, eta, cdiag_all[leaf]) @ u[leaf]
        for face in range(6):
            nbr = grid.neighbor(leaf, face)
            if nbr < 0:
                continue
            src = (face ^ 1) * q2
            y[leaf, ni + face * q2:ni + (face + 1) * q2] += G[src:src + q2, :] @ u[nbr]
    return y.reshape(-1)


def full_rhs(grid, s_int, t_face_gauss):
    """Right-hand side of the global system; t given at Gauss points is moved to the
    Chebyshev face nodes by P^{-1} (face by face)."""
    L = grid.layout
    n, ni = L.n, L.ni
    q2 = grid.q * grid.q
    Pf = face_interp(grid.p)
    rhs = np.zeros((grid.nleaves, n), dtype=np.complex128)
    for leaf in range(grid.nleaves):
        if s_int is not None:
            rhs[leaf, :ni] = np.asarray(s_int).reshape(grid.nleaves, -1)[leaf]
        if t_face_gauss is None:
            continue
        t = np.asarray(t_face_gauss).reshape(grid.nleaves, 6, q2)
        for face in range(6):
            if grid.neighbor(leaf, face) < 0:
                rhs[leaf, ni + face * q2:ni + (face + 1) * q2] = np.linalg.solve(Pf, t[leaf, face])
    return rhs.reshape(-1)


def full_to_face(grid, eta, u):
    """Incoming impedance data at the Gauss points, P F u_b, of every leaf face."""
    L = grid.layout
    q2 = grid.q * grid.q
    F = leaf_incoming_op(grid.p, grid.h, eta)
    Pf = face_interp(grid.p)
    u = np.asarray(u).reshape(grid.nleaves, L.n)
    f = np.zeros((grid.nleaves, 6, q2), dtype=np.complex128)
    for leaf in range(grid.nleaves):
        fc = F @ u[leaf]
        for face in range(6):
            f[leaf, face] = Pf @ fc[face * q2:(face + 1) * q2]
    return f.reshape(-1)


def full_lambdas(grid, kappa, b_int):
    """lambda^tau of every leaf (Sec. 4.1)."""
    b_int = np.asarray(b_int).reshape(grid.nleaves, -1)
    return np.array([homogenized_lambda(cdiag_from_b(kappa, b_int[i])) for i in range(grid.nleaves)])


class FullBlockJacobi:
    """Per-leaf homogenized block-Jacobi preconditioner of the global system (Sec. 4,
    eq. (block_pc), Algorithms 3 and 4).  Leaves with equal lambda share S~^{-1}."""

    def __init__(self, grid, eta, lams):
        self.grid = grid
        L = grid.layout
        self.ni, self.n = L.ni, L.n
        self.lams = np.asarray(lams, dtype=np.complex128)
        self.blocks = {}
        for lam in self.lams:
            key = complex(lam)
            if key in self.blocks:
                continue
            A = leaf_matrix(grid.p, grid.h, eta, np.full(L.ni, key, dtype=np.complex128))
            Aib, Fbi, Fbb = A[:L.ni, L.ni:], A[L.ni:, :L.ni], A[L.ni:, L.ni:]
            X = np.stack([alg3_apply_Aii_homog_inv(grid.p, grid.h, key, Aib[:, c]) for c in range(L.nb)], axis=1)
            S = Fbb - Fbi @ X
            self.blocks[key] = (Aib, Fbi, np.linalg.inv(S))

    def solve_leaf(self, leaf, r):
        lam = complex(self.lams[leaf])
        Aib, Fbi, Sinv = self.blocks[lam]
        ni = self.ni
        p, h = self.grid.p, self.grid.h
        y = alg3_apply_Aii_homog_inv(p, h, lam, r[:ni])
        zb = Sinv @ (r[ni:] - Fbi @ y)
        zi = alg3_apply_Aii_homog_inv(p, h, lam, r[:ni] - Aib @ zb)
        return np.concatenate([zi, zb])

    def __call__(self, r):
        r = np.asarray(r, dtype=np.complex128).reshape(self.grid.nleaves, self.n)
        return np.concatenate([self.solve_leaf(i, r[i]) for i in range(self.grid.nleaves)])
