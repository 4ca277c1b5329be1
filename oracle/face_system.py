"""The face (impedance-data) form of the HPS system (oracle; test infrastructure only).

Eliminating each leaf's own nodes with its exact leaf solve turns the global
system of Sec. 3 into a system for the incoming impedance data f on every
leaf face (6 q^2 values per leaf, Gauss points):

* each leaf maps incoming to outgoing data, g^tau = R^tau f^tau + h^tau,
  with h^tau the response to the body load s (Sec. 2.1, eq. (leaf));
* across a shared face the interface condition f^alpha = -g^beta holds
  (eq. (inter)); on a face on the boundary of (0,1)^3, f = t.

With Pi the face swap (Pi g)[alpha, k] = g[nbr(alpha, k), opp(k)] (zero on
boundary faces), this reads

    (I + Pi R) f = tbar - Pi h,

tbar = t on boundary faces and 0 elsewhere.  Vectors are laid out
[leaf][face 0..5][j2][j1] (j1 fastest), leaves numbered x fastest.

The preconditioner follows Sec. 4 (block Jacobi with locally homogenized
leaf solves): leaves are grouped into 2x2x2 clusters (1-wide at the end of
an odd axis); on each cluster the exact face system with homogenized maps
R~ (C replaced by lambda^tau, Sec. 4.1) is solved, faces leaving the
cluster acting as given impedance data:  z_c = (I + Pi_c R~)^{-1} r_c.
"""

import numpy as np

from .discretization import (
    Grid, LeafLayout, binned_lambdas, homogenized_lambda, leaf_iti,
)

__all__ = [
    "Problem", "build_problem", "swap", "apply_face", "rhs_face", "recover_interior",
    "dense_face_matrix", "gmres", "clusters", "Preconditioner",
    "cdiag_from_b", "relative_error",
]


def cdiag_from_b(kappa, b_int):
    """C = kappa^2 (1 - b) at interior nodes (Sec. 2.1)."""
    return kappa * kappa * (1.0 - np.asarray(b_int, dtype=np.complex128))


class Problem:
    """Leaf maps of a whole grid: R (N_l, n_b, n_b) and H (N_l, n_b, n_i).

    With homogenized=True the maps are R~, H~ (C replaced by lambda^tau,
    Sec. 4.1), lambda^tau optionally binned over the whole grid
    (`binned_lambdas`, lambda_bin = delta).
    """

    def __init__(self, grid, kappa, eta, b_int, leaves=None, homogenized=False, lambda_bin=0.0):
        self.grid = grid
        self.kappa = kappa
        self.eta = eta
        self.b_int = np.asarray(b_int, dtype=np.complex128)
        L = grid.layout
        leaves = range(grid.nleaves) if leaves is None else leaves
        self.leaves = list(leaves)
        self.R = {}
        self.H = {}
        self.lam = None
        if homogenized:
            lams = [homogenized_lambda(cdiag_from_b(kappa, self.b_int[i])) for i in range(grid.nleaves)]
            self.lam = binned_lambdas(lams, lambda_bin)
        for leaf in self.leaves:
            if homogenized:
                c = np.full(L.ni, self.lam[leaf], dtype=np.complex128)
            else:
                c = cdiag_from_b(kappa, self.b_int[leaf])
            self.R[leaf], self.H[leaf] = leaf_iti(grid.p, grid.h, eta, c)

    def R_array(self):
        return np.stack([self.R[i] for i in range(self.grid.nleaves)])


def build_problem(grid, kappa, eta, b_int, leaves=None, homogenized=False, lambda_bin=0.0):
    return Problem(grid, kappa, eta, b_int, leaves, homogenized, lambda_bin)


def _faces(grid, v):
    return np.asarray(v).reshape(grid.nleaves, 6, grid.q * grid.q)


def swap(grid, g):
    """Pi: outgoing data of the neighbour across each face; 0 on the boundary (eq. (inter))."""
    g = _faces(grid, g)
    y = np.zeros_like(g)
    for leaf in range(grid.nleaves):
        for face in range(6):
            nbr = grid.neighbor(leaf, face)
            if nbr >= 0:
                y[leaf, face] = g[nbr, face ^ 1]
    return y.reshape(-1)


def apply_face(grid, R, f):
    """y = (I + Pi R) f for one right-hand side."""
    f = _faces(grid, f)
    g = np.zeros_like(f)
    for leaf in range(grid.nleaves):
        g[leaf] = (R[leaf] @ f[leaf].reshape(-1)).reshape(6, -1)
    return f.reshape(-1) + swap(grid, g)


def rhs_face(grid, H, s_int, t_face):
    """b = tbar - Pi h, h^tau = H^tau s^tau; tbar = t on boundary faces, else 0."""
    nb = grid.nb
    h = np.zeros((grid.nleaves, nb), dtype=np.complex128)
    if s_int is not None:
        s = np.asarray(s_int).reshape(grid.nleaves, -1)
        for leaf in range(grid.nleaves):
            h[leaf] = H[leaf] @ s[leaf]
    b = -swap(grid, h)
    if t_face is not None:
        t = _faces(grid, t_face)
        bb = _faces(grid, b).copy()
        for leaf in range(grid.nleaves):
            for face in range(6):
                if grid.neighbor(leaf, face) < 0:
                    bb[leaf, face] = t[leaf, face]
        b = bb.reshape(-1)
    return b


def recover_interior(grid, kappa, eta, b_int, s_int, f_face, with_faces=False):
    """Leaf solution at interior nodes from face data (eq. (leaf)):
    u^tau = A^{tau,-1} [s^tau; P^{-1} f^tau], f^tau moved from Gauss points to the
    Chebyshev face nodes by P^{-1}.  Returns (N_l, n_i), and with with_faces
    also the leaf solution at its Chebyshev face nodes (N_l, n_b)."""
    from .discretization import face_interp, leaf_matrix
    L = grid.layout
    Pf = face_interp(grid.p)
    q2 = grid.q * grid.q
    f = np.asarray(f_face).reshape(grid.nleaves, 6, q2)
    u = np.zeros((grid.nleaves, L.ni), dtype=np.complex128)
    ub = np.zeros((grid.nleaves, L.nb), dtype=np.complex128)
    b_int = np.asarray(b_int).reshape(grid.nleaves, -1)
    for leaf in range(grid.nleaves):
        A = leaf_matrix(grid.p, grid.h, eta, cdiag_from_b(kappa, b_int[leaf]))
        rhs = np.zeros(L.n, dtype=np.complex128)
        if s_int is not None:
            rhs[:L.ni] = np.asarray(s_int).reshape(grid.nleaves, -1)[leaf]
        for face in range(6):
            rhs[L.ni + face * q2:L.ni + (face + 1) * q2] = np.linalg.solve(Pf, f[leaf, face])
        sol = np.linalg.solve(A, rhs)
        u[leaf] = sol[:L.ni]
        ub[leaf] = sol[L.ni:]
    return (u, ub) if with_faces else u


def dense_face_matrix(grid, R):
    """I + Pi blockdiag(R) as a dense N_f x N_f matrix (tiny grids only)."""
    nb, nf = grid.nb, grid.nf
    q2 = grid.q * grid.q
    M = np.eye(nf, dtype=np.complex128)
    for leaf in range(grid.nleaves):
        for face in range(6):
            nbr = grid.neighbor(leaf, face)
            if nbr < 0:
                continue
            rows = slice(leaf * nb + face * q2, leaf * nb + (face + 1) * q2)
            src = (face ^ 1) * q2
            M[rows, nbr * nb:(nbr + 1) * nb] += R[nbr][src:src + q2, :]
    return M


def gmres(matvec, b, tol=1e-12, restart=50, maxit=10000, precond=None, x0=None):
    """Restarted GMRES with right preconditioning (Saad and Schultz 1986).

    Modified Gram-Schmidt Arnoldi, complex Givens rotations, least squares
    by back substitution.  Solves A M^{-1} u = b and returns x = M^{-1} u.
    Stops on the true relative residual ||b - A x|| / ||b|| <= tol, checked
    at every restart.  Returns (x, iterations, relative residual history).
    """
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    M = (lambda v: v) if precond is None else precond
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n, dtype=np.complex128), 0, [0.0]
    history = []
    its = 0
    while True:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        history.append(beta / bnorm)
        if beta / bnorm <= tol or its >= maxit:
            return x, its, history
        V = np.zeros((restart + 1, n), dtype=np.complex128)
        Hm = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(restart):
            w = matvec(M(V[j]))
            for i in range(j + 1):
                Hm[i, j] = np.vdot(V[i], w)
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            if Hm[j + 1, j] != 0.0:
                V[j + 1] = w / Hm[j + 1, j]
            for i in range(j):
                a, bb = Hm[i, j], Hm[i + 1, j]
                Hm[i, j] = cs[i] * a + sn[i] * bb
                Hm[i + 1, j] = -np.conj(sn[i]) * a + cs[i] * bb
            a, bb = Hm[j, j], Hm[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            if abs(a) == 0.0:
                cs[j], sn[j] = 0.0, 1.0
            else:
                cs[j] = abs(a) / den
                sn[j] = (a / abs(a)) * np.conj(bb) / den
            Hm[j, j] = cs[j] * a + sn[j] * bb
            Hm[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            its += 1
            if abs(g[j + 1]) / bnorm <= 0.5 * tol or its >= maxit:
                break
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - Hm[i, i + 1:k] @ y[i + 1:k]) / Hm[i, i]
        x = x + M(V[:k].T @ y)


def clusters(grid, size=2):
    """Partition of the leaves into blocks of `size` leaves per axis.

    Blocks start at multiples of `size`; at the end of an axis whose leaf
    count is not a multiple of `size` the last block is narrower.  Returns a
    list of leaf-id lists (leaves inside a block in lexicographic order).
    """
    out = []
    for cz in range(0, grid.nz, size):
        for cy in range(0, grid.ny, size):
            for cx in range(0, grid.nx, size):
                leaves = []
                for iz in range(cz, min(cz + size, grid.nz)):
                    for iy in range(cy, min(cy + size, grid.ny)):
                        for ix in range(cx, min(cx + size, grid.nx)):
                            leaves.append(grid.leaf_id(ix, iy, iz))
                out.append(leaves)
    return out


class Preconditioner:
    """Cluster block-Jacobi preconditioner with homogenized leaf maps (Sec. 4).

    For each cluster c the matrix J_c = I + Pi_c R~ acts on the 6 q^2 |c|
    face values of the cluster's leaves; Pi_c swaps only across faces shared
    by two leaves of the cluster.  The preconditioner is z_c = J_c^{-1} r_c,
    formed here by a dense solve per cluster.
    """

    def __init__(self, grid, Rt, size=2):
        self.grid = grid
        self.blocks = clusters(grid, size)
        nb = grid.nb
        q2 = grid.q * grid.q
        self.J = []
        for leaves in self.blocks:
            pos = {leaf: i for i, leaf in enumerate(leaves)}
            m = len(leaves) * nb
            J = np.eye(m, dtype=np.complex128)
            for leaf in leaves:
                for face in range(6):
                    nbr = grid.neighbor(leaf, face)
                    if nbr < 0 or nbr not in pos:
                        continue
                    r0 = pos[leaf] * nb + face * q2
                    src = (face ^ 1) * q2
                    J[r0:r0 + q2, pos[nbr] * nb:(pos[nbr] + 1) * nb] += Rt[nbr][src:src + q2, :]
            self.J.append(J)

    def __call__(self, r):
        grid = self.grid
        nb = grid.nb
        r = np.asarray(r).reshape(grid.nleaves, nb)
        z = np.zeros_like(r)
        for leaves, J in zip(self.blocks, self.J):
            rc = np.concatenate([r[leaf] for leaf in leaves])
            zc = np.linalg.solve(J, rc)
            for i, leaf in enumerate(leaves):
                z[leaf] = zc[i * nb:(i + 1) * nb]
        return z.reshape(-1)


def relative_error(a, b):
    """||a - b||_2 / ||b||_2 over all entries (complex l2)."""
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
