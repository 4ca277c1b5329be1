"""Leaf discretization of the HPS method (oracle; test infrastructure only).

Follows Sec. 2.1 of arXiv:2112.02211 ("Leaf discretization"):

* the n_c x n_c x n_c Chebyshev tensor grid on a leaf box with its corner
  and edge nodes removed, interior nodes first, then the six faces in the
  order -x, +x, -y, +y, -z, +z (Fig. 2, index vector I = [I_i, I_1..I_6]);
* the collocation operator A_c = -D_x^2 - D_y^2 - D_z^2 - C with
  C = diag(kappa^2 (1 - b(x_k))) (interior rows of eq. (leaf));
* the outward normal derivative N (eq. (flux)) and the incoming impedance
  operator F = N + i eta I(I_b, :) (boundary rows of eq. (leaf));
* the outgoing impedance operator G = N - i eta I(I_b, :) (eq. (G)).

From the leaf system A [u_i; u_b] = [s; f] the leaf ItI map follows:
g = G u = F u - 2 i eta u_b = f - 2 i eta u_b, so
    R_C = I - 2 i eta (A^{-1})_{bb},   h_C = -2 i eta (A^{-1} [s; 0])_b.
Face data is then moved from the (n_c-2)^2 Chebyshev face nodes to q x q
Gauss-Legendre points (q = n_c - 2) with the invertible interpolation P:
R = P R_C P^{-1}, h = P h_C.

Notation: p = n_c, n1 = p - 2, n_i = n1^3, n_b = 6 n1^2, n = n_i + n_b.
"""

import functools

import numpy as np

__all__ = [
    "FACE_AXIS", "FACE_SIGN", "IN_FACE_AXES",
    "chebyshev_lobatto", "chebyshev_diff", "gauss_legendre", "lagrange_matrix",
    "LeafLayout", "Grid", "leaf_matrix", "leaf_maps", "face_interp",
    "leaf_iti", "interior_nodes", "face_nodes", "cheb_face_nodes", "face_normals",
    "homogenized_lambda", "binned_lambdas", "leaf_incoming_op", "leaf_outgoing_op",
]

# Face k in 0..5 is -x, +x, -y, +y, -z, +z (Sec. 2.1, "I_1 the left ...").
FACE_AXIS = (0, 0, 1, 1, 2, 2)
FACE_SIGN = (-1, 1, -1, 1, -1, 1)
# In-face coordinates (first one fastest): +-x faces -> (y, z),
# +-y faces -> (x, z), +-z faces -> (x, y).
IN_FACE_AXES = ((1, 2), (1, 2), (0, 2), (0, 2), (0, 1), (0, 1))


def chebyshev_lobatto(p):
    """Ascending Chebyshev extreme points cos(j pi/(p-1)) on [-1, 1].

    The classic Chebyshev grid of Sec. 2.1 (the paper cites Trefethen 2000
    and Boyd 2001 for it), listed from -1 to 1.
    """
    j = np.arange(p, dtype=np.float64)
    return -np.cos(np.pi * j / (p - 1))


def chebyshev_diff(p):
    """p x p Chebyshev differentiation matrix on [-1, 1] (Sec. 2.1).

    Off-diagonal entries (c_i/c_j)(-1)^{i+j}/(x_i - x_j) with c_0 = c_{p-1}
    = 2 and c_j = 1 otherwise; each diagonal entry makes its row sum zero
    (the derivative of a constant vanishes).
    """
    x = chebyshev_lobatto(p)
    c = np.ones(p)
    c[0] = c[-1] = 2.0
    D = np.zeros((p, p))
    for i in range(p):
        for j in range(p):
            if i != j:
                D[i, j] = (c[i] / c[j]) * (-1.0) ** (i + j) / (x[i] - x[j])
    for i in range(p):
        D[i, i] = -np.sum(D[i, :])
    return D


def gauss_legendre(q):
    """q Gauss-Legendre nodes (ascending) and weights on [-1, 1]."""
    x, w = np.polynomial.legendre.leggauss(q)
    return x, w


def lagrange_matrix(xsrc, xdst):
    """Matrix of the polynomial interpolant through xsrc evaluated at xdst.

    Entry [a, j] is the j-th Lagrange basis polynomial of the nodes xsrc,
    evaluated at xdst[a].
    """
    xsrc = np.asarray(xsrc, dtype=np.float64)
    xdst = np.asarray(xdst, dtype=np.float64)
    M = np.ones((len(xdst), len(xsrc)))
    for j in range(len(xsrc)):
        for m in range(len(xsrc)):
            if m != j:
                M[:, j] *= (xdst - xsrc[m]) / (xsrc[j] - xsrc[m])
    return M


class LeafLayout:
    """Local node numbering of one leaf (Sec. 2.1 and Fig. 2).

    Grid index triples (i, j, k) run over 0..p-1; interior nodes have all
    three in 1..p-2, face nodes have exactly one coordinate at 0 or p-1.
    Interior nodes come first with x fastest (column-major, the "reshape by
    columns" of Algorithms 1 and 3); face k follows with its n1 x n1 nodes,
    first in-face coordinate fastest.
    """

    def __init__(self, p):
        self.p = p
        self.n1 = p - 2
        self.ni = self.n1 ** 3
        self.nb = 6 * self.n1 ** 2
        self.n = self.ni + self.nb

    def index(self, i, j, k):
        n1, last = self.n1, self.p - 1
        ijk = (i, j, k)
        on = [a for a in range(3) if ijk[a] in (0, last)]
        if not on:
            return (i - 1) + n1 * (j - 1) + n1 * n1 * (k - 1)
        if len(on) != 1:
            raise ValueError("edge or corner node is not part of the leaf grid")
        axis = on[0]
        face = 2 * axis + (0 if ijk[axis] == 0 else 1)
        a0, a1 = IN_FACE_AXES[face]
        return self.ni + face * n1 * n1 + (ijk[a0] - 1) + n1 * (ijk[a1] - 1)


class Grid:
    """Uniform partition of (0,1)^3 into nx x ny x nz leaf boxes (Sec. 2).

    Leaves are numbered lexicographically, x fastest, then y, then z
    (Fig. 4(a)).  Each leaf carries the modified Chebyshev grid of order p
    and q = p - 2 Gauss points per face edge.
    """

    def __init__(self, nx, ny, nz, p):
        self.nx, self.ny, self.nz, self.p = nx, ny, nz, p
        self.q = p - 2
        self.layout = LeafLayout(p)
        self.h = (1.0 / nx, 1.0 / ny, 1.0 / nz)
        self.nleaves = nx * ny * nz
        self.nb = 6 * self.q * self.q
        self.nf = self.nleaves * self.nb

    def coords(self, leaf):
        ix = leaf % self.nx
        iy = (leaf // self.nx) % self.ny
        iz = leaf // (self.nx * self.ny)
        return ix, iy, iz

    def leaf_id(self, ix, iy, iz):
        return ix + self.nx * (iy + self.ny * iz)

    def neighbor(self, leaf, face):
        """Leaf across face `face` of `leaf`, or -1 when the face is on the boundary."""
        c = list(self.coords(leaf))
        axis = FACE_AXIS[face]
        c[axis] += FACE_SIGN[face]
        dims = (self.nx, self.ny, self.nz)
        if c[axis] < 0 or c[axis] >= dims[axis]:
            return -1
        return self.leaf_id(*c)

    def corner(self, leaf):
        ix, iy, iz = self.coords(leaf)
        return np.array([ix * self.h[0], iy * self.h[1], iz * self.h[2]])

    def paper_unknowns(self):
        """N = N_l * n, the size of the paper's global system (Sec. 3.1)."""
        return self.nleaves * self.layout.n


def _leaf_node_coords(p, h, corner):
    """Physical coordinates of the nodes of one leaf in the local order."""
    L = LeafLayout(p)
    t = chebyshev_lobatto(p)
    xyz = np.zeros((L.n, 3))
    for k in range(p):
        for j in range(p):
            for i in range(p):
                ijk = (i, j, k)
                nb_edges = sum(1 for a in ijk if a in (0, p - 1))
                if nb_edges > 1:
                    continue
                r = L.index(i, j, k)
                for a in range(3):
                    xyz[r, a] = corner[a] + 0.5 * h[a] * (t[ijk[a]] + 1.0)
    return xyz


def interior_nodes(grid):
    """Coordinates of all leaf-interior Chebyshev nodes, shape (N_l, n1^3, 3)."""
    out = np.zeros((grid.nleaves, grid.layout.ni, 3))
    for leaf in range(grid.nleaves):
        out[leaf] = _leaf_node_coords(grid.p, grid.h, grid.corner(leaf))[: grid.layout.ni]
    return out


def face_nodes(grid):
    """Coordinates of the q x q Gauss points of every leaf face, shape (N_l, 6, q^2, 3)."""
    q = grid.q
    xg, _ = gauss_legendre(q)
    out = np.zeros((grid.nleaves, 6, q * q, 3))
    for leaf in range(grid.nleaves):
        c = grid.corner(leaf)
        for face in range(6):
            axis = FACE_AXIS[face]
            a0, a1 = IN_FACE_AXES[face]
            for j2 in range(q):
                for j1 in range(q):
                    pt = np.zeros(3)
                    pt[axis] = c[axis] + (0.0 if FACE_SIGN[face] < 0 else grid.h[axis])
                    pt[a0] = c[a0] + 0.5 * grid.h[a0] * (xg[j1] + 1.0)
                    pt[a1] = c[a1] + 0.5 * grid.h[a1] * (xg[j2] + 1.0)
                    out[leaf, face, j1 + q * j2] = pt
    return out


def cheb_face_nodes(grid):
    """Coordinates of the n1 x n1 Chebyshev nodes of every leaf face (the face
    part of the leaf grid, Sec. 2.1 and Fig. 2), shape (N_l, 6, n1^2, 3), in the
    order of LeafLayout's face nodes."""
    n1 = grid.p - 2
    x = chebyshev_lobatto(grid.p)
    out = np.zeros((grid.nleaves, 6, n1 * n1, 3))
    for leaf in range(grid.nleaves):
        c = grid.corner(leaf)
        for face in range(6):
            axis = FACE_AXIS[face]
            a0, a1 = IN_FACE_AXES[face]
            for j2 in range(n1):
                for j1 in range(n1):
                    pt = np.zeros(3)
                    pt[axis] = c[axis] + (0.0 if FACE_SIGN[face] < 0 else grid.h[axis])
                    pt[a0] = c[a0] + 0.5 * grid.h[a0] * (x[j1 + 1] + 1.0)
                    pt[a1] = c[a1] + 0.5 * grid.h[a1] * (x[j2 + 1] + 1.0)
                    out[leaf, face, j1 + n1 * j2] = pt
    return out


def face_normals():
    """Outward unit normal of each face k (6, 3)."""
    n = np.zeros((6, 3))
    for face in range(6):
        n[face, FACE_AXIS[face]] = FACE_SIGN[face]
    return n


def _diff_matrices(p, h):
    D1 = chebyshev_diff(p)
    return [D1 * (2.0 / h[a]) for a in range(3)]


def leaf_matrix(p, h, eta, cdiag):
    """Dense leaf matrix A^tau of eq. (leaf), size n x n.

    Interior rows: -(D_x^2 + D_y^2 + D_z^2) - C, with C = diag(cdiag)
    (cdiag holds kappa^2 (1 - b) at the interior nodes).  The second
    derivative along each axis is the square of the full 1D Chebyshev matrix;
    the line through an interior node ends on two face nodes.
    Face rows: F = N + i eta I(I_b, :), N the outward normal derivative of
    eq. (flux) (-D_x on face 1, +D_x on face 2, ...).
    """
    L = LeafLayout(p)
    A = _leaf_matrix_without_c(p, tuple(float(v) for v in h), complex(eta)).copy()
    idx = np.arange(L.ni)
    A[idx, idx] -= np.asarray(cdiag, dtype=np.complex128)
    return A


@functools.lru_cache(maxsize=16)
def _leaf_matrix_without_c(p, h, eta):
    """eq. (leaf) with C = 0; the same for every leaf of a uniform grid."""
    L = LeafLayout(p)
    D = _diff_matrices(p, h)
    D2 = [Da @ Da for Da in D]
    A = np.zeros((L.n, L.n), dtype=np.complex128)
    last = p - 1
    for k in range(1, last):
        for j in range(1, last):
            for i in range(1, last):
                r = L.index(i, j, k)
                for m in range(p):
                    A[r, L.index(m, j, k)] -= D2[0][i, m]
                    A[r, L.index(i, m, k)] -= D2[1][j, m]
                    A[r, L.index(i, j, m)] -= D2[2][k, m]
    A[L.ni:, :] = leaf_incoming_op(p, h, eta)
    A.setflags(write=False)
    return A


def _normal_derivative(p, h):
    """N of eq. (flux): n_b x n rows of the outward normal derivative."""
    L = LeafLayout(p)
    D = _diff_matrices(p, h)
    N = np.zeros((L.nb, L.n), dtype=np.complex128)
    last = p - 1
    for face in range(6):
        axis = FACE_AXIS[face]
        sgn = FACE_SIGN[face]
        e = 0 if sgn < 0 else last
        a0, a1 = IN_FACE_AXES[face]
        for b in range(1, last):
            for a in range(1, last):
                pt = [0, 0, 0]
                pt[axis] = e
                pt[a0] = a
                pt[a1] = b
                r = L.index(*pt) - L.ni
                for m in range(p):
                    qq = list(pt)
                    qq[axis] = m
                    N[r, L.index(*qq)] += sgn * D[axis][e, m]
    return N


def leaf_incoming_op(p, h, eta):
    """F = N + i eta I(I_b, :) (Sec. 2.1): incoming impedance data from nodal values."""
    L = LeafLayout(p)
    F = _normal_derivative(p, h)
    F[:, L.ni:] += 1j * eta * np.eye(L.nb)
    return F


def leaf_outgoing_op(p, h, eta):
    """G = N - i eta I(I_b, :) (eq. (G)): outgoing impedance data from nodal values."""
    L = LeafLayout(p)
    G = _normal_derivative(p, h)
    G[:, L.ni:] -= 1j * eta * np.eye(L.nb)
    return G


def leaf_maps(A, ni, eta):
    """Chebyshev-basis leaf maps from the leaf matrix.

    Returns (R_C, H_C) with R_C = I - 2 i eta (A^{-1})_{bb} (incoming to
    outgoing impedance data) and H_C = -2 i eta (A^{-1})_{bi} (body load to
    outgoing data), both following from g = F u - 2 i eta u_b.
    """
    n = A.shape[0]
    Ainv = np.linalg.solve(A, np.eye(n, dtype=np.complex128))
    nb = n - ni
    R_C = np.eye(nb, dtype=np.complex128) - 2j * eta * Ainv[ni:, ni:]
    H_C = -2j * eta * Ainv[ni:, :ni]
    return R_C, H_C


def face_interp(p):
    """P_face = Q kron Q: face values at Chebyshev face nodes -> Gauss points.

    Q (q x n1) interpolates from the n1 = p-2 interior Chebyshev nodes of an
    edge to the q = p-2 Gauss-Legendre points; it is square and invertible.
    In-face vectors use the first in-face coordinate fastest, so the 2D map
    is kron(Q, Q) acting on the C-order flattening F[j2, j1].
    """
    xc = chebyshev_lobatto(p)[1:-1]
    xg, _ = gauss_legendre(p - 2)
    Q = lagrange_matrix(xc, xg)
    return np.kron(Q, Q)


def leaf_iti(p, h, eta, cdiag):
    """Gauss-basis ItI map R and body-load map H of one leaf.

    R = P R_C P^{-1}, H = P H_C with P = blockdiag_6(Q kron Q).
    """
    L = LeafLayout(p)
    A = leaf_matrix(p, h, eta, cdiag)
    R_C, H_C = leaf_maps(A, L.ni, eta)
    Pf = face_interp(p)
    P = np.kron(np.eye(6), Pf)
    R = P @ np.linalg.solve(P.T, R_C.T).T
    H = P @ H_C
    return R, H


def homogenized_lambda(cdiag):
    """lambda^tau = (max diag C_ii + min diag C_ii)/2 (Sec. 4.1).

    For complex C the real and imaginary parts are taken separately.
    """
    c = np.asarray(cdiag)
    re = 0.5 * (c.real.max() + c.real.min())
    im = 0.5 * (c.imag.max() + c.imag.min())
    return re + 1j * im


def binned_lambdas(lams, delta):
    """Homogenized constants rounded so that leaves with nearly the same medium share one solver.

    Sec. 4.1 remarks that the local approximate solver can be reused for
    leaves whose medium is roughly the same.  Here "roughly the same" is a
    bin: with w = delta * max_tau |lambda^tau|, each lambda^tau is replaced by
    the nearest multiple of w, real and imaginary parts separately (ties to
    even).  delta = 0 keeps every lambda^tau as it is.  Leaves with equal
    binned values get bitwise equal homogenized maps.
    """
    lams = np.asarray(lams, dtype=np.complex128)
    if delta <= 0 or lams.size == 0:
        return lams.copy()
    w = float(delta) * float(np.abs(lams).max())
    if w == 0.0:
        return lams.copy()
    return w * np.rint(lams.real / w) + 1j * (w * np.rint(lams.imag / w))
