"""Kronecker-product forms of the interior operator (oracle; test infrastructure only).

* Lemma 1 (Roth): (M kron N) vec(X) = vec(N X M^T), vec stacking columns.
* eq. (leafmat): A_ii = -I(x)I(x)L1 - I(x)L1(x)I - L1(x)I(x)I - C_ii, with L1
  the interior block of the squared 1D Chebyshev differentiation matrix.
* Algorithm 1: A_ii v by 1D products along each axis (here the minus sign on
  C_ii of eq. (leafmat) is used; Algorithm 1 prints +C v).
* Algorithm 3 / Sec. 4.1: the homogenized operator
  A~_ii = V~ (-E_Delta - lambda I) V~^{-1} with L1 = V E V^{-1}, applied to a
  vector by 1D mode products with V^{-1}, a diagonal scaling, and V (the
  text's (-E_Delta - lambda I)^{-1} is used).

Interior vectors are indexed (i, j, k) with i (x) fastest.  Leaves may have
different widths per axis, so each axis carries its own L1.
"""

import numpy as np

from .discretization import chebyshev_diff

__all__ = ["lemma1_apply", "interior_L1", "alg1_apply_Aii", "dense_Aii",
           "alg3_apply_Aii_homog_inv", "dense_Aii_homog"]


def lemma1_apply(M, N, x):
    """(M kron N) x evaluated as vec(N X M^T) with X = reshape(x) by columns."""
    m, n = M.shape[1], N.shape[1]
    X = np.reshape(x, (n, m), order="F")
    return np.reshape(N @ X @ M.T, -1, order="F")


def interior_L1(p, h):
    """L1 = (D~^2)[1:p-1, 1:p-1] for one axis of width h."""
    D = chebyshev_diff(p) * (2.0 / h)
    return (D @ D)[1:p - 1, 1:p - 1]


def _mode(T, M, axis):
    """Multiply the 3-tensor T (i, j, k) by M along `axis`."""
    return np.moveaxis(np.tensordot(M, T, axes=([1], [axis])), 0, axis)


def alg1_apply_Aii(p, h, cdiag, v):
    """A_ii v (eq. (leafmat)) by 1D second-derivative products along x, y, z."""
    n1 = p - 2
    V = np.reshape(np.asarray(v, dtype=np.complex128), (n1, n1, n1), order="F")
    W = np.zeros_like(V)
    for axis in range(3):
        W -= _mode(V, interior_L1(p, h[axis]), axis)
    w = np.reshape(W, -1, order="F")
    return w - np.asarray(cdiag) * np.asarray(v)


def dense_Aii(p, h, cdiag):
    """The interior block A_ii of eq. (leafmat) written out with np.kron."""
    n1 = p - 2
    I1 = np.eye(n1)
    Lx, Ly, Lz = (interior_L1(p, h[a]) for a in range(3))
    A = -(np.kron(I1, np.kron(I1, Lx)) + np.kron(I1, np.kron(Ly, I1)) + np.kron(Lz, np.kron(I1, I1)))
    return A.astype(np.complex128) - np.diag(np.asarray(cdiag, dtype=np.complex128))


def dense_Aii_homog(p, h, lam):
    """A~_ii = -(Kronecker sum of L1) - lambda I (Sec. 4.1)."""
    n1 = p - 2
    return dense_Aii(p, h, np.full(n1 ** 3, lam, dtype=np.complex128))


def alg3_apply_Aii_homog_inv(p, h, lam, v):
    """A~_ii^{-1} v via L1 = V E V^{-1} along each axis (Algorithm 3)."""
    n1 = p - 2
    Vs, Vinv, E = [], [], []
    for axis in range(3):
        ev, V = np.linalg.eig(interior_L1(p, h[axis]))
        Vs.append(V)
        Vinv.append(np.linalg.inv(V))
        E.append(ev)
    T = np.reshape(np.asarray(v, dtype=np.complex128), (n1, n1, n1), order="F")
    for axis in range(3):
        T = _mode(T, Vinv[axis], axis)
    ED = E[0][:, None, None] + E[1][None, :, None] + E[2][None, None, :]
    T = T / (-ED - lam)
    for axis in range(3):
        T = _mode(T, Vs[axis], axis)
    return np.reshape(T, -1, order="F")
