"""Shared set-up for the GPU parity tests: the same seeded workload evaluated at
the oracle's nodes and at the nodes the CUDA library reports."""

import numpy as np

import oracle as O


class OracleCase:
    """Oracle maps, preconditioner and inputs of a workload (CPU, FP64)."""

    def __init__(self, w, with_precond=True, leaves=None):
        # with_precond builds the oracle's cluster preconditioner (dense per-cluster solves)
        self.w = w
        self.grid = O.Grid(w.nx, w.ny, w.nz, w.p)
        g = self.grid
        self.xi = O.interior_nodes(g)
        self.xf = O.face_nodes(g)
        self.nrm = np.broadcast_to(O.face_normals()[None, :, None, :], self.xf.shape)
        self.b = w.sample_b(self.xi)
        self.s = w.sample_s(self.xi)
        self.t = w.sample_t(self.xf, self.nrm)
        self.prob = O.build_problem(g, w.kappa, w.eta, self.b, leaves=leaves)
        self._cache = {}
        self.hom = None
        self.M = None
        if with_precond and leaves is None:
            self.hom = O.build_problem(g, w.kappa, w.eta, self.b, homogenized=True)
            self.M = O.Preconditioner(g, self.hom.R)

    def rhs(self, r=0):
        s = None if self.s is None else self.s[r]
        t = None if self.t is None else self.t[r]
        return O.rhs_face(self.grid, self.prob.H, s, t)

    def apply(self, f):
        return O.apply_face(self.grid, self.prob.R, f)

    def solve(self, r=0):
        """Oracle solution to round-off: dense LU on small grids, else GMRES to 1e-13
        (unpreconditioned: the preconditioner never changes the solution)."""
        key = ("solve", r)
        if key in self._cache:
            return self._cache[key]
        rhs = self.rhs(r)
        g = self.grid
        if g.nf <= 4000:
            f = np.linalg.solve(O.dense_face_matrix(g, self.prob.R), rhs)
        else:
            f, its, hist = O.gmres(self.apply, rhs, tol=1e-13, restart=50)
        self._cache[key] = f
        return f


def gpu_inputs(w, hps):
    """b, s, t of workload w at the GPU library's own nodes (numpy, flattened per RHS)."""
    xi, xf = hps.nodes(w.nx, w.ny, w.nz, w.p)
    nrm = np.broadcast_to(hps.face_normals()[None, :, None, :], xf.shape)
    b = w.sample_b(xi).reshape(-1)
    s = None if w.s is None else w.sample_s(xi).reshape(w.nrhs, -1)
    t = None if w.t is None else w.sample_t(xf, nrm).reshape(w.nrhs, -1)
    return xi, xf, b, s, t


def rel(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
