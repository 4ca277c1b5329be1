"""GB300-native iterative HPS Helmholtz solver (arXiv:2112.02211), Python binding.

The compute path is the CUDA library ``libhps.so`` (C ABI in include/hps.h);
this module only marshals arguments: device buffers are torch tensors on the
GPU, streams are torch streams.  There is no CPU fallback: every call runs
the library's kernels and raises ``HPSError`` when the library or the GPU is
missing.

    import paper_2112_02211_gb300 as hps
    xi, xf = hps.nodes(16, 16, 16, p=10)             # interior / face points
    solver = hps.Solver(16, 16, 16, p=10, kappa=40.0, eta=40.0, b=b_at_xi)
    f, info = solver.solve(s=s_at_xi, tol=1e-6, form="mixed")
"""

import ctypes

import numpy as np

from . import _native as N
from ._native import HPSError

__all__ = ["Solver", "nodes", "face_normals", "plan_blocks", "HPSError", "load"]

load = N.load


def _torch():
    import torch
    return torch


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def nodes(nx, ny, nz, p, cheb_faces=False):
    """Interior Chebyshev nodes (nl, n1^3, 3) and face Gauss points (nl, 6, q^2, 3), from the device;
    with cheb_faces also the Chebyshev face nodes (nl, 6, n1^2, 3) of `Solver.recover(faces=True)`."""
    lib = N.load()
    q = p - 2
    nl = nx * ny * nz
    xi = np.zeros((nl, (p - 2) ** 3, 3))
    xf = np.zeros((nl, 6, q * q, 3))
    xc = np.zeros((nl, 6, q * q, 3)) if cheb_faces else None
    g = N.Grid(nx, ny, nz, p, q)
    N.check(lib.hps_nodes(ctypes.byref(g), xi.ctypes.data_as(ctypes.c_void_p), xf.ctypes.data_as(ctypes.c_void_p),
                          None if xc is None else xc.ctypes.data_as(ctypes.c_void_p)))
    return (xi, xf, xc) if cheb_faces else (xi, xf)


def plan_blocks(nx, ny, nz, p, lambda_q):
    """Shared preconditioner blocks for the binned constants `lambda_q` (complex, one per leaf),
    planned on the host as hps_setup does (no GPU): returns (B block of every leaf, K_c block of
    every 2x2x2 cluster), both numbered in order of first appearance."""
    lib = N.load()
    lam = np.ascontiguousarray(np.asarray(lambda_q, dtype=np.complex128).reshape(-1))
    nl = nx * ny * nz
    if lam.size != nl:
        raise ValueError(f"lambda_q has {lam.size} entries, expected {nl}")
    ncl = -(-nx // 2) * -(-ny // 2) * -(-nz // 2)
    leaf_b = np.zeros(nl, dtype=np.int32)
    cl_k = np.zeros(ncl, dtype=np.int32)
    g = N.Grid(nx, ny, nz, p, p - 2)
    c = ctypes.c_int()
    N.check(lib.hps_plan_blocks(ctypes.byref(g), lam.ctypes.data_as(ctypes.c_void_p),
                                leaf_b.ctypes.data_as(ctypes.c_void_p), cl_k.ctypes.data_as(ctypes.c_void_p),
                                ctypes.byref(c), None, None))
    if c.value != ncl:
        raise HPSError(N.HPS_EINVAL, f"hps_plan_blocks returned {c.value} clusters, expected {ncl}")
    return leaf_b, cl_k


def face_normals():
    """Outward unit normal of face k = -x, +x, -y, +y, -z, +z."""
    n = np.zeros((6, 3))
    for k in range(6):
        n[k, k // 2] = -1.0 if k % 2 == 0 else 1.0
    return n


_FORMS = {"fp64": N.HPS_FORM_FP64, "mixed": N.HPS_FORM_MIXED}


class Solver:
    """One medium on one grid: leaf ItI maps, preconditioner and Krylov workspace on the GPU."""

    def __init__(self, nx, ny, nz, p, kappa, eta=None, b=None, forms=("fp64", "mixed"), restart=50,
                 cluster=2, maxit=5000, max_rhs=1, hbm_budget=0, device=0, precond_fp16=True, tc_apply=True,
                 lean=False, lambda_bin=0.0, full_system=False, autotune=True):
        self.lib = N.load()
        self.nx, self.ny, self.nz, self.p, self.q = nx, ny, nz, p, p - 2
        self.nl = nx * ny * nz
        self.ni = (p - 2) ** 3
        self.nb = 6 * self.q * self.q
        self.nf = self.nl * self.nb
        self.kappa = float(kappa)
        self.eta = float(kappa if eta is None else eta)
        self.max_rhs = max_rhs
        grid = N.Grid(nx, ny, nz, p, p - 2)
        opt = N.Options()
        self.lib.hps_default_options(ctypes.byref(opt))
        opt.forms = sum(_FORMS[f] for f in forms)
        opt.restart = restart
        opt.cluster = cluster
        opt.maxit = maxit
        opt.max_rhs = max_rhs
        opt.hbm_budget = hbm_budget
        opt.device = device
        opt.precond_fp16 = 1 if precond_fp16 else 0
        opt.tc_apply = 1 if tc_apply else 0
        opt.lean = 1 if lean else 0
        opt.lambda_bin = float(lambda_bin)
        opt.full_system = 1 if full_system else 0
        opt.autotune = 1 if autotune else 0
        self.n = self.ni + self.nb  # global-system unknowns per leaf
        bb = None
        if b is not None:
            bb = np.ascontiguousarray(np.asarray(b, dtype=np.complex128).reshape(-1))
            if bb.size != self.nl * self.ni:
                raise ValueError("b must hold one value per interior node")
        h = ctypes.c_void_p()
        N.check(self.lib.hps_setup(ctypes.byref(grid), self.kappa, self.eta,
                                   None if bb is None else bb.ctypes.data_as(ctypes.c_void_p),
                                   ctypes.byref(opt), ctypes.byref(h)))
        self.handle = h

    # -- operators on device tensors ---------------------------------------------------------
    def _nrhs(self, t):
        n = t.numel()
        if n % self.nf:
            raise ValueError("face vectors must hold a multiple of N_f values")
        return n // self.nf

    def apply(self, f, out=None, stream=None):
        """y = (I + Pi R) f; f complex128 (FP64 maps) or complex64 (FP32 maps) on the GPU."""
        torch = _torch()
        dt = N.HPS_C128 if f.dtype == torch.complex128 else N.HPS_C64
        y = torch.empty_like(f) if out is None else out
        N.check(self.lib.hps_apply(self.handle, dt, _ptr(f), _ptr(y), self._nrhs(f), _stream(stream)))
        return y

    def precond(self, r, out=None, stream=None, fp16_blocks=False):
        """z = J^{-1} r (cluster block Jacobi with homogenized leaf maps).  complex64 input
        reads the FP32 blocks, or their FP16 copies with fp16_blocks=True."""
        torch = _torch()
        dt = N.HPS_C128 if r.dtype == torch.complex128 else (N.HPS_C64_H16 if fp16_blocks else N.HPS_C64)
        z = torch.empty_like(r) if out is None else out
        N.check(self.lib.hps_precond(self.handle, dt, _ptr(r), _ptr(z), self._nrhs(r), _stream(stream)))
        return z

    def rhs(self, s=None, t=None, nrhs=1, stream=None):
        """b = tbar - Pi (H s) on the GPU (complex128 tensors)."""
        torch = _torch()
        out = torch.empty(nrhs * self.nf, dtype=torch.complex128, device="cuda")
        N.check(self.lib.hps_rhs(self.handle, _ptr(s), _ptr(t), nrhs, _ptr(out), _stream(stream)))
        return out

    def solve(self, s=None, t=None, tol=1e-10, form="fp64", nrhs=None, out=None, stream=None, precond=True,
              x0=None, graph=True, cgs2=False):
        """Solve (I + Pi R) f = tbar - Pi H s.  s, t, out: torch tensors (device or host) or numpy
        arrays (host).  x0: initial guess (copied into out first).  graph=False launches every
        Arnoldi step from the host; cgs2=True always orthogonalizes twice.  Returns (f, info dict)."""
        torch = _torch()

        def as_arg(a):
            if a is None:
                return None, None
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a.astype(np.complex128, copy=False))
                return a, a.ctypes.data_as(ctypes.c_void_p)
            return a, _ptr(a)

        if nrhs is None:
            if s is not None:
                nrhs = int(np.prod(s.shape)) // (self.nl * self.ni)
            elif t is not None:
                nrhs = int(np.prod(t.shape)) // self.nf
            else:
                nrhs = 1
        if out is None:
            out = torch.empty(nrhs * self.nf, dtype=torch.complex128, device="cuda")
        if x0 is not None:
            if isinstance(out, np.ndarray):
                out[...] = np.asarray(x0).reshape(out.shape)
            else:
                out.copy_(torch.as_tensor(np.asarray(x0) if isinstance(x0, np.ndarray) else x0).reshape(out.shape))
        s_keep, s_ptr = as_arg(s)
        t_keep, t_ptr = as_arg(t)
        o_keep, o_ptr = as_arg(out)
        info = N.SolveInfo()
        code = _FORMS[form] | (0 if precond else N.HPS_SOLVE_NO_PRECOND) | (N.HPS_SOLVE_X0 if x0 is not None else 0) \
            | (0 if graph else N.HPS_SOLVE_NO_GRAPH) | (N.HPS_SOLVE_CGS2 if cgs2 else 0)
        rc = self.lib.hps_gmres_solve(self.handle, code, s_ptr, t_ptr, nrhs, float(tol), o_ptr,
                                      ctypes.byref(info), _stream(stream))
        if rc not in (N.HPS_OK, N.HPS_ENOCONV):
            N.check(rc)
        if isinstance(out, np.ndarray) and o_keep is not out:
            out[...] = o_keep
        d = {"iterations": info.iterations, "cycles": info.cycles, "converged": bool(info.converged),
             "rel_residual": info.rel_residual, "seconds": info.seconds, "status": rc,
             "reorth_steps": info.reorth_steps}
        return out, d

    def recover(self, f, s=None, nrhs=None, stream=None, faces=False):
        """Leaf solutions at the interior nodes, u = A^{-1}[s; P^{-1} f] per leaf (device tensors);
        with faces=True also u at the Chebyshev face nodes (face layout)."""
        torch = _torch()
        nrhs = nrhs or self._nrhs(f)
        u = torch.empty(nrhs * self.nl * self.ni, dtype=torch.complex128, device="cuda")
        uf = torch.empty(nrhs * self.nf, dtype=torch.complex128, device="cuda") if faces else None
        N.check(self.lib.hps_recover(self.handle, _ptr(s), _ptr(f), nrhs, _ptr(u), _ptr(uf), _stream(stream)))
        return (u, uf) if faces else u

    # ---- the paper's iterative path on the global system (full_system=True) ----
    def full_apply(self, u, out=None, stream=None):
        """y = A u for the global system of Sec. 3.1 (device tensors, complex128 or complex64)."""
        torch = _torch()
        nrhs = u.numel() // (self.nl * self.n)
        y = torch.empty_like(u) if out is None else out
        dt = N.HPS_C128 if u.dtype == torch.complex128 else N.HPS_C64
        N.check(self.lib.hps_full_apply(self.handle, dt, _ptr(u), _ptr(y), nrhs, _stream(stream)))
        return y

    def full_precond(self, r, out=None, stream=None):
        """z = blockdiag(A~)^{-1} r, the per-leaf homogenized block-Jacobi of Sec. 4."""
        torch = _torch()
        nrhs = r.numel() // (self.nl * self.n)
        z = torch.empty_like(r) if out is None else out
        dt = N.HPS_C128 if r.dtype == torch.complex128 else N.HPS_C64
        N.check(self.lib.hps_full_precond(self.handle, dt, _ptr(r), _ptr(z), nrhs, _stream(stream)))
        return z

    def full_solve(self, s=None, t=None, tol=1e-10, form="fp64", nrhs=1, stream=None, precond=True, graph=True,
                   cgs2=False):
        """GMRES on the global system with the per-leaf block-Jacobi preconditioner; returns
        (u, info) with u at every node of every leaf (device complex128)."""
        torch = _torch()
        u = torch.empty(nrhs * self.nl * self.n, dtype=torch.complex128, device="cuda")
        info = N.SolveInfo()
        f = _FORMS[form] | (0 if precond else N.HPS_SOLVE_NO_PRECOND) | (0 if graph else N.HPS_SOLVE_NO_GRAPH) \
            | (N.HPS_SOLVE_CGS2 if cgs2 else 0)
        rc = self.lib.hps_full_solve(self.handle, f, _ptr(s), _ptr(t), nrhs, float(tol), _ptr(u), ctypes.byref(info),
                                     _stream(stream))
        if rc not in (0, N.HPS_ENOCONV):
            N.check(rc)
        return u, {"iterations": info.iterations, "cycles": info.cycles, "converged": bool(info.converged),
                   "rel_residual": info.rel_residual, "seconds": info.seconds, "status": rc,
                   "reorth_steps": info.reorth_steps}

    def precond_info(self):
        """(clusters, distinct K_c blocks, distinct B blocks) of the preconditioner."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        N.check(self.lib.hps_precond_info(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def export(self, what, index):
        """Copy one stored operator block to the host (numpy complex128)."""
        codes = {"R": N.HPS_EXPORT_R, "H": N.HPS_EXPORT_H, "lambda": N.HPS_EXPORT_LAMBDA,
                 "Kc": N.HPS_EXPORT_KC, "B": N.HPS_EXPORT_B}
        n = N.check(self.lib.hps_export(self.handle, codes[what], index, None))
        buf = np.zeros(n // 2, dtype=np.complex128)
        N.check(self.lib.hps_export(self.handle, codes[what], index, buf.ctypes.data_as(ctypes.c_void_p)))
        return buf

    def import_map(self, index, R):
        """Replace leaf `index`'s stored ItI map with R (6q^2 x 6q^2 complex, host)."""
        a = np.ascontiguousarray(np.asarray(R, dtype=np.complex128))
        if a.shape != (self.nb, self.nb):
            raise ValueError(f"R must be {self.nb} x {self.nb}")
        N.check(self.lib.hps_import_map(self.handle, N.HPS_EXPORT_R, index, a.ctypes.data_as(ctypes.c_void_p)))

    def launch_shapes(self):
        """Rows per warp and CTAs per SM of the apply (FP32 maps, FP64 maps) and of stage K, per
        right-hand-side group (1, 2, <=4, <=8), as chosen at setup."""
        sh = N.LaunchShapes()
        N.check(self.lib.hps_get_launch_shapes(self.handle, ctypes.byref(sh)))
        return {"apply_rows_per_warp": [list(r) for r in sh.apply_rows_per_warp],
                "apply_ctas_per_sm": [list(r) for r in sh.apply_ctas_per_sm],
                "stage_k_rows_per_warp": list(sh.stage_k_rows_per_warp),
                "stage_k_ctas_per_sm": list(sh.stage_k_ctas_per_sm), "tuned": bool(sh.tuned)}

    def profile(self, enable=None, reset=False):
        """Per-phase device times (ms) and kernel launch count since the last reset."""
        if enable is not None:
            N.check(self.lib.hps_profile_enable(self.handle, 1 if enable else 0))
        p = N.Profile()
        N.check(self.lib.hps_profile_read(self.handle, ctypes.byref(p), 1 if reset else 0))
        return {"launches": p.launches,
                "ms": {name: p.ms[i] for i, name in enumerate(N.PHASES)},
                "count": {name: p.count[i] for i, name in enumerate(N.PHASES)}}

    @property
    def memory_bytes(self):
        return self.lib.hps_memory_bytes(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.hps_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
