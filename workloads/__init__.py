"""Seeded synthetic workloads for the HPS Helmholtz solver.

This module only produces input data: the medium b(x), body loads s(x) and
boundary data t(x, n) of problem (1.1) of arXiv:2112.02211,

    -Lap u - kappa^2 (1 - b) u = s  in (0,1)^3,   du/dn + i eta u = t  on the boundary,

as plain functions of points, plus the grid and solver parameters of each
workload.  It holds none of the method's arithmetic (no nodes, no operators):
both the CPU oracle and the CUDA path's harness evaluate these functions at
points they compute themselves.  All randomness comes from NumPy PCG64
generators with fixed seeds.

Workloads (sizes: leaves per axis L, Chebyshev order p, q = p - 2 Gauss
points per face edge):

* ``plane_wave``  b = 0, s = 0, u = exp(i kappa d.x): t and the exact
  incoming data on every leaf face are i (kappa d.n + eta) u.
* ``manufactured``  the paper's test solution of Sec. 6.2,
  u = e^{i kappa (x+y+z)} e^x cosh(y) (z+1)^2, with the Gaussian bump medium
  b = -1.5 exp(-160 |x - 0.5|^2) of eq. (source); s and t follow from u.
* ``plane_wave_4cubed``  4^3 leaves, p = 8, kappa = eta = 10, plane wave with
  a seeded direction (seed 1), GMRES(50), tol 1e-10.
* ``bump_16cubed``  16^3 leaves, p = 10, kappa = eta = 40,
  b = 1.5 exp(-160 |x - c|^2) (c seeded), s = exp(-400 |x - x0|^2), t = 0,
  tol 1e-6.
* ``multi_rhs_16cubed``  16^3 leaves, p = 12, kappa = eta = 60, five seeded
  Gaussian bumps, 64 Gaussian point sources of width 0.02.
* ``large_32cubed``  32^3 leaves, p = 10, kappa = eta = 200, smooth random
  complex medium from 16 Fourier modes, one Gaussian source of width 0.01.
* ``serving_stream``  500 requests with Poisson arrivals.
"""

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

__all__ = ["Workload", "plane_wave", "manufactured", "plane_wave_4cubed", "bump_16cubed",
           "multi_rhs_16cubed", "large_32cubed", "serving_stream", "gaussian_bumps",
           "scaled", "by_name"]


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    p: int
    kappa: float
    eta: float
    b: Callable  # b(xyz[..., 3]) -> complex
    s: Optional[List[Callable]] = None  # one function of xyz per right-hand side
    t: Optional[List[Callable]] = None  # one function of (xyz, outward normal) per RHS
    exact_f: Optional[List[Callable]] = None  # exact incoming data f(xyz, normal)
    tol: float = 1e-10
    restart: int = 50
    meta: dict = field(default_factory=dict)

    @property
    def q(self):
        return self.p - 2

    @property
    def nrhs(self):
        if self.s is not None:
            return len(self.s)
        if self.t is not None:
            return len(self.t)
        return 1

    @property
    def nleaves(self):
        return self.nx * self.ny * self.nz

    @property
    def face_unknowns(self):
        return self.nleaves * 6 * self.q * self.q

    def sample_b(self, xyz):
        return np.asarray(self.b(np.asarray(xyz)), dtype=np.complex128)

    def sample_s(self, xyz):
        """Body loads at points xyz[..., 3] -> (nrhs, ...) complex, or None."""
        if self.s is None:
            return None
        return np.stack([np.asarray(fn(xyz), dtype=np.complex128) for fn in self.s])

    def sample_t(self, xyz, normals):
        """Boundary data at face points with their outward normals -> (nrhs, ...)."""
        if self.t is None:
            return None
        return np.stack([np.asarray(fn(xyz, normals), dtype=np.complex128) for fn in self.t])


def _zero(xyz):
    return np.zeros(np.asarray(xyz).shape[:-1], dtype=np.complex128)


def _plane_wave_fns(kappa, eta, d):
    d = np.asarray(d, dtype=np.float64)

    def u(xyz):
        return np.exp(1j * kappa * (np.asarray(xyz) @ d))

    def impedance(xyz, n):
        dn = np.sum(np.asarray(n) * d, axis=-1)
        return 1j * (kappa * dn + eta) * u(xyz)

    return impedance


def plane_wave(L=2, p=8, kappa=10.0, eta=None, d=None, seed=1, tol=1e-12, name="plane_wave"):
    """b = 0, s = 0 and t from u = exp(i kappa d.x), |d| = 1."""
    eta = kappa if eta is None else eta
    if d is None:
        rng = np.random.default_rng(seed)
        d = rng.standard_normal(3)
    d = np.asarray(d, dtype=np.float64)
    d = d / np.linalg.norm(d)
    imp = _plane_wave_fns(kappa, eta, d)
    return Workload(name=name, nx=L, ny=L, nz=L, p=p, kappa=kappa, eta=eta, b=_zero,
                    s=None, t=[imp], exact_f=[imp], tol=tol, meta={"d": d.tolist()})


def _paper_bump(xyz):
    r2 = np.sum((np.asarray(xyz) - 0.5) ** 2, axis=-1)
    return (-1.5 * np.exp(-160.0 * r2)).astype(np.complex128)


def manufactured(L=2, p=10, kappa=10.0, eta=None, tol=1e-12, with_bump=True):
    """u = e^{i kappa (x+y+z)} e^x cosh(y) (z+1)^2 (Sec. 6.2) with s, t built from it."""
    eta = kappa if eta is None else eta
    k = kappa
    bfun = _paper_bump if with_bump else _zero

    def parts(xyz):
        xyz = np.asarray(xyz)
        x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
        ex = np.exp((1j * k + 1.0) * x)
        ey = np.exp(1j * k * y)
        ez = np.exp(1j * k * z)
        f1, f1p, f1pp = ex, (1j * k + 1.0) * ex, (1j * k + 1.0) ** 2 * ex
        f2 = ey * np.cosh(y)
        f2p = ey * (1j * k * np.cosh(y) + np.sinh(y))
        f2pp = ey * ((1.0 - k * k) * np.cosh(y) + 2j * k * np.sinh(y))
        f3 = ez * (z + 1.0) ** 2
        f3p = ez * (1j * k * (z + 1.0) ** 2 + 2.0 * (z + 1.0))
        f3pp = ez * (-k * k * (z + 1.0) ** 2 + 4j * k * (z + 1.0) + 2.0)
        return (f1, f1p, f1pp), (f2, f2p, f2pp), (f3, f3p, f3pp)

    def u(xyz):
        a, b_, c = parts(xyz)
        return a[0] * b_[0] * c[0]

    def s(xyz):
        a, b_, c = parts(xyz)
        lap = a[2] * b_[0] * c[0] + a[0] * b_[2] * c[0] + a[0] * b_[0] * c[2]
        return -lap - k * k * (1.0 - bfun(xyz)) * a[0] * b_[0] * c[0]

    def imp(xyz, n):
        a, b_, c = parts(xyz)
        grad = np.stack([a[1] * b_[0] * c[0], a[0] * b_[1] * c[0], a[0] * b_[0] * c[1]], axis=-1)
        dn = np.sum(grad * np.asarray(n), axis=-1)
        return dn + 1j * eta * a[0] * b_[0] * c[0]

    return Workload(name="manufactured", nx=L, ny=L, nz=L, p=p, kappa=kappa, eta=eta, b=bfun,
                    s=[s], t=[imp], exact_f=[imp], tol=tol, meta={"u": u})


def manufactured_bumps(L=2, p=10, kappa=10.0, eta=None, tol=1e-12, with_bump=True):
    """u = (1 + e^{i kappa x})(1 + e^{i kappa y})(1 + e^{i kappa z}) ln(1 + x^2 + y^2 + z^2)
    (Sec. 6.3, eq. (bumps), not separable) with s, t built from it; medium b of eq. (source)."""
    eta = kappa if eta is None else eta
    k = kappa
    bfun = _paper_bump if with_bump else _zero

    def parts(xyz):
        xyz = np.asarray(xyz)
        e = [np.exp(1j * k * xyz[..., a]) for a in range(3)]
        f = [1.0 + ea for ea in e]
        fp = [1j * k * ea for ea in e]
        fpp = [-k * k * ea for ea in e]
        r2 = np.sum(xyz * xyz, axis=-1)
        g = np.log1p(r2)
        gp = [2.0 * xyz[..., a] / (1.0 + r2) for a in range(3)]
        lapg = (6.0 + 2.0 * r2) / (1.0 + r2) ** 2
        return f, fp, fpp, g, gp, lapg

    def u(xyz):
        f, fp, fpp, g, gp, lapg = parts(xyz)
        return f[0] * f[1] * f[2] * g

    def grad(xyz):
        f, fp, fpp, g, gp, lapg = parts(xyz)
        F = f[0] * f[1] * f[2]
        dF = [fp[0] * f[1] * f[2], f[0] * fp[1] * f[2], f[0] * f[1] * fp[2]]
        return np.stack([dF[a] * g + F * gp[a] for a in range(3)], axis=-1)

    def s(xyz):
        f, fp, fpp, g, gp, lapg = parts(xyz)
        F = f[0] * f[1] * f[2]
        dF = [fp[0] * f[1] * f[2], f[0] * fp[1] * f[2], f[0] * f[1] * fp[2]]
        lapF = fpp[0] * f[1] * f[2] + f[0] * fpp[1] * f[2] + f[0] * f[1] * fpp[2]
        lap = lapF * g + 2.0 * sum(dF[a] * gp[a] for a in range(3)) + F * lapg
        return -lap - k * k * (1.0 - bfun(xyz)) * F * g

    def imp(xyz, n):
        dn = np.sum(grad(xyz) * np.asarray(n), axis=-1)
        return dn + 1j * eta * u(xyz)

    return Workload(name="manufactured_bumps", nx=L, ny=L, nz=L, p=p, kappa=kappa, eta=eta, b=bfun,
                    s=[s], t=[imp], exact_f=[imp], tol=tol, meta={"u": u})


def plane_wave_4cubed():
    """Plain FP64 workload: 4^3 leaves, p = 8, q = 6, kappa = eta = 10, b = 0, s = 0."""
    w = plane_wave(L=4, p=8, kappa=10.0, eta=10.0, seed=1, tol=1e-10, name="plane_wave_4cubed")
    return w


def gaussian(center, width=None, exponent=None):
    """exp(-|x-c|^2/(2 width^2)), or exp(-exponent |x-c|^2) when `exponent` is given."""
    c = np.asarray(center, dtype=np.float64)
    a = exponent if exponent is not None else 1.0 / (2.0 * width * width)

    def fn(xyz):
        r2 = np.sum((np.asarray(xyz) - c) ** 2, axis=-1)
        return np.exp(-a * r2).astype(np.complex128)

    return fn


def gaussian_bumps(rng, count, amp=(-0.5, 0.5), sigma=(0.05, 0.15), lo=0.1, hi=0.9):
    """Sum of `count` Gaussian bumps with seeded amplitudes, widths and centres."""
    a = rng.uniform(amp[0], amp[1], size=count)
    sg = rng.uniform(sigma[0], sigma[1], size=count)
    c = rng.uniform(lo, hi, size=(count, 3))

    def fn(xyz):
        xyz = np.asarray(xyz)
        out = np.zeros(xyz.shape[:-1], dtype=np.complex128)
        for i in range(count):
            r2 = np.sum((xyz - c[i]) ** 2, axis=-1)
            out += a[i] * np.exp(-r2 / (2.0 * sg[i] ** 2))
        return out

    return fn, {"amp": a.tolist(), "sigma": sg.tolist(), "centre": c.tolist()}


def bump_16cubed(L=16, p=10, kappa=40.0):
    """Variable coefficient, one RHS: b = 1.5 exp(-160|x-c|^2), s = exp(-400|x-x0|^2), t = 0."""
    c = np.random.default_rng(2).uniform(0.3, 0.7, size=3)
    x0 = np.random.default_rng(3).uniform(0.2, 0.8, size=3)
    bump = gaussian(c, exponent=160.0)

    def b(xyz):
        return 1.5 * bump(xyz)

    return Workload(name="bump_16cubed", nx=L, ny=L, nz=L, p=p, kappa=kappa, eta=kappa, b=b,
                    s=[gaussian(x0, exponent=400.0)], t=None, tol=1e-6,
                    meta={"c": c.tolist(), "x0": x0.tolist()})


def multi_rhs_16cubed(L=16, p=12, kappa=60.0, nrhs=64):
    """Five seeded bumps, `nrhs` Gaussian sources of width 0.02, t = 0."""
    rng = np.random.default_rng(4)
    b, meta = gaussian_bumps(rng, 5)
    xr = np.random.default_rng(5).uniform(0.1, 0.9, size=(nrhs, 3))
    s = [gaussian(xr[i], width=0.02) for i in range(nrhs)]
    meta["sources"] = xr.tolist()
    return Workload(name="multi_rhs_16cubed", nx=L, ny=L, nz=L, p=p, kappa=kappa, eta=kappa,
                    b=b, s=s, t=None, tol=1e-6, meta=meta)


def large_32cubed(L=32, p=10, kappa=200.0):
    """Smooth random complex medium from 16 Fourier modes; Gaussian source (width 0.01) at the centre."""
    rng = np.random.default_rng(6)
    modes = []
    while len(modes) < 16:
        k = rng.integers(-3, 4, size=3)
        if np.any(k != 0) and not any(np.array_equal(k, m) for m in modes):
            modes.append(k)
    modes = np.array(modes, dtype=np.float64)
    amp_re = rng.standard_normal(16)
    ph_re = rng.uniform(0, 2 * np.pi, 16)
    amp_im = rng.standard_normal(16)
    ph_im = rng.uniform(0, 2 * np.pi, 16)

    def field_(xyz, amp, ph):
        xyz = np.asarray(xyz)
        arg = 2 * np.pi * (xyz @ modes.T) + ph
        return np.cos(arg) @ amp

    # Normalisation over a fixed 32^3 lattice of cell centres.
    g = (np.arange(32) + 0.5) / 32
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    sre = 0.295 / np.max(np.abs(field_(lat, amp_re, ph_re)))
    sim = 1.0 / np.max(np.abs(field_(lat, amp_im, ph_im)))

    def b(xyz):
        fi = np.clip(field_(xyz, amp_im, ph_im) * sim, -1.0, 1.0)
        return sre * field_(xyz, amp_re, ph_re) + 1j * 0.025 * (1.0 + fi)

    return Workload(name="large_32cubed", nx=L, ny=L, nz=L, p=p, kappa=kappa, eta=kappa, b=b,
                    s=[gaussian([0.5, 0.5, 0.5], width=0.01)], t=None, tol=1e-5,
                    meta={"modes": modes.tolist()})


def serving_stream(n=500, rate=20.0, seed=7, L_range=(8, 24), p_choices=(8, 10, 12), kappa_range=(20.0, 120.0),
                   max_sources=16):
    """Request stream: Poisson arrivals (mean `rate`/s); per request L in L_range (inclusive),
    p in p_choices, kappa ~ U[kappa_range], 3-8 Gaussian bumps, 1-max_sources Gaussian sources
    (width 0.02).  The defaults are the serving workload; smaller ranges give a scaled stream
    with the same recipe."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        L = int(rng.integers(L_range[0], L_range[1] + 1))
        p = int(rng.choice(list(p_choices)))
        kappa = float(rng.uniform(kappa_range[0], kappa_range[1]))
        nb = int(rng.integers(3, 9))
        b, meta = gaussian_bumps(rng, nb)
        ns = int(rng.integers(1, max_sources + 1))
        xs = rng.uniform(0.1, 0.9, size=(ns, 3))
        s = [gaussian(xs[j], width=0.02) for j in range(ns)]
        w = Workload(name=f"request_{i}", nx=L, ny=L, nz=L, p=p, kappa=kappa, eta=kappa, b=b,
                     s=s, t=None, tol=1e-6, meta=dict(meta, arrival=t))
        out.append(w)
    return out


def scaled(w, L):
    """The same medium, sources and parameters on an L^3 grid (a smaller instance)."""
    return Workload(name=f"{w.name}@{L}", nx=L, ny=L, nz=L, p=w.p, kappa=w.kappa, eta=w.eta,
                    b=w.b, s=w.s, t=w.t, exact_f=w.exact_f, tol=w.tol, restart=w.restart,
                    meta=w.meta)


def by_name(name):
    return {
        "plane_wave_4cubed": plane_wave_4cubed,
        "bump_16cubed": bump_16cubed,
        "multi_rhs_16cubed": multi_rhs_16cubed,
        "large_32cubed": large_32cubed,
    }[name]()
