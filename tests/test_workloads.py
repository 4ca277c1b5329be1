"""The seeded input generators against the recipes they state: grid and solver parameters,
value ranges, source widths and the request mix of the serving stream.  They are the only code
the oracle and the CUDA path share, so a drift here would move both sides at once and no parity
test would see it."""

import numpy as np
import pytest

import workloads as W


def _points(n, seed=0):
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=(n, 3))


def test_bump_16cubed_recipe():
    w = W.bump_16cubed()
    assert (w.nx, w.ny, w.nz, w.p, w.q) == (16, 16, 16, 10, 8)
    assert w.kappa == w.eta == 40.0 and w.tol == 1e-6 and w.t is None
    c, x0 = np.array(w.meta["c"]), np.array(w.meta["x0"])
    assert np.all((0.3 < c) & (c < 0.7)) and np.all((0.2 < x0) & (x0 < 0.8))
    # b = 1.5 exp(-160 r^2): peak 1.5 at c, exp(-160 r^2) decay along any direction
    d = np.array([0.05, -0.02, 0.03])
    assert w.sample_b(c[None])[0] == pytest.approx(1.5)
    assert w.sample_b((c + d)[None])[0] == pytest.approx(1.5 * np.exp(-160.0 * d @ d))
    assert w.sample_s(x0[None])[0, 0] == pytest.approx(1.0)
    assert w.sample_s((x0 + d)[None])[0, 0] == pytest.approx(np.exp(-400.0 * d @ d))
    assert w.face_unknowns == 16 ** 3 * 6 * 64


def test_multi_rhs_recipe():
    w = W.multi_rhs_16cubed()
    assert (w.nx, w.p, w.q, w.kappa, w.eta, w.nrhs, w.tol) == (16, 12, 10, 60.0, 60.0, 64, 1e-6)
    amp, sg = np.array(w.meta["amp"]), np.array(w.meta["sigma"])
    assert len(amp) == len(sg) == 5
    assert np.all(np.abs(amp) <= 0.5) and np.all((0.05 <= sg) & (sg <= 0.15))
    xs = np.array(w.meta["sources"])
    assert xs.shape == (64, 3) and len(set(map(tuple, xs))) == 64
    # width 0.02: exp(-r^2 / (2 * 0.02^2)), so exp(-1/2) at distance 0.02
    s = w.sample_s(np.stack([xs[7], xs[7] + [0.02, 0.0, 0.0]]))
    assert s.shape == (64, 2)
    assert s[7, 0] == pytest.approx(1.0) and s[7, 1] == pytest.approx(np.exp(-0.5))
    # the medium is the sum of the five bumps
    c = np.array(w.meta["centre"])
    x = _points(200, 1)
    ref = sum(a * np.exp(-np.sum((x - ci) ** 2, axis=-1) / (2 * g * g)) for a, g, ci in zip(amp, sg, c))
    assert np.allclose(w.sample_b(x), ref, rtol=0, atol=1e-14)


def test_large_recipe():
    w = W.large_32cubed()
    assert (w.nx, w.p, w.q, w.kappa, w.eta, w.tol) == (32, 10, 8, 200.0, 200.0, 1e-5)
    modes = np.array(w.meta["modes"])
    assert modes.shape == (16, 3) and len(set(map(tuple, modes))) == 16
    b = w.sample_b(_points(200_000, 2))
    assert np.max(np.abs(b.real)) <= 0.3
    assert b.imag.min() >= 0.0 and b.imag.max() <= 0.05
    assert np.max(np.abs(b.real)) > 0.2  # normalised to the bound, not far below it
    centre = np.array([[0.5, 0.5, 0.5], [0.51, 0.5, 0.5]])
    s = w.sample_s(centre)[0]
    assert s[0] == pytest.approx(1.0) and s[1] == pytest.approx(np.exp(-0.5))
    assert w.face_unknowns == 32 ** 3 * 6 * 64


def test_serving_stream_recipe():
    reqs = W.serving_stream()
    assert len(reqs) == 500
    arrivals = np.array([r.meta["arrival"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], arrivals]))
    assert np.all(gaps > 0)
    # exponential gaps with mean 1/20 s: the sample mean of 500 is within 4 standard errors
    assert abs(gaps.mean() - 0.05) < 4 * 0.05 / np.sqrt(500)
    Ls = {r.nx for r in reqs}
    assert min(Ls) >= 8 and max(Ls) <= 24 and len(Ls) > 10
    assert {r.p for r in reqs} == {8, 10, 12}
    kap = np.array([r.kappa for r in reqs])
    assert kap.min() >= 20.0 and kap.max() <= 120.0
    nb = [len(r.meta["amp"]) for r in reqs]
    assert min(nb) >= 3 and max(nb) <= 8
    ns = [r.nrhs for r in reqs]
    assert min(ns) >= 1 and max(ns) <= 16
    for r in reqs[:20]:
        assert r.nx == r.ny == r.nz and r.eta == r.kappa and r.tol == 1e-6 and r.t is None
        assert np.all(np.abs(r.meta["amp"]) <= 0.5)


def test_generators_are_seeded():
    a, b = W.large_32cubed(), W.large_32cubed()
    x = _points(50, 3)
    assert np.array_equal(a.sample_b(x), b.sample_b(x))
    r1, r2 = W.serving_stream(n=5), W.serving_stream(n=5)
    assert [(r.nx, r.p, r.kappa) for r in r1] == [(r.nx, r.p, r.kappa) for r in r2]


def test_scaled_keeps_the_medium():
    w = W.bump_16cubed()
    s = W.scaled(w, 4)
    assert (s.nx, s.ny, s.nz) == (4, 4, 4) and (s.p, s.kappa, s.tol) == (w.p, w.kappa, w.tol)
    x = _points(30, 4)
    assert np.array_equal(s.sample_b(x), w.sample_b(x))
