"""Pins of the oracle's leaf maps (Sec. 2.1) against closed-form solutions and
the energy identity behind the unitarity of the ItI map (no GPU)."""

import numpy as np
import pytest

import oracle as O
import workloads as W


def _leaf_exact(w, grid, leaf):
    """Exact incoming f and outgoing g of workload w on one leaf's Gauss points."""
    xf = O.face_nodes(grid)[leaf]
    nrm = np.broadcast_to(O.face_normals()[:, None, :], xf.shape)
    f = w.exact_f[0](xf, nrm).reshape(-1)
    # g = du/dn - i eta u = f - 2 i eta u
    u_fn = w.meta.get("u")
    if u_fn is None:
        d = np.array(w.meta["d"])
        u = np.exp(1j * w.kappa * (xf @ d))
    else:
        u = u_fn(xf)
    g = f - 2j * w.eta * u.reshape(-1)
    return f, g


def _leaf_error(w, leaf=5):
    grid = O.Grid(w.nx, w.ny, w.nz, w.p)
    xi = O.interior_nodes(grid)[leaf]
    c = O.cdiag_from_b(w.kappa, w.sample_b(xi))
    R, H = O.leaf_iti(grid.p, grid.h, w.eta, c)
    f, g = _leaf_exact(w, grid, leaf)
    g_h = R @ f
    if w.s is not None:
        g_h = g_h + H @ w.sample_s(xi)[0]
    return np.linalg.norm(g_h - g) / np.linalg.norm(g)


def test_plane_wave_leaf_map_converges_spectrally():
    errs = [_leaf_error(W.plane_wave(L=3, p=p, kappa=12.0, seed=4)) for p in (6, 8, 10, 12)]
    assert errs[-1] < 5e-6
    for a, b in zip(errs, errs[1:]):
        assert b < a / 8.0


def test_manufactured_leaf_maps_converge_spectrally():
    """u of Sec. 6.2 with the Gaussian bump: pins R, H and the C = kappa^2(1-b) term."""
    errs = [_leaf_error(W.manufactured(L=3, p=p, kappa=8.0), leaf=13) for p in (6, 8, 10, 12)]
    assert errs[-1] < 1e-6
    for a, b in zip(errs, errs[1:]):
        assert b < a / 8.0


def test_manufactured_without_bump_differs_from_with_bump():
    """A dropped C term would make the two equal; they are not."""
    w1 = W.manufactured(L=2, p=8, kappa=8.0, with_bump=True)
    grid = O.Grid(2, 2, 2, 8)
    xi = O.interior_nodes(grid)[7]
    c1 = O.cdiag_from_b(w1.kappa, w1.sample_b(xi))
    c0 = O.cdiag_from_b(w1.kappa, np.zeros_like(xi[:, 0]))
    R1, _ = O.leaf_iti(8, grid.h, w1.eta, c1)
    R0, _ = O.leaf_iti(8, grid.h, w1.eta, c0)
    assert np.linalg.norm(R1 - R0) > 1e-3 * np.linalg.norm(R0)


def _weighted_norm_ratio(p, kappa, bval, leaf_h=0.25):
    grid = O.Grid(4, 4, 4, p)
    xg, wg = O.gauss_legendre(grid.q)
    wsq = np.sqrt(np.tile(np.kron(wg, wg), 6))
    c = np.full(grid.layout.ni, kappa ** 2 * (1 - bval), dtype=np.complex128)
    R, _ = O.leaf_iti(p, grid.h, kappa, c)
    # smooth incoming data: a plane wave's impedance trace
    w = W.plane_wave(L=4, p=p, kappa=kappa, seed=11)
    f, _ = _leaf_exact(w, grid, 21)
    return np.linalg.norm(wsq * (R @ f)) / np.linalg.norm(wsq * f)


def test_iti_preserves_energy_on_smooth_data():
    """Real kappa, b, eta: ||g||_{L2} = ||f||_{L2} (Green's identity), the ItI
    map is unitary on resolved data (Sec. 1.1); the defect decays with p."""
    defects = [abs(_weighted_norm_ratio(p, 10.0, 0.2) - 1.0) for p in (6, 8, 10, 12)]
    assert defects[-1] < 1e-5
    assert defects[-1] < defects[0] / 100.0


def test_iti_dissipates_for_absorbing_medium():
    """Im b > 0: ||f||^2 - ||g||^2 = 4 eta kappa^2 int Im(b)|u|^2 > 0."""
    r = _weighted_norm_ratio(12, 10.0, 0.2 + 0.05j)
    assert r < 1.0 - 1e-4


def test_face_nodes_lie_on_faces():
    grid = O.Grid(2, 3, 4, 6)
    xf = O.face_nodes(grid)
    for leaf in range(grid.nleaves):
        c = grid.corner(leaf)
        for face in range(6):
            a = O.FACE_AXIS[face]
            want = c[a] + (grid.h[a] if O.FACE_SIGN[face] > 0 else 0.0)
            assert np.allclose(xf[leaf, face, :, a], want)
