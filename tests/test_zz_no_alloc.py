"""hps_precond_noalloc (scratch in a static device array, no allocation in the
call) must give what hps_precond gives, call after call.

Kept in a file pytest collects last, so a failure here cannot hide the other
GPU tests of a run that stops at the first failure."""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

hps = pytest.importorskip("paper_2112_02211_gb300")
from paper_2112_02211_gb300 import _native as N  # noqa: E402

import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def solver():
    w = W.scaled(W.bump_16cubed(), 4)
    w.p = 8
    xi, xf = hps.nodes(4, 4, 4, 8)
    s = hps.Solver(4, 4, 4, 8, kappa=w.kappa, eta=w.eta, b=w.sample_b(xi), max_rhs=2)
    yield s
    s.close()


def _call(solver, dtype, r, z, nrhs):
    lib = N.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.hps_precond_noalloc(solver.handle, dtype, ctypes.c_void_p(r.data_ptr()),
                                   ctypes.c_void_p(z.data_ptr()), nrhs, stream)


@pytest.mark.parametrize("dtype,cdt,tol", [(N.HPS_C128, torch.complex128, 1e-13),
                                            (N.HPS_C64, torch.complex64, 1e-6)])
def test_matches_hps_precond_twice(solver, dtype, cdt, tol):
    rng = np.random.default_rng(7)
    for call in range(2):
        nrhs = 1 + call
        r = rng.standard_normal(nrhs * solver.nf) + 1j * rng.standard_normal(nrhs * solver.nf)
        r = torch.from_numpy(r).to(cdt).cuda()
        ref = solver.precond(r)
        z = torch.full_like(r, float("nan"))
        assert _call(solver, dtype, r, z, nrhs) == N.HPS_OK, N.load().hps_last_error()
        torch.cuda.synchronize()
        err = (torch.linalg.norm(z - ref) / torch.linalg.norm(ref)).item()
        assert err <= tol, (call, err)


def test_rejects_sizes_beyond_the_static_buffer(solver):
    lib = N.load()
    per_rhs = 8 * 24 * 36 * 16  # clusters x internal slots x q^2 x complex double
    nrhs = N.HPS_PRECOND_NOALLOC_MAX_BYTES // per_rhs + 1
    r = torch.zeros(1, dtype=torch.complex128, device="cuda")
    rc = lib.hps_precond_noalloc(solver.handle, N.HPS_C128, ctypes.c_void_p(r.data_ptr()),
                                 ctypes.c_void_p(r.data_ptr()), int(nrhs), None)
    assert rc == N.HPS_EINVAL
    assert b"static buffer" in lib.hps_last_error()
