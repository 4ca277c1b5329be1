"""hps_precond_noalloc (scratch in a static device array, no allocation in the
call) must give what hps_precond gives, call after call.  It is for callers
that cannot let a library allocate device memory mid-call (processes that own
the GPU's memory through their own pool or a fixed budget).

Covered: both element types on a small grid; on an 8^3-leaf grid with shared
blocks, the tensor-core stage K (blocks shared by >= 16 clusters, TMA tensor
maps built over the static array's address), the FP16 blocks, and a call with
more right-hand sides than the handle's max_rhs (the one case hps_precond
rejects).

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


@pytest.fixture(scope="module")
def shared():
    """8^3 leaves, p = 8, binned constants: most clusters share one K_c block."""
    w = W.scaled(W.bump_16cubed(), 8)
    w.p = 8
    xi, xf = hps.nodes(8, 8, 8, 8)
    s = hps.Solver(8, 8, 8, 8, kappa=w.kappa, eta=w.eta, b=w.sample_b(xi), forms=("mixed",), max_rhs=1,
                   lambda_bin=0.01)
    yield s
    s.close()


def test_shared_blocks_run_on_tensor_cores_from_the_static_array(shared):
    import oracle as O
    lam = np.array([shared.export("lambda", i)[0] for i in range(shared.nl)])
    _, cl_k = hps.plan_blocks(8, 8, 8, 8, O.binned_lambdas(lam, 0.01))
    assert np.bincount(cl_k).max() >= 16  # at least one block on the tensor-core path
    rng = np.random.default_rng(9)
    for call in range(2):
        r = torch.from_numpy(rng.standard_normal(shared.nf) + 1j * rng.standard_normal(shared.nf)).to(
            torch.complex64).cuda()
        for dtype, fp16 in ((N.HPS_C64, False), (N.HPS_C64_H16, True)):
            ref = shared.precond(r, fp16_blocks=fp16)
            z = torch.full_like(r, float("nan"))
            assert _call(shared, dtype, r, z, 1) == N.HPS_OK, N.load().hps_last_error()
            torch.cuda.synchronize()
            err = (torch.linalg.norm(z - ref) / torch.linalg.norm(ref)).item()
            assert err <= 1e-6, (call, dtype, err)


def test_more_right_hand_sides_than_max_rhs(shared):
    """nrhs = 3 > max_rhs = 1: hps_precond refuses it; the no-alloc call takes it (it fits the
    array) and each right-hand side equals hps_precond's single-RHS result."""
    rng = np.random.default_rng(10)
    nrhs = 3
    r = torch.from_numpy(rng.standard_normal(nrhs * shared.nf) + 1j * rng.standard_normal(nrhs * shared.nf)).to(
        torch.complex64).cuda()
    z = torch.full_like(r, float("nan"))
    assert _call(shared, N.HPS_C64, r, z, nrhs) == N.HPS_OK, N.load().hps_last_error()
    torch.cuda.synchronize()
    for k in range(nrhs):
        sl = slice(k * shared.nf, (k + 1) * shared.nf)
        ref = shared.precond(r[sl].clone())
        err = (torch.linalg.norm(z[sl] - ref) / torch.linalg.norm(ref)).item()
        assert err <= 1e-6, (k, err)


def test_rejects_sizes_beyond_the_static_buffer(solver):
    lib = N.load()
    per_rhs = 8 * 24 * 36 * 16  # clusters x internal slots x q^2 x complex double
    nrhs = N.HPS_PRECOND_NOALLOC_MAX_BYTES // per_rhs + 1
    r = torch.zeros(1, dtype=torch.complex128, device="cuda")
    rc = lib.hps_precond_noalloc(solver.handle, N.HPS_C128, ctypes.c_void_p(r.data_ptr()),
                                 ctypes.c_void_p(r.data_ptr()), int(nrhs), None)
    assert rc == N.HPS_EINVAL
    assert b"static buffer" in lib.hps_last_error()
