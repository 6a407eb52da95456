"""Failure detection without a GPU fault.

Two host-side injections (bae_inject_fault):
- the fused Arnoldi step's grid-barrier waits are made to run out (the
  launch waits for one CTA more than its grid has, with a ~1 ms poll limit):
  the solve returns BAE_ERR_TIMEOUT promptly, and the next solve on the same
  context matches the oracle;
- a cap on the size of one device allocation: problem creation and a solve
  return BAE_ERR_OOM, and after the cap is cleared the same context solves
  correctly.
Nothing here faults, traps or hangs the GPU: every device wait is bounded.
"""
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from oracle import solve as S
    from paper_2502_05507_gb300 import Context
    P = W.sphere_exp(32)
    ref = S.solve(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, P.kappa2, tol=1e-12)
    c = Context(0)
    yield c, P, ref
    c.close()


def _solve(ctx, P, precision="mixed"):
    import torch
    from paper_2502_05507_gb300 import Problem
    pr = Problem(ctx, torch.from_numpy(P.phi).cuda(), P.grid.h, P.grid.origin, P.kappa2, "double")
    try:
        g = torch.from_numpy(P.g_at(np.asarray(pr.boundary_points()))).cuda()
        f = torch.from_numpy(P.f()).cuda()
        return pr.solve(f, g, tol=1e-10, precision=precision)
    finally:
        pr.close()


def _err(u, ref):
    m = ref.cls.nplus
    u = u.cpu().numpy()
    return np.max(np.abs(u[m] - ref.u[m])) / np.max(np.abs(ref.u[m]))


def test_barrier_timeout_reports_and_context_recovers(env):
    from paper_2502_05507_gb300 import bae
    ctx, P, ref = env
    q, u, st = _solve(ctx, P)            # warm: kernels configured, spectrum cached
    assert _err(u, ref) < 1e-8
    bae.inject_fault(bae.FAULT_BARRIER, 1)
    try:
        t = time.perf_counter()
        with pytest.raises(bae.BAEError) as ei:
            _solve(ctx, P)
        dt = time.perf_counter() - t
    finally:
        bae.inject_fault(bae.FAULT_NONE)
    assert ei.value.code == bae.ERR_TIMEOUT, str(ei.value)
    assert "barrier" in str(ei.value)
    assert dt < 5.0                       # a ~1 ms poll limit per wait, not the half-second one
    # the same context: a correct solve right after
    q, u, st = _solve(ctx, P)
    assert _err(u, ref) < 1e-8
    q, u, st = _solve(ctx, P, "fp64")
    assert _err(u, ref) < 1e-8


def test_allocation_cap_reports_oom_and_context_recovers(env):
    import torch
    from paper_2502_05507_gb300 import Problem, bae
    ctx, P, ref = env
    Pbig = W.torus_helmholtz(64, kappa2=10.0)
    bae.inject_fault(bae.FAULT_ALLOC_CAP, 64 << 10)    # no device allocation above 64 KiB
    try:
        with pytest.raises(bae.BAEError) as ei:
            Problem(ctx, torch.from_numpy(Pbig.phi).cuda(), Pbig.grid.h, Pbig.grid.origin, Pbig.kappa2, "double")
        assert ei.value.code == bae.ERR_OOM, str(ei.value)
    finally:
        bae.inject_fault(bae.FAULT_NONE)
    # a solve whose work space has to grow fails the same way
    pr = Problem(ctx, torch.from_numpy(Pbig.phi).cuda(), Pbig.grid.h, Pbig.grid.origin, Pbig.kappa2, "double")
    g = torch.from_numpy(Pbig.g_at(np.asarray(pr.boundary_points()))).cuda()
    f = torch.from_numpy(Pbig.f()).cuda()
    bae.inject_fault(bae.FAULT_ALLOC_CAP, 1 << 20)
    try:
        with pytest.raises(bae.BAEError) as ei:
            pr.solve_batched(torch.stack([f] * 8), torch.stack([g] * 8), tol=1e-10, precision="mixed")
        assert ei.value.code == bae.ERR_OOM, str(ei.value)
    finally:
        bae.inject_fault(bae.FAULT_NONE)
    pr.close()
    # cleared: the same context solves correctly
    q, u, st = _solve(ctx, P)
    assert _err(u, ref) < 1e-8


def test_inject_fault_rejects_unknown_kind():
    pytest.importorskip("torch")
    from paper_2502_05507_gb300 import bae
    assert bae.lib().bae_inject_fault(99, 0) == bae.ERR_INVALID_ARG
