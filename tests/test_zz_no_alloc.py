"""bae_potential_apply_noalloc against bae_potential_apply, through the C ABI.

The no-allocation variant exists for callers that cannot allocate device
memory while they run; it keeps its work buffers in a fixed file-scope
device array. This file is collected last so that, if it fails, a run that
stops at the first failure has already run every other test; it also
passes on its own in a fresh process (the first call does the one-time
per-device set-up)."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-6}   # the potential-apply tolerances of the parity tests


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_05507_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _problem(ctx, P, layer="double"):
    import torch
    from paper_2502_05507_gb300 import Problem
    return Problem(ctx, torch.from_numpy(P.phi).cuda(), P.grid.h, P.grid.origin, P.kappa2, layer)


# the last case runs a smaller float64 problem after the larger float32 one
# has left its data in the shared array
CASES = [(32, "fp64", "double"), (32, "fp32", "double"), (32, "fp64", "single"), (32, "fp32", "direct"),
         (64, "fp32", "double"), (64, "fp32", "direct"), (32, "fp64", "double")]


@pytest.mark.parametrize("N,precision,layer", CASES)
def test_noalloc_matches_allocating_apply_twice(ctx, N, precision, layer):
    import torch
    from paper_2502_05507_gb300 import bae
    L = bae.lib()
    P = W.torus_helmholtz(N, kappa2=10.0)
    prob = _problem(ctx, P, layer)
    prec = bae._PREC[precision]
    for call in range(2):   # two calls in a row share the same static scratch
        q = torch.from_numpy(W.random_density(prob.n_unknowns, seed=100 + call)).cuda()
        ref = torch.empty((N,) * 3, dtype=torch.float64, device="cuda")
        got = torch.full((N,) * 3, float("nan"), dtype=torch.float64, device="cuda")
        assert L.bae_potential_apply(prob._h, prec, q.data_ptr(), ref.data_ptr()) == bae.OK
        rc = L.bae_potential_apply_noalloc(prob._h, prec, q.data_ptr(), got.data_ptr())
        assert rc == bae.OK, L.bae_last_error()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.max(np.abs(g - r)) <= TOL[precision] * np.max(np.abs(r))
    prob.close()


def test_noalloc_rejects_oversize_and_host_arrays(ctx):
    import torch
    from paper_2502_05507_gb300 import bae
    L = bae.lib()
    P = W.torus_helmholtz(128, kappa2=10.0)
    prob = _problem(ctx, P)
    q = torch.zeros(prob.n_unknowns, dtype=torch.float64, device="cuda")
    v = torch.zeros((128,) * 3, dtype=torch.float64, device="cuda")
    rc = L.bae_potential_apply_noalloc(prob._h, bae.FP32, q.data_ptr(), v.data_ptr())
    assert rc == bae.ERR_INVALID_ARG
    assert b"scratch" in L.bae_last_error()
    prob.close()
    P = W.sphere_exp(16)
    prob = _problem(ctx, P)
    qh = np.zeros(prob.n_unknowns)
    vh = np.zeros((16,) * 3)
    rc = L.bae_potential_apply_noalloc(prob._h, bae.FP64, qh.ctypes.data, vh.ctypes.data)
    assert rc == bae.ERR_INVALID_ARG
    prob.close()


def test_noalloc_restores_current_device(ctx):
    """The call switches to the problem's device while it runs and gives
    the caller back the device that was current before."""
    import torch
    from paper_2502_05507_gb300 import bae
    L = bae.lib()
    P = W.sphere_exp(16)
    prob = _problem(ctx, P)
    q = torch.zeros(prob.n_unknowns, dtype=torch.float64, device="cuda")
    v = torch.zeros((16,) * 3, dtype=torch.float64, device="cuda")
    before = torch.cuda.current_device()
    assert L.bae_potential_apply_noalloc(prob._h, bae.FP64, q.data_ptr(), v.data_ptr()) == bae.OK
    assert torch.cuda.current_device() == before
    prob.close()
