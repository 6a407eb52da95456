"""The fused Arnoldi step (one cooperative kernel with grid barriers) and the
two-kernel step use the same partition and order for every sum, so a solve
gives bit-identical densities, solutions and iteration counts with either
(GMRES of Section 4.1 around the BAE of eq. [double_bae], Gram-Schmidt with
delayed reorthogonalisation). The two-kernel step runs in a child process
with BAE_ARNOLDI_COOP=0."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, json, numpy as np, torch
sys.path.insert(0, {root!r})
import workloads as W
from paper_2502_05507_gb300 import Context, Problem
out = {{}}
P = W.torus_helmholtz(64, kappa2=10.0)
ctx = Context(0)
prob = Problem(ctx, torch.from_numpy(P.phi).cuda(), P.grid.h, P.grid.origin, P.kappa2, "double")
g = torch.from_numpy(P.g_at(prob.boundary_points())).cuda()
f = torch.from_numpy(P.f()).cuda()
for prec in ("mixed", "fp64"):
    q, u, st = prob.solve(f, g, tol=1e-10, precision=prec)
    np.save({path!r} + "_" + prec + "_q.npy", q.cpu().numpy())
    np.save({path!r} + "_" + prec + "_u.npy", u.cpu().numpy())
    out[prec] = st["iterations"]
# short restart cycles (the last column of every cycle, the restart
# boundary) and an iteration cap that stops a cycle in the middle
q, u, st = prob.solve(f, g, tol=1e-10, precision="fp64", restart=7)
np.save({path!r} + "_r7_u.npy", u.cpu().numpy())
out["r7"] = st["iterations"]
q, u, st = prob.solve(f, g, tol=1e-10, precision="fp64", restart=11, max_iter=30, allow_not_converged=True)
np.save({path!r} + "_cap_u.npy", u.cpu().numpy())
out["cap"] = [st["iterations"], st["rel_residual"]]
xyz = np.asarray(prob.boundary_points())
G = np.stack([P.g_at(xyz), np.sin(xyz[:, 0]) + xyz[:, 1] * xyz[:, 2], np.cos(2 * xyz[:, 2])])
F = np.stack([P.f(), np.zeros_like(P.f()), P.f()])
qb, ub, stb = prob.solve_batched(torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda(), tol=1e-10,
                                 precision="mixed")
np.save({path!r} + "_batch_u.npy", ub.cpu().numpy())
out["batch"] = [s["iterations"] for s in stb]
print(json.dumps(out))
"""


def _run(tmp_path, tag, env_extra):
    path = str(tmp_path / tag)
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, path=path)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return path, json.loads(r.stdout.strip().splitlines()[-1])


def test_fused_step_bit_identical_to_three_kernel_step(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    p_on, it_on = _run(tmp_path, "coop", {})
    p_off, it_off = _run(tmp_path, "three", {"BAE_ARNOLDI_COOP": "0"})
    assert it_on == it_off
    assert it_on["cap"][0] == 30, it_on
    for name in ("mixed_q", "mixed_u", "fp64_q", "fp64_u", "batch_u", "r7_u", "cap_u"):
        a = np.load(p_on + "_" + name + ".npy")
        b = np.load(p_off + "_" + name + ".npy")
        assert np.array_equal(a, b), name
