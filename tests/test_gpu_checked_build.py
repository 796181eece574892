"""The debug build (device index checks, ENUF_CHECK) on the GPU: evaluations
in both precisions, both force modes and a few DPD steps record no failed
check and give the release build's forces."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np, torch
from paper_1303_4523_gb300 import enuf, workloads as W
assert enuf.lib.enuf_built_with_checks() == 1
out = []
for prec, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
    for deriv in (0, 1):
        for s in (W.electrolyte_small("paper"), W.electrolyte(3000, 15.0, n_charged=600, seed_offset=7)):
            P = dict(L=s.L, M=s.M, **s.params)
            plan = enuf.Plan(enuf.make_params(prec=prec, deriv=deriv, **P), s.N)
            pos = torch.tensor(s.pos, dtype=dt, device="cuda")
            q = torch.tensor(s.q, dtype=dt, device="cuda")
            F = torch.empty_like(pos)
            plan.energy_forces(pos, q, F)
            plan.energy_forces(pos, q, F)
            assert plan.check_word() == 0, (prec, deriv, s.name)
            out.append(F.double().cpu().numpy())
            plan.close()
    s = W.polyelectrolyte(L=10.0, density=4.0, n_chains=2, chain_len=48, f=1.0, salt_fraction=0.05,
                          seed_offset=44)
    dp = W.dpd_params(5)
    plan = enuf.Plan(enuf.make_params(prec=prec, L=s.L, M=s.M, **s.params), s.N)
    sysm = enuf.DpdSystem(plan, dp["a"], dp["gamma"], dp["sigma"], dp["dt"], s.pos, s.vel, s.types, s.q,
                          s.bonds, lambda_vv=dp["lambda_vv"], K_bond=dp["K_bond"], r0_bond=dp["r0_bond"],
                          seed=dp["seed"])
    sysm.step(5)
    assert plan.check_word() == 0, (prec, "dpd")
    out.append(sysm.get_state()[2].astype(np.float64))
    sysm.close()
    plan.close()
np.savez(OUT, *out)
print("checked ok")
"""


def _run(env_check, path):
    env = dict(os.environ, ENUF_CHECK="1" if env_check else "0", PYTHONPATH=ROOT)
    code = SCRIPT.replace("OUT", repr(path))
    if not env_check:
        code = code.replace("assert enuf.lib.enuf_built_with_checks() == 1", "")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, cwd=ROOT,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return r


def test_checked_build_runs_clean(tmp_path):
    import numpy as np
    from paper_1303_4523_gb300 import build
    build.build(check=True)
    build.build()
    _run(True, str(tmp_path / "chk.npz"))
    _run(False, str(tmp_path / "rel.npz"))
    a, b = np.load(tmp_path / "chk.npz"), np.load(tmp_path / "rel.npz")
    for k in a.files:
        x, y = a[k], b[k]
        rel = np.sqrt(((x - y) ** 2).sum() / max((y ** 2).sum(), 1e-300))
        assert rel < 1e-4, (k, rel)
