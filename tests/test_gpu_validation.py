"""The validation-run drivers on the GPU path, short: the systems of Table 3
sets 3 and 5 step at the paper's density and parameters, hold their
temperature, and give finite structure."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    from paper_1303_4523_gb300 import build
    build.build()


@pytest.mark.parametrize("f,theta,valency", [(0.0, 0.0, 1), (1.0, 0.0, 1), (1.0, 1.0, 3)])
def test_single_polyelectrolyte_run(built, f, theta, valency):
    from paper_1303_4523_gb300 import validation as V
    out = V.run_polyelectrolyte(f, steps=400, equil=400, every=100, theta=theta, valency=valency)
    assert out["N"] == 108000 and out["steps"] == 400
    assert abs(out["kT"] - 1.0) < 0.05                  # DPD thermostat at kT = 1
    assert 0.6 < out["bond_mean"] < 0.9                 # harmonic bonds about r_eq = 0.7
    assert 1.0 < out["rg_mean"] < 10.0


def test_electrolyte_rdf_run(built):
    from paper_1303_4523_gb300 import validation as V
    out = V.run_electrolyte_rdf(steps=800, equil=400, every=200)
    assert out["N"] == 4000 and abs(out["kT"] - 1.0) < 0.05
    g00 = np.array(out["g00"])
    r = np.array(out["r"])
    assert np.all(np.isfinite(g00)) and abs(g00[r > 2.0].mean() - 1.0) < 0.05
    assert np.all(np.isfinite(out["g_opposite"])) and np.isfinite(out["relation_mean"])
