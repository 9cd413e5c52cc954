"""Consistency of the stored oracle images (``tests/golden/*.npz``, written by
``tests/golden/make_pd_golden.py`` from ``synth`` and the oracle only): the stored noise level,
eps and gamma follow from the regenerated inputs by their rules, and the stored residual
norm is ||y - Phi x|| of the stored image under the oracle's Phi."""

import importlib.util
import os

import numpy as np
import pytest

from oracle import solvers as so

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _mk():
    spec = importlib.util.spec_from_file_location("make_pd_golden", os.path.join(GOLDEN, "make_pd_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name", ["small", "large"])
def test_stored_image_consistent_with_oracle(name):
    mk = _mk()
    p = mk.PROBLEMS[name]
    st = np.load(os.path.join(GOLDEN, p["file"]))
    x_true, uvw, geo, ops, y, sigma = mk.inputs(p["n"], p["M"], p["npts"], p["nblobs"], p["seed"])
    assert float(st["sigma"]) == pytest.approx(sigma, rel=1e-12)
    assert float(st["eps"]) == pytest.approx(so.epsilon_from_sigma(sigma, p["M"]), rel=1e-14)
    x = st["x"].astype(np.float64)
    assert x.shape == (p["n"], p["n"]) and np.all(x >= 0) and int(st["iters"]) == p["iters"]
    res = float(np.linalg.norm(y.astype(np.complex128) - ops[0](x)))
    # FP32 storage of the large image perturbs the residual by ~1e-7 relative
    assert res == pytest.approx(float(st["residual_norm"]), rel=1e-12 if p["store"] is np.float64 else 1e-5)
    if name == "small":
        gam = so.default_gamma(y.astype(np.complex128), ops[1], ops[3], float(st["op_norm_sq"]))
        assert float(st["gamma"]) == pytest.approx(gam, rel=1e-12)
