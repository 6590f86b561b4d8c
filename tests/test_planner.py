"""The product's planner (host code, psht_plan_params) against the oracle's plan_params on the CPU:
ring count, band limits, grid sizes, kept rows and polar cutoffs exactly, the apodisation length
and ring colatitudes to rounding, the window weights to 1e-12, over spins, band limits, patch
sizes, tolerances, both bells, kappa, the cost-minimising apodisation and the full-sky route."""
import math

import numpy as np
import pytest

import oracle as O

CASES = [
    # lmax, s, theta* (deg), eps, kwargs
    (64, 0, 10.0, 1e-10, {}),
    (4096, 2, 34.744, 1e-5, {}),
    (4096, 2, 34.744, 1e-10, {}),
    (6000, 0, 18.2, 1e-10, {}),
    (16384, 2, 34.7, 1e-12, {}),
    (1000, 1, 25.0, 1e-8, {"window": "kb"}),
    (2048, 2, 30.0, 1e-7, {"kappa": 0.8}),
    (4000, 0, 7.0, 1e-7, {"apodisation": "cost"}),
    (4000, 2, 35.0, 1e-7, {"apodisation": "cost"}),
    (300, 0, 80.0, 1e-6, {}),        # large cap: full sky by the planner's rule
    (500, 2, 20.0, 1e-9, {"full_sky": True}),
]


@pytest.mark.parametrize("lmax,s,deg,eps,kw", CASES)
def test_planner_matches_oracle(lmax, s, deg, eps, kw):
    from paper_2603_17166_gb300 import plan_params

    ts = math.radians(deg)
    info, th, w, mj = plan_params(s, lmax, ts, eps, precision="fp64", **kw)
    okw = {}
    if "window" in kw:
        okw["window_kind"] = kw["window"]
    if "kappa" in kw:
        okw["kappa"] = kw["kappa"]
    if "apodisation" in kw:
        okw["eps_apo_choice"] = kw["apodisation"]
    if kw.get("full_sky"):
        P = None  # the oracle's full-sky rule: theta_max = pi, w = 1, Lmax = lmax
        assert info["full_sky"] == 1 and info["Lmax"] == lmax and info["nring"] == info["L"] + 1
        assert np.all(w == 1.0) and info["theta_max"] == math.pi
        return
    P = O.plan_params(lmax, s, eps, np.array([ts]), **okw)
    assert info["full_sky"] == int(P["full"])
    for k in ("Lmax", "L", "nring", "M", "W", "nTheta", "nphi", "r_lo", "nrows"):
        assert info[k] == P[k], (k, info[k], P[k])
    assert info["eps_apo"] == pytest.approx(P["eps_apo"], rel=1e-15, abs=0)
    assert info["theta_max"] == pytest.approx(P["theta_max"], rel=1e-15)
    assert np.array_equal(mj, P["Mj"])
    assert np.allclose(th, P["theta_j"], rtol=1e-15, atol=0)
    assert np.allclose(w, P["w_j"], rtol=0, atol=1e-12)
    assert info["recursion_triples"] == O.legendre_cost(lmax, s, P["Mj"])


def test_planner_rejects_bad_arguments():
    from paper_2603_17166_gb300 import PshtError, plan_params

    for args in ((-1, 10, 0.5, 1e-5), (2, 1, 0.5, 1e-5), (0, 10, 4.0, 1e-5), (0, 10, 0.5, 1.0)):
        with pytest.raises(PshtError):
            plan_params(*args)
