"""P5: rough physics pin of the oracle against the paper's printed slopes.

At the finite-size critical force f_c^L (random field, L = 4096, found with the oracle alone by
``tests/golden/make_fc_rf_oracle.py`` from the decade 50 < t < 500), the relaxation from the
flat start must show the paper's mesoscopic behaviour (Sec. IV.B, Fig. 5):
  - v decays with an effective exponent of about 0.16 for 1 < t < 30 (a window the bisection
    did not use);
  - w grows with an effective exponent between about 0.67 and 0.84, i.e. w2 with 1.3 .. 1.7;
and the transition must be there: below f_c the velocity collapses, above it saturates
(Sec. III.A).  Tolerances are wide: these are effective exponents on a small system.

Case 3 (Gaussian random-bond potential, linear spline; Sec. IV.C) gets the same treatment from
its own oracle-bisected f_c^L (``tests/golden/fc_rbg_linear_L4096.json``), plus one more pin:
with N(0,1) potential values its f_c^L lands on Table I's Case 3 value, 1.565 at L = 4096, so
the amplitude, the spline and the sign of the force are checked against a printed number.
Case 1 (Gaussian potential, cubic spline) is compared with Table I more loosely, since its
spline here is the local Catmull-Rom one.
"""
import json
import os

import numpy as np
import pytest

from qew_workloads import SEED, log_spaced_steps

HERE = os.path.dirname(os.path.abspath(__file__))


def _load(name):
    with open(os.path.join(HERE, "golden", name)) as fh:
        return json.load(fh)


def _slope(t, y, lo, hi):
    sel = (t >= lo) & (t <= hi)
    return np.polyfit(np.log(t[sel]), np.log(y[sel]), 1)[0]


def _relax_around_fc(orc, fixture, kind):
    fc = _load(fixture)
    steps = log_spaced_steps(fc["n_steps"], 30, include_zero=False)
    t = steps * fc["dt"]
    out = {}
    for label, f in (("fc", fc["f_c"]), ("below", fc["f_c"] - 0.1), ("above", fc["f_c"] + 0.2)):
        r = orc.run([fc["L"]] * fc["samples"], f, fc["dt"], kind, fc["seed"], steps)
        out[label] = (r["v"].mean(axis=1), r["w2"].mean(axis=1))
    return t, out


@pytest.fixture(scope="module")
def runs(orc):
    return _relax_around_fc(orc, "fc_rf_L4096.json", orc.KIND_RF)


@pytest.fixture(scope="module")
def runs_case3(orc):
    return _relax_around_fc(orc, "fc_rbg_linear_L4096.json", orc.KIND_RBG_LINEAR)


def test_short_time_velocity_exponent(runs):
    paper = _load("paper_values.json")["effective_slopes"]
    t, out = runs
    V, _ = out["fc"]
    s = -_slope(t, V, 1, 30)
    assert abs(s - paper["v_short"]) < 0.04, s


def test_width_exponent(runs):
    paper = _load("paper_values.json")["effective_slopes"]
    t, out = runs
    _, W2 = out["fc"]
    s = _slope(t, W2, 50, 500)
    assert 2 * paper["w_short"] - 0.05 < s < 2 * paper["w_long"] + 0.05, s


def test_transition_brackets(runs):
    t, out = runs
    assert -_slope(t, out["below"][0], 50, 500) > 0.3
    assert abs(_slope(t, out["above"][0], 50, 500)) < 0.05


@pytest.mark.parametrize("name", ["rf", "rbg_linear", "rbg_cubic"])
def test_fc_fixture_provenance(name):
    fc = _load(f"fc_{name}_L4096.json")
    assert fc["_made_by"].startswith(f"tests/golden/make_fc_oracle.py {name}")
    assert fc["seed"] == SEED


def test_case3_fc_matches_table1():
    paper = _load("paper_values.json")["critical_forces"]
    fc = _load("fc_rbg_linear_L4096.json")
    assert fc["L"] == 4096
    # Table I quotes 1.565 +- 0.002; the bisection here uses 8 samples and a shorter time
    # window, so allow 1% (a wrong amplitude, spline or sign moves it by tens of percent)
    assert abs(fc["f_c"] - paper["case3_rb_gauss_linear_L4096"]) < 0.01 * paper["case3_rb_gauss_linear_L4096"]


def test_case1_fc_near_table1():
    """Case 1 here interpolates with the local Catmull-Rom cubic, not the paper's cubic spline over
    the whole periodic column (only the microscopic correlator differs, Sec. III.B), so its f_c^L
    is compared loosely: within 5% of Table I's 1.915."""
    paper = _load("paper_values.json")["critical_forces"]
    fc = _load("fc_rbg_cubic_L4096.json")
    assert abs(fc["f_c"] - paper["case1_rb_gauss_cubic_L4096"]) < 0.05 * paper["case1_rb_gauss_cubic_L4096"]


def test_case3_exponents_at_fc(runs_case3):
    t, out = runs_case3
    V, W2 = out["fc"]
    # beta / nu z: asymptotically 0.128, mesoscopic effective values up to ~0.16 (Sec. IV.B)
    assert 0.11 < -_slope(t, V, 50, 500) < 0.17
    # 2 zeta / z: between 2 x 0.67 and 2 x 0.84 in the mesoscopic regime, 1.745 asymptotically
    assert 1.3 < _slope(t, W2, 50, 500) < 1.8


def test_case3_transition_brackets(runs_case3):
    t, out = runs_case3
    assert -_slope(t, out["below"][0], 50, 500) > 0.3
    assert abs(_slope(t, out["above"][0], 50, 500)) < 0.05
