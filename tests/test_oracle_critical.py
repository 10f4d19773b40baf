"""Pins of the oracle's critical force f_c^s of a periodic L x M sample (Sec. III.B of
arXiv:1211.7275: the pinned configuration with the largest drive in the long-time dynamics).

  - L = 1 has no elasticity: a single site in a force landscape periodic in u, pinned while
    f + F_p(u) = 0 has a solution.  For the random field, linear between the nodes, that is
    f_c^s = -min_{n < M} R(n) exactly;
  - the critical configuration is static: at the largest pinned drive every velocity vanishes;
  - by no-passing f_c^s does not depend on the pinned configuration the search starts from (a
    line relaxed at f = 0.3 instead of f = 0);
  - the mean over samples lies near the short-time-dynamics threshold (Sec. IV.A: the
    thermodynamic f_c is the STD threshold; finite L and M move it).
"""
import json
import os

import numpy as np
import pytest

from qew_workloads import SEED


@pytest.mark.parametrize("s,M", [(0, 16), (1, 16), (2, 5), (3, 64)])
def test_single_site_closed_form(orc, s, M):
    r = orc.critical_force(1, M, orc.KIND_RF, SEED, s, tol=1e-5)
    R = orc.disorder_values(orc.KIND_RF, SEED, s, np.zeros(M, np.int64), np.arange(M))
    assert r["bracket"][0] <= -R.min() <= r["bracket"][1]


def test_critical_configuration_is_static(orc):
    L, M = 48, 32
    r = orc.critical_force(L, M, orc.KIND_RF, SEED, 0)
    F = orc.pinning_force(orc.KIND_RF, SEED, 0, np.arange(L), r["u_c"], period=M)
    u = r["u_c"]
    lap = np.roll(u, -1) + np.roll(u, 1) - 2 * u
    vel = lap + r["bracket"][0] + F
    assert np.max(np.abs(vel)) < 1e-9


def test_independent_of_the_start(orc):
    a = orc.critical_force(64, 64, orc.KIND_RF, SEED, 1)
    b = orc.critical_force(64, 64, orc.KIND_RF, SEED, 1, f_start=0.3)
    assert abs(a["f_c"] - b["f_c"]) <= 2e-4


def test_mean_near_the_short_time_threshold(orc):
    """8 samples of 128 x 128: the mean f_c^s within 8% of the oracle's STD threshold at L = 4096
    (finite L and M move f_c^s; Sec. IV.A takes both to infinity)."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "fc_rf_L4096.json")) as fh:
        fc_std = json.load(fh)["f_c"]
    fcs = [orc.critical_force(128, 128, orc.KIND_RF, SEED, s, tol=1e-3)["f_c"] for s in range(8)]
    assert abs(np.mean(fcs) - fc_std) < 0.08 * fc_std, (np.mean(fcs), fc_std)
