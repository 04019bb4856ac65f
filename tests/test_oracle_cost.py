"""Pins for the oracle's cost metric C = N_mat / P_acc (Section 3.1), CPU only:
closed forms (every or no trajectory accepted, a single trajectory) and, for
dH drawn from N(mu, 2 mu) (the large-volume form of the dH distribution of a
reversible, area-preserving integrator), <exp(-dH)> = 1 and
<min(1, exp(-dH))> = erfc(sqrt(mu) / 2), within five standard errors."""
import math

import numpy as np

from oracle.cost import cost


def test_closed_forms():
    r = cost([100, 300], [1, 1], [0.0, 0.0])
    assert r["C"] == 200.0 and r["p_acc"] == 1.0 and r["p_acc_est"] == 1.0 and r["exp_mdH"] == 1.0
    r = cost([100, 300, 200, 400], [1, 0, 0, 1], [0.2, 1.0, 3.0, -0.5])
    assert r["C"] == 500.0 and r["p_acc"] == 0.5
    assert abs(r["p_acc_est"] - (math.exp(-0.2) + math.exp(-1.0) + math.exp(-3.0) + 1.0) / 4) < 1e-15
    r = cost([50], [0], [2.0])
    assert math.isinf(r["C"]) and r["exp_mdH_err"] == 0.0 and abs(r["exp_mdH"] - math.exp(-2.0)) < 1e-16


def test_gaussian_dH_identities():
    rng = np.random.default_rng(7)
    for mu in (0.05, 0.5, 2.0):
        dH = rng.normal(mu, math.sqrt(2 * mu), 200_000)
        acc = (rng.random(dH.size) < np.minimum(1.0, np.exp(-dH))).astype(int)
        r = cost(np.full(dH.size, 1000), acc, dH)
        assert abs(r["exp_mdH"] - 1.0) < 5 * r["exp_mdH_err"], (mu, r)
        want = math.erfc(math.sqrt(mu) / 2)
        x = np.minimum(1.0, np.exp(-dH))
        assert abs(r["p_acc_est"] - want) < 5 * x.std() / math.sqrt(dH.size), (mu, r["p_acc_est"], want)
        assert abs(r["p_acc"] - want) < 5 * math.sqrt(want * (1 - want) / dH.size)
        assert abs(r["C"] - 1000 / r["p_acc"]) < 1e-9
