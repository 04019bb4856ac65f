"""Cost of an HMC action for the oracle (test infrastructure only).

Section 3.1 of the paper measures an action by C = N_mat / P_acc: N_mat the
multiplications by K of one trajectory, P_acc the Metropolis acceptance rate,
both averaged over the trajectories of a run.  The companion quantities are
the smoother acceptance estimator <min(1, exp(-dH))>, whose expectation is
P_acc because the test accepts with probability min(1, exp(-dH)), and
<exp(-dH)>, which is 1 at equilibrium for a reversible, area-preserving
integrator.  Written as plain definitions; pinned in tests/test_oracle_cost.py
by closed forms (all or no trajectories accepted) and by the Gaussian-dH
identities <exp(-dH)> = 1 and P_acc = erfc(sqrt(mu) / 2) for dH ~ N(mu, 2 mu).
"""
import math


def cost(n_mat, accepted, dH):
    n = len(n_mat)
    assert n >= 1 and len(accepted) == n and len(dH) == n
    mean_nmat = sum(float(v) for v in n_mat) / n
    p_acc = sum(int(a) for a in accepted) / n
    x = [math.exp(-float(d)) for d in dH]
    p_acc_est = sum(min(1.0, v) for v in x) / n
    exp_mdH = sum(x) / n
    if n > 1:
        var = sum((v - exp_mdH) ** 2 for v in x) / (n - 1)
        err = math.sqrt(var / n)
    else:
        err = 0.0
    C = mean_nmat / p_acc if p_acc > 0 else math.inf
    C_est = mean_nmat / p_acc_est if p_acc_est > 0 else math.inf
    return {"C": C, "p_acc": p_acc, "p_acc_est": p_acc_est, "mean_nmat": mean_nmat,
            "exp_mdH": exp_mdH, "exp_mdH_err": err, "C_est": C_est}
