"""HMC steps, integrators and Metropolis test for the oracle (test
infrastructure only).

Section 2 of the paper: momenta P ~ exp(-sum tr P^2),
H = sum tr P^2 + S, steps T[eps]: (P, U) -> (P, exp(i eps P) U) and
S[eps]: (P, U) -> (P - eps F, U), and a Metropolis accept/reject test.
Section 3.2: leapfrog (S[h/2] T[h] S[h/2])^n, the nested multi-scale scheme
(outer S_1 steps, each T replaced by m inner steps of S_2), and the
generalised scheme that overlays the per-term integrators in "time".

An integrator is a list of operations ("T", eps) or ("S", g, eps) where g is
the index of a group of action terms.  The Omelyan 2MN step
S[l h] T[h/2] S[(1-2l) h] T[h/2] S[l h], l = 0.1931833275037836
(Omelyan, Mryglod, Folk 2003) is not in the paper; the full-trajectory
workload asks for it.  Consecutive S steps of one group are NOT merged here.
"""
import numpy as np

from .su3 import alg_to_matrix, expm, reunitarize

OMELYAN_LAMBDA = 0.1931833275037836


def step_T(U, P, eps):
    """U <- exp(i eps P) U, reunitarised."""
    X = 1j * eps * alg_to_matrix(P, U.dtype)
    return reunitarize(expm(X) @ U)


def step_S(P, F, eps):
    return P - eps * F


def kinetic(P):
    """sum tr P^2 = (1/2) sum_a P_a^2 (tr T_a T_b = delta_ab / 2)."""
    return 0.5 * float(np.sum(P.astype(np.float64) ** 2))


def leapfrog(n, tau, g):
    h = tau / n
    return [op for _ in range(n) for op in (("S", g, h / 2), ("T", h), ("S", g, h / 2))]


def omelyan(n, tau, g, lam=OMELYAN_LAMBDA):
    h = tau / n
    return [op for _ in range(n) for op in
            (("S", g, lam * h), ("T", h / 2), ("S", g, (1 - 2 * lam) * h), ("T", h / 2),
             ("S", g, lam * h))]


def merge_adjacent(ops):
    """Join consecutive S steps of one group (S_g[a] S_g[b] = S_g[a+b], as in the
    printed two-step leapfrog I_1 of Section 3.2)."""
    out = []
    for op in ops:
        if out and op[0] == "S" and out[-1][0] == "S" and out[-1][1] == op[1]:
            out[-1] = ("S", op[1], out[-1][2] + op[2])
        else:
            out.append(op)
    return out


def nested(levels, tau, kind="leapfrog"):
    """levels = [(group, n_steps), ...], outermost first; each T of one level is
    replaced by n_steps steps of the next level over that T's length."""
    make = leapfrog if kind == "leapfrog" else omelyan
    g, n = levels[0]
    ops = make(n, tau, g)
    if len(levels) == 1:
        return ops
    out = []
    for op in ops:
        if op[0] == "T":
            out += nested(levels[1:], op[1], kind)
        else:
            out.append(op)
    return out


def generalised(schemes, tau):
    """Overlay per-group integrators (Section 3.2): each S event sits at the time
    t reached by the T steps before it in its own scheme; events are merged by
    t with T steps between distinct times.  Ties: ascending group index for
    t < tau/2, descending otherwise (reading that reproduces the printed
    example and keeps the result symmetric)."""
    events = []
    for gi, ops in enumerate(schemes):
        t = 0.0
        for op in ops:
            if op[0] == "T":
                t += op[1]
            else:
                events.append((t, gi, op))
    times = sorted({round(e[0] / tau, 12) for e in events})
    out = []
    prev = 0.0
    for tt in times:
        t = tt * tau
        if t - prev > 1e-12 * tau:
            out.append(("T", t - prev))
        evs = [e for e in events if abs(e[0] - t) <= 1e-12 * tau]
        evs.sort(key=lambda e: e[1], reverse=(t >= tau / 2 - 1e-12 * tau))
        out += [e[2] for e in evs]
        prev = t
    if tau - prev > 1e-12 * tau:
        out.append(("T", tau - prev))
    return out


def integrate(U, P, ops, force_of_group):
    """Run an operation list; force_of_group(g, U) returns the force of group g."""
    for op in ops:
        if op[0] == "T":
            U = step_T(U, P, op[1])
        else:
            P = step_S(P, force_of_group(op[1], U), op[2])
    return U, P


def metropolis(dH, u):
    """Accept iff u < exp(-dH), u uniform in [0, 1)."""
    return bool(u < np.exp(-dH))
