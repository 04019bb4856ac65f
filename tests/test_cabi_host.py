"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every function include/wdhmc.h declares, and its host-only logic
(integrator schedules, Metropolis test, argument checks) matches the oracle
and the schedule printed in Section 3.2 of the paper."""
import os
import re
from fractions import Fraction

import numpy as np
import pytest

from oracle import hmc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def wd():
    from paper_1702_00124_gb300 import _build
    _build.build()
    from paper_1702_00124_gb300 import wdhmc
    return wdhmc


def _declared():
    src = open(os.path.join(ROOT, "include", "wdhmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(wd):
    names = _declared()
    assert len(names) >= 30
    for n in names:
        assert hasattr(wd.lib, n), n
    assert set(wd.EXPORTED) == set(names)


def _golden():
    ops = []
    for line in open(os.path.join(ROOT, "tests", "golden", "generalised_scheme_example.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        ops.append((0, 0, float(Fraction(f[1]))) if f[0] == "T" else (1, int(f[1]), float(Fraction(f[2]))))
    return ops


def test_generalised_schedule_printed_example(wd):
    ops = wd.wd_schedule_generalised(0, 1.0, [1, 2], [2, 3])
    want = _golden()
    assert len(ops) == len(want)
    for a, b in zip(ops, want):
        assert a[0] == b[0] and (a[0] == 0 or a[1] == b[1]) and abs(a[2] - b[2]) < 1e-14


def _canon(ops):
    """Sum the S steps of each group between consecutive T steps."""
    out, run = [], {}
    for o in ops:
        if o[0] in ("T", 0):
            if run:
                out.append(("S", tuple(sorted(run.items()))))
                run = {}
            out.append(("T", round(o[-1], 14)))
        else:
            run[o[1]] = round(run.get(o[1], 0.0) + o[2], 14)
    if run:
        out.append(("S", tuple(sorted(run.items()))))
    return out


@pytest.mark.parametrize("kind", [0, 1])
def test_nested_schedule_matches_oracle(wd, kind):
    levels = [(0, 3), (1, 2), (-1, 4)]
    g = wd.wd_schedule_nested(kind, 1.0, [a for a, _ in levels], [b for _, b in levels])
    o = hmc.nested(levels, 1.0, "leapfrog" if kind == 0 else "omelyan")
    cg_, co = _canon(g), _canon(o)
    assert len(cg_) == len(co)
    for a, b in zip(cg_, co):
        assert a[0] == b[0]
        if a[0] == "T":
            assert abs(a[1] - b[1]) < 1e-13
        else:
            assert [k for k, _ in a[1]] == [k for k, _ in b[1]]
            assert all(abs(x - y) < 1e-13 for (_, x), (_, y) in zip(a[1], b[1]))
    assert abs(sum(op[2] for op in g if op[0] == 0) - 1.0) < 1e-13


def test_metropolis_host(wd):
    assert wd.metropolis(-1.0, 0.99)
    assert not wd.metropolis(0.5, 0.61)
    assert wd.metropolis(0.5, 0.60)
    with pytest.raises(wd.WdError):
        wd.metropolis(0.1, 1.5)


def test_metropolis_from_seed_and_counter(wd):
    """u of the (seed, counter) form is the oracle's Philox4x64-10 draw
    (first word of counter (counter, 2^63, 0, 0) under key (seed, 0)), bit for
    bit, and the decision is u < exp(-dH)."""
    from oracle import philox
    rng = np.random.default_rng(5)
    for seed, counter in [(0, 0), (170200124, 7), (2**64 - 1, 2**63 + 5)] + \
            [(int(a), int(b)) for a, b in rng.integers(0, 2**63, size=(6, 2), dtype=np.int64)]:
        x0 = philox.philox4x64_10(counter, 2**63, 0, 0, seed, 0)[0]
        u_ref = (float(int(x0) >> 11) + 0.5) * 2.0**-53
        for dH in (-0.3, 0.0, 0.7, 5.0):
            acc, u = wd.metropolis_philox(dH, seed, counter)
            assert u == u_ref
            assert acc == (u_ref < np.exp(-dH))


def test_cost_matches_oracle(wd):
    """wd_cost (C = N_mat / P_acc, Section 3.1) against the oracle's definition on
    seeded trajectory records, and its argument checks."""
    import math
    from oracle.cost import cost
    rng = np.random.default_rng(11)
    for n in (1, 2, 37, 500):
        nm = rng.integers(1000, 50000, n)
        dH = rng.normal(0.3, 0.8, n)
        acc = (rng.random(n) < np.minimum(1, np.exp(-dH))).astype(int)
        got, want = wd.wd_cost(nm, acc, dH), cost(nm, acc, dH)
        for k, v in want.items():
            if math.isinf(v):
                assert math.isinf(got[k]), k
            else:
                assert abs(got[k] - v) <= 1e-12 * max(1.0, abs(v)), (n, k, got[k], v)
    assert math.isinf(wd.wd_cost([10, 20], [0, 0], [5.0, 6.0])["C"])
    for bad in (([1], [2], [0.0]), ([-1], [1], [0.0]), ([1], [1], [float("nan")]), ([], [], [])):
        with pytest.raises(wd.WdError):
            wd.wd_cost(*bad)


def test_schedule_argument_errors(wd):
    with pytest.raises(wd.WdError) as e:
        wd.wd_schedule_nested(3, 1.0, [0], [1])
    assert e.value.code == 1
    with pytest.raises(wd.WdError):
        wd.wd_schedule_nested(0, 1.0, [0], [0])
    with pytest.raises(wd.WdError):
        wd.wd_schedule_generalised(0, -1.0, [0], [2])
