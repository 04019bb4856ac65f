"""Host-side checks of the cost driver (no GPU): every action of Sections 3.1-3.3 and
4.1-4.2 is built from the right term kinds, hopping parameters and filters, outermost
term first, and its generalised schedule gives every group (and the gauge force) the
trajectory length in S steps and in T steps."""
import pytest


@pytest.fixture(scope="module")
def mods():
    from paper_1702_00124_gb300 import _build
    _build.build()
    from paper_1702_00124_gb300 import cost, wdhmc
    return cost, wdhmc


def _desc(t):
    return (t.kind, round(t.kappa, 6), round(t.kappa_h, 6), t.poly.n, t.poly_lo.n)


def test_actions(mods):
    cost, wd = mods
    k, kh, k2 = 0.15825, 0.145, 0.15
    P, P2 = (4, 0.005, 8.0), (24, 0.005, 8.0)
    want = {
        "1PF": [(wd.FILTERED, k, 0, 4, 0), (wd.POLY, k, 0, 4, 0)],
        "1MP": [(wd.HASENBUSCH, k, kh, 0, 0), (wd.PLAIN, kh, 0, 0, 0)],
        "PF-MP": [(wd.HASENBUSCH, k, kh, 0, 0), (wd.FILTERED, kh, 0, 4, 0), (wd.POLY, kh, 0, 4, 0)],
        "2PF": [(wd.FILTERED, k, 0, 24, 0), (wd.RATIO, k, 0, 24, 4), (wd.POLY, k, 0, 4, 0)],
        "2MP": [(wd.HASENBUSCH, k, k2, 0, 0), (wd.HASENBUSCH, k2, kh, 0, 0), (wd.PLAIN, kh, 0, 0, 0)],
        "1PF-2MP": [(wd.HASENBUSCH, k, k2, 0, 0), (wd.HASENBUSCH, k2, kh, 0, 0), (wd.FILTERED, kh, 0, 4, 0),
                    (wd.POLY, kh, 0, 4, 0)],
        "2PF-1MP": [(wd.HASENBUSCH, k, kh, 0, 0), (wd.FILTERED, kh, 0, 24, 0), (wd.RATIO, kh, 0, 24, 4),
                    (wd.POLY, kh, 0, 4, 0)],
    }
    assert set(want) == set(cost.ACTION_TERMS)
    for name, w in want.items():
        got = [_desc(t) for t in cost.action(name, k, kh, P, P2, kappa_2=k2)]
        assert got == [(a, round(b, 6), round(c, 6), d, e) for a, b, c, d, e in w], name
        assert len(cost.ACTION_TERMS[name]) == len(w)
    with pytest.raises(ValueError):
        cost.action("3PF", k)


@pytest.mark.parametrize("kind", [0, 1])
def test_schedule_lengths(mods, kind):
    cost, _ = mods
    ops = cost.schedule([3, 5, 7], 11, tau=0.8, kind=kind)
    assert abs(sum(e for o, g, e in ops if o == 0) - 0.8) < 1e-12
    for g in (0, 1, 2, -1):
        assert abs(sum(e for o, gg, e in ops if o == 1 and gg == g) - 0.8) < 1e-12, g
