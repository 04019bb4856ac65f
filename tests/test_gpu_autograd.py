"""The torch.autograd.Function of the pseudofermion action: forward = the
action (one solve, keeping X and Y), backward = the force kernel without a
solve.  Checked against the oracle force (FP64 1e-9, FP32 1e-5 relative),
against pf_action for the value (1e-12), and against a central finite
difference of the action along a random algebra direction (1e-6)."""
import numpy as np
import pytest

from oracle import actions, force, lattice
from oracle.poly import ChebyshevFilter
from paper_1702_00124_gb300 import synthetic

pytestmark = pytest.mark.gpu

POLY = (4, 0.05, 5.0)
K, KH = 0.125, 0.115


@pytest.fixture(scope="module", params=[(4, 4, 4, 4), (6, 4, 6, 10)], ids=["4x4x4x4", "6x4x6x10"])
def setup(request):
    from paper_1702_00124_gb300 import wdhmc
    from tests import gpu_util as gu
    dims = request.param
    U = synthetic.gauge_field(dims, 0.5, 701 + dims[3])
    phi = lattice.mask(synthetic.spinor_field(dims, 702 + dims[3]), dims, 0)
    lat = wdhmc.Lattice(dims)
    Ud = gu.dev(U)
    lat.wd_gauge_load(Ud)
    yield dict(dims=dims, U=U, Ud=Ud, phi=phi, lat=lat, gu=gu, wd=wdhmc)
    lat.close()


def _terms(wd):
    pf = ChebyshevFilter(*POLY)
    return {"plain": (wd.term(wd.PLAIN, K), actions.term("plain", K)),
            "hasenbusch": (wd.term(wd.HASENBUSCH, K, KH), actions.term("hasenbusch", K, KH)),
            "poly": (wd.term(wd.POLY, KH, poly=POLY), actions.term("poly", KH, poly=pf)),
            "filtered": (wd.term(wd.FILTERED, KH, poly=POLY), actions.term("filtered", KH, poly=pf))}


@pytest.mark.parametrize("name", ["plain", "hasenbusch", "poly", "filtered"])
def test_autograd_force(setup, name):
    import torch
    from paper_1702_00124_gb300.autograd import pf_action
    s = setup
    lat, gu, wd = s["lat"], s["gu"], s["wd"]
    tg, to = _terms(wd)[name]
    phi = gu.pack(lat, s["phi"], 0)
    F_ref = force.fermion_force(s["U"], to, s["phi"])
    p = wd.cg_params(tol=1e-13)
    for prec, tol in ((wd.F64, 1e-9), (wd.F32, 1e-5)):
        w = torch.zeros(64 * lat.Vh, dtype=torch.float64, device="cuda", requires_grad=True)
        S = pf_action(w, lat, tg, phi, p, prec)
        assert abs(float(S) - lat.pf_action(tg, phi, p)) < 1e-12 * abs(float(S))
        S.backward()
        err = np.linalg.norm(gu.alg_to_host(lat, w.grad.detach()) - F_ref) / np.linalg.norm(F_ref)
        assert err < tol, (prec, err)
    # chain rule: d(3 S)/dw = 3 F
    w = torch.zeros(64 * lat.Vh, dtype=torch.float64, device="cuda", requires_grad=True)
    (3.0 * pf_action(w, lat, tg, phi, p)).backward()
    assert np.linalg.norm(gu.alg_to_host(lat, w.grad.detach()) - 3 * F_ref) < 1e-9 * 3 * np.linalg.norm(F_ref)


def test_autograd_directional_fd(setup):
    import torch
    from paper_1702_00124_gb300.autograd import pf_action
    s = setup
    lat, gu, wd = s["lat"], s["gu"], s["wd"]
    tg, _ = _terms(wd)["hasenbusch"]
    phi = gu.pack(lat, s["phi"], 0)
    p = wd.cg_params(tol=1e-13)
    w = torch.zeros(64 * lat.Vh, dtype=torch.float64, device="cuda", requires_grad=True)
    pf_action(w, lat, tg, phi, p).backward()
    Om = lat.algebra_field()
    lat.gaussian_draw(1, 0, 5, 6, Om)
    deriv = float(torch.dot(w.grad, Om))
    h = 1e-5
    S = []
    for sg in (+1, -1):
        lat.wd_gauge_load(s["Ud"])
        lat.step_T(Om, sg * h)
        S.append(lat.pf_action(tg, phi, p))
    lat.wd_gauge_load(s["Ud"])
    fd = (S[0] - S[1]) / (2 * h)
    assert abs(fd - deriv) < 1e-6 * abs(fd)


def test_autograd_rejects_nonzero_point(setup):
    import torch
    from paper_1702_00124_gb300.autograd import pf_action
    s = setup
    lat, gu, wd = s["lat"], s["gu"], s["wd"]
    w = torch.ones(64 * lat.Vh, dtype=torch.float64, device="cuda", requires_grad=True)
    with pytest.raises(ValueError):
        pf_action(w, lat, _terms(wd)["plain"][0], gu.pack(lat, s["phi"], 0), wd.cg_params())
