"""HMC exactness of the oracle's method reading (Section 2), CPU only.

For a reversible, area-preserving integrator with momenta drawn from exp(-sum tr P^2)
and pseudofermions from exp(-S_F) (phi from Gaussian chi with density
exp(-chi^dag chi)), every trajectory from an equilibrated field satisfies
<exp(-dH)> = 1 whatever the step size.  Checked on 2^3 x 4 with one plain term and
the gauge action; a noise of the wrong variance, a heat bath of the wrong
distribution, a force inconsistent with its action or an irreversible schedule
moves the mean far outside the statistical error."""
import numpy as np
import pytest

from oracle import actions, force, hmc, lattice
from paper_1702_00124_gb300 import synthetic


@pytest.mark.slow
def test_exp_minus_dH_is_one():
    dims, beta, kappa = (2, 2, 2, 4), 5.6, 0.12
    rng = np.random.default_rng(2017)
    U = synthetic.gauge_field(dims, 0.5, 3)
    term = actions.term("plain", kappa)
    ops = hmc.nested([(0, 3), (-1, 2)], 1.0, "leapfrog")
    shp = lattice.shape(dims)

    def trajectory(U):
        P0 = rng.standard_normal(shp + (4, 8))                    # exp(-sum tr P^2)
        chi = (rng.standard_normal(shp + (4, 3)) + 1j * rng.standard_normal(shp + (4, 3))) / np.sqrt(2)
        phi = actions.heatbath(U, term, lattice.mask(chi, dims, 0))

        def H(V, P):
            return hmc.kinetic(P) + force.gauge_action(V, beta) + actions.action(V, term, phi)[0]

        def fog(g, V):
            return force.gauge_force(V, beta) if g == -1 else force.fermion_force(V, term, phi)

        U1, P1 = hmc.integrate(U, P0, ops, fog)
        dH = H(U1, P1) - H(U, P0)
        return (U1 if rng.random() < np.exp(-dH) else U), dH

    for _ in range(30):                                            # thermalise
        U, _ = trajectory(U)
    x = []
    for _ in range(120):
        U, dH = trajectory(U)
        x.append(np.exp(-dH))
    x = np.array(x)
    err = x.std() / np.sqrt(x.size)
    assert abs(x.mean() - 1.0) < 4 * err + 0.02, (x.mean(), err)
