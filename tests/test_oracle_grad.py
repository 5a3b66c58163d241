"""Pins of oracle.grad (discrete adjoint of the compliance): exact identities of
2D linear elasticity and central finite differences of the same model."""
import numpy as np
import pytest

import lattice_inputs as LI
from oracle import grad, rom as orom


@pytest.fixture(scope="module")
def setup():
    R = orom.train(0, 0, 3, 2, 1, 8, 0.2, 0.36, LI.lhs(12, 0.2, 0.36, seed=3))
    lat = LI.lattice(3, 2, 3, 2, seed=5, mu_mode="uniform", mu_range=(0.22, 0.34), rho=5e-4)
    c, dx, dmu, _ = grad.compliance_gradient(lat, {0: R})
    return R, lat, c, dx, dmu


def test_translation_invariance(setup):
    # moving every control point by the same vector changes nothing: sum dc/dx = 0
    _, _, c, dx, _ = setup
    assert np.abs(dx.sum(axis=0)).max() < 1e-11 * abs(c)


def test_scaling_homogeneity(setup):
    # x -> s x: K unchanged in 2D, f and u scale with s, so c is homogeneous of
    # degree 2 and sum_cp x_cp . dc/dx_cp = 2 c (Euler)
    _, lat, c, dx, _ = setup
    assert abs((dx * lat.ctrl).sum() - 2 * c) < 1e-11 * abs(c)


def test_central_finite_differences(setup):
    R, lat, c, dx, dmu = setup
    rng = np.random.default_rng(7)
    h = 1e-6
    for _ in range(3):
        vx = rng.standard_normal(lat.ctrl.shape)
        vm = rng.standard_normal(lat.mu.shape)
        lp = LI.Lattice(**{**lat.__dict__, "ctrl": lat.ctrl + h * vx, "mu": lat.mu + h * vm})
        lm = LI.Lattice(**{**lat.__dict__, "ctrl": lat.ctrl - h * vx, "mu": lat.mu - h * vm})
        fd = (grad.compliance(lp, {0: R}) - grad.compliance(lm, {0: R})) / (2 * h)
        an = (dx * vx).sum() + (dmu * vm).sum()
        assert abs(fd - an) <= 1e-6 * abs(an)


def test_compliance_matches_direct_solve(setup):
    R, lat, c, _, _ = setup
    assert abs(grad.compliance(lat, {0: R}) - c) < 1e-10 * abs(c)
