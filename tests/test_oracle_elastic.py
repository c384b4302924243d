"""Pins of the oracle's elastic (Navier-Lame) regularizer.  The paper names
elastic models without defining one; the reading taken is
S = 1/2 dt h^d sum_k [mu |B v_k|^2 + (lam + mu) (div v_k)^2], with B the
forward differences between neighbouring cell centres and div the centred
differences with mirrored ends.  The pins do not retype that formula: they
use fields on which the differences are exact (linear in the cell centres),
so the energy has a closed form by hand, and the exact reduction of the
model to mu times the diffusion regularizer when lam + mu = 0."""
import numpy as np
import pytest

from oracle import lagrangian as L
from oracle.objective import Problem, reg_operator, reg_value


def _prob(m, K, reg, mu=1.0, lam=0.0):
    return Problem(L.Grid(tuple(2 * a for a in m)), L.Grid(m), K=K, N=2, reg=reg, alpha=1.0, mu=mu, lam=lam)


def _centres(g, a):
    """Coordinate a of every cell centre, shaped like a grid array."""
    return L.cell_centres(g)[a].reshape(g.shape)


@pytest.mark.parametrize("m", [(7, 5), (6, 5, 4)])
def test_elastic_reduces_to_scaled_diffusion_when_lam_plus_mu_vanishes(m):
    """lam = -mu removes the divergence term: value and operator are mu times
    those of the diffusion regularizer (pinned by its own tests)."""
    rng = np.random.default_rng(3)
    mu = 0.7
    pe, pd = _prob(m, 2, "elastic", mu=mu, lam=-mu), _prob(m, 2, "diffusion")
    v = rng.normal(size=pe.vshape)
    assert reg_value(pe, v) == pytest.approx(mu * reg_value(pd, v), rel=1e-13)
    np.testing.assert_allclose(reg_operator(pe, v), mu * reg_operator(pd, v), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("m", [(9, 6), (8, 5, 4)])
def test_elastic_energy_of_a_stretch(m):
    """v_x = c x, the other components zero.  Forward differences along x are
    c on each of the (m_x - 1) interior faces of a line and zero along the
    other axes; the centred divergence is c at interior cells and c / 2 at
    the two end cells of a line (the mirrored ghost repeats the end value).
    With P lines along x (the product of the other cell counts):
    S = 1/2 dt h^d P [mu c^2 (m_x - 1) + (lam + mu)((m_x - 2) c^2 + 2 (c / 2)^2)]."""
    mu, lam, c = 1.3, 0.4, 0.25
    p = _prob(m, 1, "elastic", mu=mu, lam=lam)
    g = p.vgrid
    v = np.zeros(p.vshape)
    v[0, 0] = c * _centres(g, 0)
    P = int(np.prod(m[1:]))
    mx = m[0]
    want = 0.5 * p.time_weight * g.cell_volume * P * (mu * c * c * (mx - 1) +
                                                      (lam + mu) * ((mx - 2) * c * c + 2 * (c / 2) ** 2))
    assert reg_value(p, v) == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("m", [(9, 6), (8, 5, 4)])
def test_elastic_energy_of_a_shear_has_no_divergence_term(m):
    """v_x = c y: div v = d v_x / dx = 0 everywhere, whatever lam, and the
    forward differences of v_x along y are c on each of the (m_y - 1) interior
    faces of the m_x (times m_z) lines along y:
    S = 1/2 dt h^d mu c^2 (m_y - 1) m_x (m_z)."""
    mu, c = 0.9, -0.6
    want = None
    for lam in (0.0, 5.0):
        p = _prob(m, 1, "elastic", mu=mu, lam=lam)
        g = p.vgrid
        v = np.zeros(p.vshape)
        v[0, 0] = c * _centres(g, 1)
        lines = int(np.prod(m)) // m[1]
        s = reg_value(p, v)
        assert s == pytest.approx(0.5 * p.time_weight * g.cell_volume * mu * c * c * (m[1] - 1) * lines, rel=1e-12)
        want = s if want is None else want
        assert s == pytest.approx(want, rel=1e-13)


def test_elastic_operator_is_the_gradient_of_the_energy_on_a_stretch():
    """S is quadratic, S(v) = 1/2 v . A v with A = reg_operator: on the stretch
    of test_elastic_energy_of_a_stretch the quadratic form reproduces the
    closed-form energy."""
    m, mu, lam, c = (9, 6), 1.3, 0.4, 0.25
    p = _prob(m, 1, "elastic", mu=mu, lam=lam)
    g = p.vgrid
    v = np.zeros(p.vshape)
    v[0, 0] = c * _centres(g, 0)
    P, mx = m[1], m[0]
    want = 0.5 * p.time_weight * g.cell_volume * P * (mu * c * c * (mx - 1) +
                                                      (lam + mu) * ((mx - 2) * c * c + 2 * (c / 2) ** 2))
    assert 0.5 * float(np.sum(v * reg_operator(p, v))) == pytest.approx(want, rel=1e-12)
