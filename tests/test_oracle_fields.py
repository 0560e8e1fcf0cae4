"""Pins of the oracle's induced density / potential / field maps (oracle/fields.py),
against mathematics the Gaussian densities fix: total charge and dipole moment by
quadrature, Gauss's law in differential form (Poisson), the field as minus the gradient
of the potential, the point-charge and point-dipole limits far away, and the
observables' dipole for a solved structure."""
import numpy as np
import pytest

from oracle import fields as FL
from oracle import model as M
from paper_2510_12731_gb300 import structures as S

RNG = np.random.default_rng(20251012)


def _two_atoms():
    pos = np.array([[-1.7, 0.4, 0.2], [2.1, -0.3, 0.9]])
    Rq = np.array([1.3, 1.6])
    Rmu = np.array([1.1, 1.4])
    q = RNG.normal(size=2) + 1j * RNG.normal(size=2)
    mu = RNG.normal(size=(2, 3)) + 1j * RNG.normal(size=(2, 3))
    return pos, Rq, Rmu, q, mu


def test_density_integrates_to_charge_and_dipole():
    pos, Rq, Rmu, q, mu = _two_atoms()
    h = 0.25
    ax = np.arange(-14.0, 14.0 + h / 2, h)
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    rho = FL.density(pos, Rq, Rmu, q, mu, pts)
    dv = h ** 3
    assert abs(rho.sum() * dv - q.sum()) < 1e-9 * abs(q).sum()
    dip = (pts * rho[:, None]).sum(axis=0) * dv
    ref = (q[:, None] * pos).sum(axis=0) + mu.sum(axis=0)
    assert np.abs(dip - ref).max() < 1e-9 * np.abs(ref).max()


def test_poisson_equation():
    """Laplacian of phi = -4 pi rho (4th-order finite differences)."""
    pos, Rq, Rmu, q, mu = _two_atoms()
    pts = RNG.uniform(-3.0, 3.0, size=(12, 3))
    h = 1e-2
    lap = np.zeros(len(pts), complex)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        f = lambda s: FL.potential(pos, Rq, Rmu, q, mu, pts + s * e)
        lap += (-f(2) + 16 * f(1) - 30 * f(0) + 16 * f(-1) - f(-2)) / (12 * h * h)
    rho = FL.density(pos, Rq, Rmu, q, mu, pts)
    assert np.allclose(lap, -4 * np.pi * rho, rtol=1e-6, atol=1e-7 * np.abs(rho).max())


def test_field_is_minus_gradient_of_potential():
    pos, Rq, Rmu, q, mu = _two_atoms()
    pts = RNG.uniform(-5.0, 5.0, size=(12, 3))
    h = 1e-3
    E = FL.field(pos, Rq, Rmu, q, mu, pts)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        f = lambda s: FL.potential(pos, Rq, Rmu, q, mu, pts + s * e)
        g = (-f(2) + 8 * f(1) - 8 * f(-1) + f(-2)) / (12 * h)
        assert np.allclose(E[:, k], -g, rtol=1e-8, atol=1e-10 * np.abs(E).max())


def test_far_away_is_point_charges_and_dipoles():
    """Beyond ~6 widths erf = 1: phi and E of point charges and point dipoles."""
    pos, Rq, Rmu, q, mu = _two_atoms()
    pts = np.array([[40.0, 3.0, -2.0], [-5.0, 35.0, 12.0], [0.0, 0.0, -60.0]])
    phi = FL.potential(pos, Rq, Rmu, q, mu, pts)
    E = FL.field(pos, Rq, Rmu, q, mu, pts)
    phi_ref = np.zeros(len(pts), complex)
    E_ref = np.zeros((len(pts), 3), complex)
    for i in range(2):
        x = pts - pos[i]
        r = np.linalg.norm(x, axis=1)
        phi_ref += q[i] / r + (x @ mu[i]) / r ** 3
        E_ref += q[i] * x / r[:, None] ** 3
        E_ref += (3 * (x @ mu[i])[:, None] * x / r[:, None] ** 2 - mu[i][None, :]) / r[:, None] ** 3
    assert np.allclose(phi, phi_ref, rtol=1e-12, atol=0)
    assert np.allclose(E, E_ref, rtol=1e-11, atol=1e-14 * np.abs(E_ref).max())


def test_potential_at_a_centre_is_the_self_limit():
    """At a charge's own centre G(0) = 2 / (sqrt(pi) R) (the limit of erf(r/R)/r);
    a dipole contributes nothing there (odd density)."""
    pos = np.zeros((1, 3))
    q = np.array([0.7 - 0.2j])
    mu = np.array([[0.3, -0.1, 0.5]], dtype=complex)
    phi0 = FL.potential(pos, np.array([1.5]), np.array([1.2]), q, mu, pos)
    phi_eps = FL.potential(pos, np.array([1.5]), np.array([1.2]), q, None, np.array([[1e-6, 0, 0]]))
    assert phi0[0] == pytest.approx(q[0] * 2 / (np.sqrt(np.pi) * 1.5), rel=1e-14)
    assert phi_eps[0] == pytest.approx(phi0[0], rel=1e-10)


def test_far_field_of_a_solved_structure_is_its_polarisability():
    """For a solved wFQFmu structure the induced potential far away is d . r / r^3 with
    d = alpha E0 (Sec. "Observables"), and the total induced charge vanishes."""
    w = S.small_cluster(element="Ag", radius=6.0, model="wfqfmu", nfreq=2, wmin=3.0, wmax=4.0)
    st = M.structure_from_types(w.xyz_ang, w.type_idx, w.types)
    res = M.solve(st, "wfqfmu", w.omega_ev, w.pol_dirs, alpha_ib=w.alpha_ib)
    f, p = 1, 0
    q, mu = res.q[f, p], res.mu[f, p]
    assert abs(q.sum()) < 1e-10 * np.abs(q).sum()
    d = res.alpha[f, :, p]       # E0 = 1
    u = np.array([0.3, -0.5, 0.81])
    u /= np.linalg.norm(u)
    pts = np.array([600.0 * u])
    phi = FL.potential(st.pos, st.Rq, st.Rmu, q, mu, pts)[0]
    assert phi == pytest.approx((d @ u) / 600.0 ** 2, rel=1e-4)
