"""Pins of the boundary-element oracle (oracle/bem.py, Sec. 2.3, Eq. 11 in the DPCM
normal-field reading): the exact quasistatic polarisability of a sphere, R^3 (e2 - e1) /
(e2 + 2 e1), approached as the mesh is refined, for two media; isotropy and charge
neutrality of the sphere; the linear (e2 -> e1) and perfect-conductor limits; a prolate
spheroid approaching its depolarisation-factor closed form; the Drude sphere's dipolar
resonance at wp / sqrt(3).  A wrong sign of the self term, of Ft, of the right-hand side
or a missing tessera area fails the sphere test (as the printed form of Eq. 11 does)."""
import math

import numpy as np
import pytest

from oracle import bem as BE
from oracle import model as M
from paper_2510_12731_gb300 import structures as S

EPS2 = np.array([-2.5 + 0.3j, 5.0 + 0.0j, -1.0 + 0.5j, 1e6 + 0.0j])


def _sphere_ratio(n, radius, eps1):
    pos, nrm, area = S.sphere_mesh(n, radius)
    a, q, rel = BE.solve(pos, nrm, area, EPS2, eps1, np.eye(3), radius_ang=radius)
    rb = radius / M.BOHR_ANG
    exact = rb ** 3 * (EPS2 - eps1) / (EPS2 + 2 * eps1)
    assert rel.max() < 1e-12
    return a, q, a[:, 0, 0] / exact


@pytest.mark.parametrize("eps1", [1.0, 1.77])
def test_sphere_converges_to_the_exact_quasistatic_polarisability(eps1):
    _, _, r800 = _sphere_ratio(800, 20.0, eps1)
    a, q, r3200 = _sphere_ratio(3200, 20.0, eps1)
    e800, e3200 = np.abs(r800 - 1), np.abs(r3200 - 1)
    assert np.all(e3200 < e800)                  # refinement approaches the exact value
    assert e3200.max() < 6e-3
    # isotropy and no cross-polarisation; the induced charge sums to ~0
    assert np.abs(a[:, 1, 1] - a[:, 0, 0]).max() < 1e-5 * np.abs(a[:, 0, 0]).max()
    assert np.abs(a[:, 0, 1]).max() < 1e-5 * np.abs(a[:, 0, 0]).max()
    assert np.abs(q.sum(axis=2)).max() < 5e-3 * np.abs(q).sum(axis=2).max()


def test_linear_and_conductor_limits():
    R = 20.0
    pos, nrm, area = S.sphere_mesh(1600, R)
    rb = R / M.BOHR_ANG
    d = 1e-6
    a, _, _ = BE.solve(pos, nrm, area, np.array([1.0 + d]), 1.0, np.eye(3)[:1], radius_ang=R)
    # e2 = 1 + d: alpha = R^3 d / 3 to first order (the weak-contrast limit is mesh-exact)
    assert a[0, 0, 0] / (rb ** 3 * d / 3.0) == pytest.approx(1.0, abs=1e-5)
    a, _, _ = BE.solve(pos, nrm, area, np.array([1e9]), 1.0, np.eye(3)[:1], radius_ang=R)
    assert a[0, 0, 0].real / rb ** 3 == pytest.approx(1.0, abs=3e-3)    # perfect conductor


def test_prolate_spheroid_approaches_depolarisation_closed_form():
    """a = b = 10 A, c = 20 A: alpha_ii = V/(4 pi) (e - 1) / (1 + L_i (e - 1)) with the
    depolarisation factors L_z = (1 - e^2)/e^2 (-1 + atanh(e)/e), L_x = (1 - L_z)/2."""
    e2 = np.array([5.0 + 0.0j, -2.5 + 0.3j])
    ab, cb = 10.0 / M.BOHR_ANG, 20.0 / M.BOHR_ANG
    ecc = math.sqrt(1 - ab * ab / (cb * cb))
    Lz = (1 - ecc * ecc) / (ecc * ecc) * (-1 + math.atanh(ecc) / ecc)
    Lx = (1 - Lz) / 2
    V = 4 * math.pi / 3 * ab * ab * cb
    errs = []
    for n in (1600, 6400):
        pos, nrm, area = S.spheroid_mesh(n, 10.0, 10.0, 20.0)
        a, _, _ = BE.solve(pos, nrm, area, e2, 1.0, np.eye(3))
        az = V / (4 * math.pi) * (e2 - 1) / (1 + Lz * (e2 - 1))
        ax = V / (4 * math.pi) * (e2 - 1) / (1 + Lx * (e2 - 1))
        errs.append(np.concatenate([np.abs(a[:, 2, 2] / az - 1), np.abs(a[:, 0, 0] / ax - 1)]))
    assert np.all(errs[1] < errs[0])
    assert errs[1].max() < 0.05


def test_drude_sphere_resonance_at_wp_over_sqrt3():
    w = S.drude_sphere_mesh(1600, nfreq=27, wmin=3.40, wmax=3.53, pols=np.eye(3)[:1])
    a, _, _ = BE.solve(w.pos_ang, w.normals, w.area_ang2, w.eps2, w.eps1, w.pol_dirs,
                       radius_ang=w.radius_ang)
    peak = w.omega_ev[np.argmax(a[:, 0, 0].imag)]
    assert peak == pytest.approx(6.0 / math.sqrt(3.0), abs=0.01)


def test_f_rows_are_the_rows_of_f_matrix():
    pos, nrm, area = S.spheroid_mesh(300, 8.0, 10.0, 14.0)
    rows = [0, 17, 299]
    full = BE.f_matrix(pos, nrm, area, 14.0)
    assert np.allclose(BE.f_rows(pos, nrm, area, 14.0, rows), full[rows], rtol=1e-13, atol=0)


# ---------------------------------------------------------------- IEFPCM (Eq. 12)
def _ief_sphere(n, eps1):
    pos, nrm, area = S.sphere_mesh(n, 20.0)
    a, q, rel = BE.solve_iefpcm(pos, nrm, area, EPS2, eps1, np.eye(3), radius_ang=20.0)
    rb = 20.0 / M.BOHR_ANG
    assert rel.max() < 1e-12
    return a, q, a[:, 0, 0] / (rb ** 3 * (EPS2 - eps1) / (EPS2 + 2 * eps1))


@pytest.mark.parametrize("eps1", [1.0, 1.77])
def test_iefpcm_sphere_converges_to_the_exact_quasistatic_polarisability(eps1):
    _, _, r800 = _ief_sphere(800, eps1)
    a, q, r3200 = _ief_sphere(3200, eps1)
    e800, e3200 = np.abs(r800 - 1), np.abs(r3200 - 1)
    assert np.all(e3200 < 0.6 * e800)            # first-order convergence in the mesh size
    assert e3200.max() < 6e-3
    assert np.abs(a[:, 1, 1] - a[:, 0, 0]).max() < 1e-5 * np.abs(a[:, 0, 0]).max()
    assert np.abs(a[:, 0, 1]).max() < 1e-5 * np.abs(a[:, 0, 0]).max()
    assert np.abs(q.sum(axis=2)).max() < 1e-4 * np.abs(q).sum(axis=2).max()


def test_iefpcm_printed_diagonal_sign_converges_slowly():
    """The reading's negative self term of F against the printed positive one."""
    R = 20.0
    pos, nrm, area = S.sphere_mesh(3200, R)
    p, a_ = pos / M.BOHR_ANG, area / M.BOHR_ANG ** 2
    F = BE.f_matrix_ief(p, nrm, a_, R / M.BOHR_ANG)
    Fp = F.copy()
    Fp[np.diag_indices_from(Fp)] *= -1.0
    G = BE.g_matrix(p, a_)
    e2 = -2.5 + 0.3j
    lam = BE.lam(e2, 1.0)
    V = -p[:, 0]
    exact = (R / M.BOHR_ANG) ** 3 * (e2 - 1) / (e2 + 2)
    errs = []
    for FF in (F, Fp):
        y = np.linalg.solve(lam * np.eye(len(V)) + FF, -(2 * np.pi * V + FF @ V).astype(complex))
        errs.append(abs((p[:, 0] @ np.linalg.solve(G, y)) / exact - 1))
    assert errs[0] < 5e-3 < 0.1 < errs[1]


def test_iefpcm_weak_contrast_resonance_and_coulomb_matrix():
    R = 20.0
    pos, nrm, area = S.sphere_mesh(1600, R)
    rb = R / M.BOHR_ANG
    a, _, _ = BE.solve_iefpcm(pos, nrm, area, np.array([1.0 + 1e-6]), 1.0, np.eye(3)[:1],
                              radius_ang=R)
    assert a[0, 0, 0] / (rb ** 3 * 1e-6 / 3.0) == pytest.approx(1.0, abs=5e-3)
    G = BE.g_matrix(pos / M.BOHR_ANG, area / M.BOHR_ANG ** 2)
    assert np.array_equal(G, G.T) and np.linalg.eigvalsh(G).min() > 0   # Coulomb: SPD
    w = S.drude_sphere_mesh(1600, nfreq=27, wmin=3.40, wmax=3.53, pols=np.eye(3)[:1])
    a, _, _ = BE.solve_iefpcm(w.pos_ang, w.normals, w.area_ang2, w.eps2, w.eps1, w.pol_dirs,
                              radius_ang=w.radius_ang)
    assert w.omega_ev[np.argmax(a[:, 0, 0].imag)] == pytest.approx(6.0 / math.sqrt(3.0), abs=0.01)


def test_iefpcm_spheroid_approaches_depolarisation_closed_form():
    e2 = np.array([5.0 + 0.0j, -2.5 + 0.3j])
    ab, cb = 10.0 / M.BOHR_ANG, 20.0 / M.BOHR_ANG
    ecc = math.sqrt(1 - ab * ab / (cb * cb))
    Lz = (1 - ecc * ecc) / (ecc * ecc) * (-1 + math.atanh(ecc) / ecc)
    Lx = (1 - Lz) / 2
    V = 4 * math.pi / 3 * ab * ab * cb
    errs = []
    for n in (1600, 3200):
        pos, nrm, area = S.spheroid_mesh(n, 10.0, 10.0, 20.0)
        a, _, _ = BE.solve_iefpcm(pos, nrm, area, e2, 1.0, np.eye(3))
        az = V / (4 * math.pi) * (e2 - 1) / (1 + Lz * (e2 - 1))
        ax = V / (4 * math.pi) * (e2 - 1) / (1 + Lx * (e2 - 1))
        errs.append(np.concatenate([np.abs(a[:, 2, 2] / az - 1), np.abs(a[:, 0, 0] / ax - 1)]))
    assert np.all(errs[1] < errs[0])
    assert errs[1].max() < 0.12
