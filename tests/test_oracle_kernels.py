"""Pins for the oracle's kernels and operators (Eqs. 2-5 and the derived dipole kernels).

Each check compares the oracle with something other than itself: a finite
difference, a textbook limit, a Taylor series, a matrix property that the
equations imply, or a symmetry of the physics.
"""
import math

import numpy as np
import pytest

from oracle import model as M
from paper_2510_12731_gb300 import structures as S


def _st(xyz_ang, element="Ag"):
    el = S.ELEMENTS[element]
    return M.structure_from_types(xyz_ang, np.zeros(len(xyz_ang), dtype=int), [el.atom_type()])


# ---------------------------------------------------------------- T, T', T''

@pytest.mark.parametrize("R", [1.0, 2.7, 4.1])
@pytest.mark.parametrize("r", [0.9, 2.5, 5.46, 11.0])
def test_T_derivatives_match_central_differences(r, R):
    # fourth-order central differences of erf(r/R)/r
    h = 1e-3
    f = lambda x: math.erf(x / R) / x
    d1 = (-f(r + 2 * h) + 8 * f(r + h) - 8 * f(r - h) + f(r - 2 * h)) / (12 * h)
    d2 = (-f(r + 2 * h) + 16 * f(r + h) - 30 * f(r) + 16 * f(r - h) - f(r - 2 * h)) / (12 * h * h)
    assert M.gauss_T1(np.array(r), R) == pytest.approx(d1, rel=1e-8, abs=1e-12)
    assert M.gauss_T2(np.array(r), R) == pytest.approx(d2, rel=1e-6, abs=1e-10)


def test_T_far_field_is_coulomb():
    R = 2.0
    r = np.array([9.0 * R, 15.0 * R, 40.0 * R])
    assert np.allclose(M.gauss_T(r, R), 1.0 / r, rtol=1e-15, atol=0)
    assert np.allclose(M.gauss_T1(r, R), -1.0 / r ** 2, rtol=1e-14, atol=0)
    assert np.allclose(M.gauss_T2(r, R), 2.0 / r ** 3, rtol=1e-14, atol=0)


def test_Tqq_diagonal_is_small_r_limit():
    # Taylor: erf(x)/r = (2/(sqrt(pi) R)) (1 - x^2/3 + x^4/10 - ...)
    xyz = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 0.0]])
    st = _st(xyz)
    T = M.tqq(st)
    Rii = math.sqrt(2.0) * st.Rq[0]
    for eps in (1e-3, 1e-4):
        val = math.erf(eps / Rii) / eps
        x = eps / Rii
        taylor = 2.0 / (math.sqrt(math.pi) * Rii) * (1 - x * x / 3 + x ** 4 / 10)
        assert val == pytest.approx(taylor, rel=1e-12)
    assert T[0, 0] == pytest.approx(2.0 / (math.sqrt(math.pi) * Rii), rel=1e-15)


def test_dipole_kernels_are_gradients_of_Tqq():
    """T^qmu_ij = d/dr_j T^qq(r_i - r_j) and T^mumu_ij = -d2/dr_i dr_j... checked by
    finite differences of the oracle's own charge kernel on displaced atoms."""
    rng = np.random.default_rng(7)
    xyz = np.array([[0.0, 0.0, 0.0], [2.7, 0.6, -0.4], [-1.1, 2.9, 1.3]])
    st = _st(xyz)
    st.Rmu = st.Rq.copy()          # same width so Tqq of displaced atoms is the parent kernel
    Tqmu = M.tqmu(st)
    Tmuq = M.tmuq(st)
    Tmumu = M.tmumu(st)
    h = 1e-5

    def tq(pos_i, pos_j, Ri, Rj):
        r = np.linalg.norm(pos_i - pos_j)
        return math.erf(r / math.sqrt(Ri ** 2 + Rj ** 2)) / r

    for i in range(3):
        for j in range(3):
            if i == j:
                continue
            for a in range(3):
                e = np.eye(3)[a] * h
                # potential at i of a unit dipole at j along a: d/d r_j,a of T(r_i - r_j)
                num = (tq(st.pos[i], st.pos[j] + e, st.Rq[i], st.Rmu[j])
                       - tq(st.pos[i], st.pos[j] - e, st.Rq[i], st.Rmu[j])) / (2 * h)
                assert Tqmu[i, j, a] == pytest.approx(num, rel=1e-7, abs=1e-11)
                num2 = (tq(st.pos[i] + e, st.pos[j], st.Rmu[i], st.Rq[j])
                        - tq(st.pos[i] - e, st.pos[j], st.Rmu[i], st.Rq[j])) / (2 * h)
                assert Tmuq[i, a, j] == pytest.approx(num2, rel=1e-7, abs=1e-11)
                for b in range(3):
                    eb = np.eye(3)[b] * 1e-4
                    # -d/dr_i,a d/dr_j,b ... = +d/dr_i,a d/dr_i,b (T depends on r_i - r_j)
                    g = lambda p: tq(p, st.pos[j], st.Rmu[i], st.Rmu[j])
                    hh = 1e-4
                    ea = np.eye(3)[a] * hh
                    d2 = (g(st.pos[i] + ea + eb) - g(st.pos[i] + ea - eb)
                          - g(st.pos[i] - ea + eb) + g(st.pos[i] - ea - eb)) / (4 * hh * hh)
                    assert Tmumu[i, a, j, b] == pytest.approx(-d2, rel=2e-5, abs=1e-9)


def test_dipole_kernel_far_field():
    # far apart: T^qmu -> rhat / r^2 ... (potential of a point dipole), T^mumu -> (I - 3 rr)/r^3
    xyz = np.array([[0.0, 0.0, 0.0], [30.0, 20.0, -10.0]])
    st = _st(xyz)
    rij = st.pos[0] - st.pos[1]
    r = np.linalg.norm(rij)
    rhat = rij / r
    assert np.allclose(M.tqmu(st)[0, 1], rhat / r ** 2, rtol=1e-13, atol=0)
    assert np.allclose(M.tmumu(st)[0, :, 1, :], (np.eye(3) - 3 * np.outer(rhat, rhat)) / r ** 3,
                       rtol=1e-12, atol=1e-20)


def test_full_T_is_symmetric_and_Tqmu_is_Tmuq_transposed():
    xyz = S.sphere("fcc", 4.09, 5.0)
    st = _st(xyz)
    st.Rmu = st.Rmu * 1.3          # different widths: symmetry must still hold
    T4 = M.t_full(st)
    assert np.array_equal(T4, T4.T)
    N = st.natoms
    assert np.array_equal(M.tqmu(st).reshape(N, 3 * N), M.tmuq(st).reshape(3 * N, N).T)


def test_Tqq_positive_definite():
    st = _st(S.sphere("fcc", 4.09, 8.0))
    T = M.tqq(st)
    assert np.array_equal(T, T.T)
    np.linalg.cholesky(T)          # raises if not positive definite


# ---------------------------------------------------------------- K, Kbar

def test_fermi_midpoint_and_cutoff():
    r0, d, s = 5.0, 12.0, 1.1
    assert M.fermi(s * r0, r0, d, s) == pytest.approx(0.5, abs=1e-15)
    rc = M.cutoff_radius(r0, d, s, 1e-6)
    assert 1.0 - M.fermi(rc, r0, d, s) == pytest.approx(1e-6, rel=1e-9)
    assert rc / r0 == pytest.approx(2.3660, abs=1e-3)


def test_Kbar_rows_sum_to_zero_symmetric_nsd():
    st = _st(S.sphere("fcc", 4.09, 9.0))
    K = M.conductance_K(st)
    Kb = M.kbar(K)
    assert np.all(np.diag(K) == 0)
    assert np.abs(Kb.sum(axis=1)).max() <= 1e-14 * np.abs(Kb).max()
    assert np.array_equal(K, K.T)
    assert np.linalg.eigvalsh(Kb).max() <= 1e-12 * np.abs(Kb).max()


def test_neighbour_counts_of_bulk_atoms():
    # kept shells for eps = 1e-6 (r_cut = 2.366 r0): fcc 12+6+24+12+24 = 78, bcc 64, honeycomb 12
    for element, xyz, expected in [
        ("Ag", S.sphere("fcc", 4.09, 14.0), 78),
        ("Na", S.sphere("bcc", 4.23, 16.0), 64),
        ("C", S.honeycomb_disk(1.42, 30.0), 12),
    ]:
        st = _st(xyz, element)
        K = M.conductance_K(st)
        i0 = int(np.argmin(np.linalg.norm(st.pos, axis=1)))
        assert np.count_nonzero(K[i0]) == expected, element


def test_K_value_matches_eq3():
    xyz = np.array([[0.0, 0.0, 0.0], [2.892, 0.0, 0.0]])
    st = _st(xyz)
    K = M.conductance_K(st)
    r = 2.892 / M.BOHR_ANG
    r0 = st.r0[0]
    f = 1.0 / (1.0 + math.exp(-12.0 * (r / (1.1 * r0) - 1.0)))
    assert K[0, 1] == pytest.approx((1 - f) * st.area[0] / r, rel=1e-14)


def test_area_literals_match_calibration():
    from oracle import calibrate
    got = calibrate.preset_areas()
    for k, v in got.items():
        assert S.ELEMENTS[k].atom_type()["area_bohr2"] == pytest.approx(v, rel=1e-12)
