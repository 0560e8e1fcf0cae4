"""Energy balance pins the oracle's absorption cross-sections (Sec. "Observables").

A structure driven by the uniform field E0 e at frequency w (amplitudes with the
e^{-iwt} convention, time averages 1/2 Re[a conj(b)]) takes from the field the
power <E(t) . d'(t)> = (w/2) E0^2 Im(e . alpha e) and dissipates the same power:

  * The charge rows of Eq. 1 / Eq. 7 read Kbar phi = z_q q, with phi = V + (T x)_q the
    total potential at the atoms.  With z_q of Eq. 6 this is the Drude bond current
    -i w q_i = D sum_j K_ij (phi_j - phi_i), D = 2 n tau / (1 - i w tau), so the bond
    network loses 1/2 Re(D) sum_{i<j} K_ij |phi_i - phi_j|^2 (Joule heat).
  * The dipole rows of Eq. 7 read mu_i = alpha^IB E_loc,i with E_loc,i = E - (T x)_mu,i,
    the local field; a dipole driven by E_loc absorbs (w/2) Im(alpha^IB) |E_loc,i|^2
    (the interband loss, Eq. 8).
  * The electrostatic energy 1/2 x^T T x is reactive (T symmetric): zero mean power.

Dividing the dissipated power by the incident intensity c E0^2 / (8 pi) gives the
absorption cross-section of the field direction e.  The tests below compute it from
the solved charges, dipoles and potentials through the losses only -- never from
alpha -- and compare with the oracle's sigma_abs_pol, and their mean over x, y, z with
the orientation average 4 pi w / (3c) Tr Im alpha.  A wrong 4 pi, 3, c or E0 factor,
or Re instead of Im of alpha, fails them.
"""
import numpy as np
import pytest

from oracle import hetero as H
from oracle import model as M
from paper_2510_12731_gb300 import structures as S

XYZ = np.eye(3)


def _dissipated_sigma(st, model, omega_au, e_dir, e0, q, mu=None, alpha_ib=None, kcut_eps=1e-6):
    """Absorption cross-section from the bond (and dipole) losses of one solved column."""
    N = st.natoms
    K = M.conductance_K(st, kcut_eps)
    assert np.allclose(K, K.T)            # uniform A: every bond carries one current
    if model == "wfq":
        phi = M.potential_V(st, e_dir, e0) + M.tqq(st) @ q
        p_dip = 0.0
    else:
        x = np.concatenate([q, mu.reshape(-1)])
        tx = M.t_full(st) @ x
        phi = M.potential_V(st, e_dir, e0) + tx[:N]
        e_loc = np.tile(e0 * np.asarray(e_dir, dtype=np.float64), N) - tx[N:]
        p_dip = 0.5 * omega_au * alpha_ib.imag * np.sum(np.abs(e_loc) ** 2)
    D = 2.0 * st.n * st.tau / (1.0 - 1j * omega_au * st.tau)
    dphi2 = np.abs(phi[:, None] - phi[None, :]) ** 2
    p_joule = 0.5 * D.real * 0.5 * np.sum(K * dphi2)     # sum over i < j of a symmetric sum
    return 8.0 * np.pi * (p_joule + p_dip) / (M.C_AU * e0 * e0)


@pytest.mark.parametrize("element,radius", [("Na", 8.0), ("Ag", 7.0)])
def test_wfq_absorption_equals_joule_loss(element, radius):
    w = S.small_cluster(element=element, radius=radius, model="wfq", nfreq=5, wmin=1.5, wmax=6.0)
    st = M.structure_from_types(w.xyz_ang, w.type_idx, w.types)
    e0 = 0.37
    res = M.solve(st, "wfq", w.omega_ev, XYZ, e0=e0)
    omega = w.omega_ev / M.HARTREE_EV
    for f, wf in enumerate(omega):
        sig = [_dissipated_sigma(st, "wfq", wf, XYZ[p], e0, res.q[f, p]) for p in range(3)]
        for p in range(3):
            assert res.sigma_abs_pol[f, p] == pytest.approx(sig[p], rel=1e-9)
        avg = M.sigma_abs(wf, np.trace(res.alpha[f]).imag)
        assert avg == pytest.approx(np.mean(sig), rel=1e-9)
        assert min(sig) > 0.0


def test_wfqfmu_absorption_equals_joule_plus_interband_loss():
    w = S.small_cluster(element="Ag", radius=6.0, model="wfqfmu", nfreq=4, wmin=2.5, wmax=5.5)
    st = M.structure_from_types(w.xyz_ang, w.type_idx, w.types)
    e0 = 1.9
    res = M.solve(st, "wfqfmu", w.omega_ev, XYZ, alpha_ib=w.alpha_ib, e0=e0)
    omega = w.omega_ev / M.HARTREE_EV
    for f, wf in enumerate(omega):
        aib = w.alpha_ib[0, f]
        sig = [_dissipated_sigma(st, "wfqfmu", wf, XYZ[p], e0, res.q[f, p], res.mu[f, p], aib)
               for p in range(3)]
        for p in range(3):
            assert res.sigma_abs_pol[f, p] == pytest.approx(sig[p], rel=1e-9)
        assert M.sigma_abs(wf, np.trace(res.alpha[f]).imag) == pytest.approx(np.mean(sig), rel=1e-9)


def test_rotated_field_triple_gives_the_same_orientation_average():
    """Tr Im alpha does not depend on the orthonormal triple used to measure it; the
    per-direction cross-sections of a rotated triple still balance their losses."""
    w = S.small_cluster(element="Ag", radius=7.0, model="wfq", nfreq=3, wmin=3.0, wmax=5.5)
    st = M.structure_from_types(w.xyz_ang, w.type_idx, w.types)
    a, b = 0.7, -0.4
    Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, np.cos(b), -np.sin(b)], [0, np.sin(b), np.cos(b)]])
    E = (Rz @ Rx).T                        # rows: three orthonormal field directions
    res = M.solve(st, "wfq", w.omega_ev, E)
    ref = M.solve(st, "wfq", w.omega_ev, XYZ)
    omega = w.omega_ev / M.HARTREE_EV
    for f, wf in enumerate(omega):
        sig = [_dissipated_sigma(st, "wfq", wf, E[p], 1.0, res.q[f, p]) for p in range(3)]
        assert np.allclose(res.sigma_abs_pol[f], sig, rtol=1e-9)
        assert np.mean(sig) == pytest.approx(M.sigma_abs(wf, np.trace(ref.alpha[f]).imag), rel=1e-9)


def test_eq10_hand_values():
    """Eq. 10 at neighbour counts where a weighted harmonic mean of the interband
    polarisabilities differs from an arithmetic one.  An A atom with 2 A and 3 B
    nearest neighbours, alpha_A = 2, alpha_B = 5: ((2+1)/2 + 3/5) / 6 = 0.35, so
    alpha = 1/0.35 = 20/7 (the arithmetic mean would be 3.5).  A B atom with the same
    counts: (2/2 + (3+1)/5) / 6 = 0.3, alpha = 10/3.  Complex case, an A atom with
    N_A = 0, N_B = 1, alpha_A = 1 + 1i, alpha_B = 2: (1/(1+1i) + 1/2) / 2 = (1 - 0.5i)/2,
    alpha = 2/(1 - 0.5i) = (8 + 4i)/5."""
    out = H.alpha_ib_hetero(np.array([0, 1]), np.array([[2, 3], [2, 3]]), np.array([2.0, 5.0]))
    assert out[0] == pytest.approx(20.0 / 7.0, rel=1e-15)
    assert out[1] == pytest.approx(10.0 / 3.0, rel=1e-15)
    c = H.alpha_ib_hetero(np.array([0]), np.array([[0, 1]]), np.array([1.0 + 1.0j, 2.0]))
    assert c[0] == pytest.approx((8.0 + 4.0j) / 5.0, rel=1e-15)
