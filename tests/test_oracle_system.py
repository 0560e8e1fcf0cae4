"""Pins for the oracle's assembled systems (Eq. 1, Eq. 7), its LU solve and observables.

Closed forms derived by hand from the equations for one, two and three atoms;
invariants the equations imply (charge conservation, reciprocity, passivity,
translation/rotation covariance); the static perfect-conductor limit; an
independent exact route (spectral); and the physical trend of the plasmon peak
toward the quasistatic Drude-sphere limit omega_p / sqrt(3).
"""
import math

import numpy as np
import pytest

from oracle import model as M
from oracle import spectral as SP
from paper_2510_12731_gb300 import structures as S

XYZ = np.eye(3)


def _st(xyz_ang, element="Ag", **over):
    el = S.ELEMENTS[element]
    t = el.atom_type()
    t.update(over)
    return M.structure_from_types(xyz_ang, np.zeros(len(xyz_ang), dtype=int), [t]), el


def _fd1(f, r, h=1e-3):
    return (-f(r + 2 * h) + 8 * f(r + h) - 8 * f(r - h) + f(r - 2 * h)) / (12 * h)


def _fd2(f, r, h=1e-3):
    return (-f(r + 2 * h) + 16 * f(r + h) - 30 * f(r) + 16 * f(r - h) - f(r - 2 * h)) / (12 * h * h)


# ------------------------------------------------------------ closed forms

@pytest.mark.parametrize("d_ang", [2.892, 3.4, 4.09])
def test_two_atom_wfq_closed_form(d_ang):
    """Atoms at -+d/2 x: q1 = -q2 reduces Eq. 1 to one equation,
    alpha_xx = k d^2 / (2 k (t0 - t1) + z_q), alpha_yy = alpha_zz = 0."""
    xyz = np.array([[-d_ang / 2, 0, 0], [d_ang / 2, 0, 0]])
    st, el = _st(xyz)
    w_ev = np.array([0.5, 2.0, 3.3, 5.0])
    res = M.solve(st, "wfq", w_ev, XYZ)
    d = d_ang / M.BOHR_ANG
    r0 = st.r0[0]
    f = 1.0 / (1.0 + math.exp(-12.0 * (d / (1.1 * r0) - 1.0)))
    k = (1.0 - f) * st.area[0] / d
    Rq = st.Rq[0]
    t0 = math.sqrt(2.0 / math.pi) / Rq
    t1 = math.erf(d / (math.sqrt(2.0) * Rq)) / d
    for i, w in enumerate(w_ev / M.HARTREE_EV):
        zq = -w * (w * st.tau + 1j) / (2.0 * st.n * st.tau)
        expect = k * d * d / (2.0 * k * (t0 - t1) + zq)
        assert res.alpha[i, 0, 0] == pytest.approx(expect, rel=1e-13)
    assert np.abs(res.alpha[:, 1:, 1:]).max() < 1e-12 * np.abs(res.alpha[:, 0, 0]).max()
    # static limit: alpha -> d^2 / (2 (t0 - t1)) > 0
    r0 = M.solve(st, "wfq", [1e-7], XYZ[:1])
    assert r0.alpha[0, 0, 0].real == pytest.approx(d * d / (2.0 * (t0 - t1)), rel=1e-9)


def test_one_atom_wfqfmu_is_interband_polarisability():
    """K = 0 for a single atom, so q = 0 and mu = alpha^IB E: alpha = alpha^IB I."""
    st, el = _st(np.zeros((1, 3)))
    w = np.linspace(2.0, 5.0, 7)
    aib = el.alpha_ib(w)[None, :]
    res = M.solve(st, "wfqfmu", w, XYZ, alpha_ib=aib)
    for f in range(len(w)):
        assert np.allclose(res.alpha[f], aib[0, f] * np.eye(3), rtol=1e-14, atol=0)
        assert np.all(res.q[f] == 0)


def test_two_atom_wfqfmu_closed_form():
    """Atoms at -+d/2 x.  Field along x: q1 = -q2 = q, mu1 = mu2 = mu x reduce Eq. 7 to
        [-2k(t0 - t1) - z_q,  -2k t1qm] [q ]   [k E0 d]
        [ t1qm,           -t2mm - z_mu] [mu] = [ E0   ],   alpha_xx = -q d + 2 mu;
    field along y: q = 0, alpha_yy = 2 / (1/alpha^IB - t1mm / d).
    The radial derivatives are taken here by finite differences of erf(r/R)/r."""
    d_ang = 2.892
    xyz = np.array([[-d_ang / 2, 0, 0], [d_ang / 2, 0, 0]])
    st, el = _st(xyz, Rmu_bohr=0.8 * S.ELEMENTS["Ag"].atom_type()["Rmu_bohr"])
    w_ev = np.array([2.5, 3.5, 4.5])
    aib = el.alpha_ib(w_ev)[None, :]
    res = M.solve(st, "wfqfmu", w_ev, XYZ, alpha_ib=aib)
    d = d_ang / M.BOHR_ANG
    Rq, Rmu = st.Rq[0], st.Rmu[0]
    f = 1.0 / (1.0 + math.exp(-12.0 * (d / (1.1 * st.r0[0]) - 1.0)))
    k = (1.0 - f) * st.area[0] / d
    t0 = math.sqrt(2.0 / math.pi) / Rq
    t1 = math.erf(d / math.sqrt(2 * Rq * Rq)) / d
    Rqm = math.sqrt(Rq * Rq + Rmu * Rmu)
    Rmm = math.sqrt(2 * Rmu * Rmu)
    t1qm = _fd1(lambda r: math.erf(r / Rqm) / r, d)
    t1mm = _fd1(lambda r: math.erf(r / Rmm) / r, d)
    t2mm = _fd2(lambda r: math.erf(r / Rmm) / r, d)
    for i, w in enumerate(w_ev / M.HARTREE_EV):
        zq = -w * (w * st.tau + 1j) / (2.0 * st.n * st.tau)
        zmu = -1.0 / aib[0, i]
        A = np.array([[-2 * k * (t0 - t1) - zq, -2 * k * t1qm], [t1qm, -t2mm - zmu]])
        q, mu = np.linalg.solve(A, np.array([k * d, 1.0]))
        assert res.alpha[i, 0, 0] == pytest.approx(-q * d + 2 * mu, rel=1e-8)
        ayy = 2.0 / (1.0 / aib[0, i] - t1mm / d)
        assert res.alpha[i, 1, 1] == pytest.approx(ayy, rel=1e-8)
        assert abs(res.alpha[i, 0, 1]) < 1e-12 * abs(res.alpha[i, 0, 0])


def test_far_apart_dipoles_reduce_to_coupled_point_dipoles():
    """Beyond the K cutoff there is no conduction (q = 0) and for separation D >> R the
    pair is two coupled point dipoles: alpha_xx = 2a/(1 - 2a/D^3), alpha_yy = 2a/(1 + a/D^3)."""
    D_ang = 60.0
    st, el = _st(np.array([[0, 0, 0], [D_ang, 0, 0]]))
    w_ev = np.array([3.0, 4.0])
    aib = el.alpha_ib(w_ev)[None, :]
    res = M.solve(st, "wfqfmu", w_ev, XYZ, alpha_ib=aib)
    D3 = (D_ang / M.BOHR_ANG) ** 3
    for i in range(2):
        a = aib[0, i]
        assert res.alpha[i, 0, 0] == pytest.approx(2 * a / (1 - 2 * a / D3), rel=1e-12)
        assert res.alpha[i, 1, 1] == pytest.approx(2 * a / (1 + a / D3), rel=1e-12)
        assert np.abs(res.q[i]).max() == 0.0


def test_far_apart_wfq_has_no_response():
    st, _ = _st(np.array([[0, 0, 0], [40.0, 0, 0], [0, 45.0, 0]]))
    res = M.solve(st, "wfq", [3.0], XYZ)
    assert np.abs(res.alpha).max() == 0.0


def _brute_matrix_wfq(st, zq, kcut_eps=1e-6):
    """Eq. 1 assembled entry by entry with scalar math (no numpy kernels)."""
    N = st.natoms
    pos = [tuple(p) for p in st.pos]
    Kf = [[0.0] * N for _ in range(N)]
    for i in range(N):
        for j in range(N):
            if i == j:
                continue
            r = math.dist(pos[i], pos[j])
            r0, d, s = st.r0[i], st.d[i], st.s[i]
            f = 1.0 / (1.0 + math.exp(-d * (r / (s * r0) - 1.0)))
            if 1.0 - f >= kcut_eps:
                Kf[i][j] = (1.0 - f) * st.area[i] / r
    Kb = [[Kf[i][j] - (sum(Kf[i]) if i == j else 0.0) for j in range(N)] for i in range(N)]
    T = [[0.0] * N for _ in range(N)]
    for i in range(N):
        for j in range(N):
            if i == j:
                T[i][j] = math.sqrt(2.0 / math.pi) / st.Rq[i]
            else:
                r = math.dist(pos[i], pos[j])
                T[i][j] = math.erf(r / math.sqrt(st.Rq[i] ** 2 + st.Rq[j] ** 2)) / r
    A = [[sum(Kb[i][k] * T[k][j] for k in range(N)) - (zq if i == j else 0.0)
          for j in range(N)] for i in range(N)]
    return A, Kb


def _det3(m):
    return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
            - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
            + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))


def test_three_atom_wfq_cramer():
    xyz = np.array([[0.0, 0.0, 0.0], [2.9, 0.3, 0.0], [1.2, 2.6, 0.4]])
    st, _ = _st(xyz)
    w_ev = 3.1
    e = np.array([0.6, 0.8, 0.0])
    res = M.solve(st, "wfq", [w_ev], [e])
    w = w_ev / M.HARTREE_EV
    zq = -w * (w * st.tau + 1j) / (2.0 * st.n * st.tau)
    A, Kb = _brute_matrix_wfq(st, zq)
    V = [-(e @ p) for p in st.pos]
    b = [-sum(Kb[i][j] * V[j] for j in range(3)) for i in range(3)]
    D = _det3(A)
    q = []
    for c in range(3):
        Ac = [[(b[i] if j == c else A[i][j]) for j in range(3)] for i in range(3)]
        q.append(_det3(Ac) / D)
    assert np.allclose(res.q[0, 0], q, rtol=1e-12, atol=1e-14 * max(abs(x) for x in q))


def _gauss_solve_longdouble(A, b):
    """Gaussian elimination with partial pivoting in extended precision (no LAPACK)."""
    n = len(b)
    M_ = [[np.clongdouble(A[i][j]) for j in range(n)] + [np.clongdouble(b[i])] for i in range(n)]
    for c in range(n):
        p = max(range(c, n), key=lambda r: abs(M_[r][c]))
        M_[c], M_[p] = M_[p], M_[c]
        for r in range(c + 1, n):
            f = M_[r][c] / M_[c][c]
            for k in range(c, n + 1):
                M_[r][k] -= f * M_[c][k]
    x = [np.clongdouble(0)] * n
    for r in range(n - 1, -1, -1):
        x[r] = (M_[r][n] - sum(M_[r][k] * x[k] for k in range(r + 1, n))) / M_[r][r]
    return [complex(v) for v in x]


def test_three_atom_wfqfmu_brute_force():
    """Eq. 7 for three atoms in general position, assembled entry by entry: the dipole
    kernels as 4th-order finite differences of the scalar potential erf(r/R)/r (a
    dipole at r_j is the limit of two charges; the field is minus the gradient), the
    12 x 12 system solved by long-double Gaussian elimination.  Pins the block layout,
    every sign and index of Eq. 7, and the observables, against the oracle's LU."""
    xyz = np.array([[0.0, 0.0, 0.0], [2.9, 0.3, 0.0], [1.2, 2.6, 0.4]])
    st, el = _st(xyz, Rmu_bohr=0.9 * S.ELEMENTS["Ag"].atom_type()["Rmu_bohr"])
    w_ev = np.array([2.8, 3.9])
    aib = el.alpha_ib(w_ev)[None, :]
    e = np.array([0.6, 0.0, 0.8])
    res = M.solve(st, "wfqfmu", w_ev, [e], alpha_ib=aib)
    N = 3
    pos = [np.array(p) for p in st.pos]
    Rq, Rmu = list(st.Rq), list(st.Rmu)
    h = 2e-3

    def pot(ri, rj, R):
        r = float(np.linalg.norm(ri - rj))
        return math.erf(r / R) / r

    def d1(f, x, u):   # 4th-order directional derivative of f at x along unit u
        return (-f(x + 2 * h * u) + 8 * f(x + h * u) - 8 * f(x - h * u) + f(x - 2 * h * u)) / (12 * h)

    E3 = np.eye(3)
    # potential at i of a unit dipole at j along b: derivative of pot with respect to r_j
    def t_qmu(i, j, b):
        R = math.sqrt(Rq[i] ** 2 + Rmu[j] ** 2)
        return d1(lambda rj: pot(pos[i], rj, R), pos[j], E3[b])

    # minus the field at i (component a) of a unit charge at j: gradient with respect to r_i
    def t_muq(i, j, a):
        R = math.sqrt(Rmu[i] ** 2 + Rq[j] ** 2)
        return d1(lambda ri: pot(ri, pos[j], R), pos[i], E3[a])

    # minus the field at i (component a) of a unit dipole at j along b
    def t_mumu(i, j, a, b):
        R = math.sqrt(Rmu[i] ** 2 + Rmu[j] ** 2)
        g = lambda ri: d1(lambda rj: pot(ri, rj, R), pos[j], E3[b])   # potential of the dipole
        return d1(g, pos[i], E3[a])   # minus the field = gradient of the potential

    A_, Kb = _brute_matrix_wfq(st, 0.0)
    n4 = 4 * N
    T = [[0.0] * n4 for _ in range(n4)]
    for i in range(N):
        for j in range(N):
            if i == j:
                T[i][i] = math.sqrt(2.0 / math.pi) / Rq[i]
                continue
            T[i][j] = pot(pos[i], pos[j], math.sqrt(Rq[i] ** 2 + Rq[j] ** 2))
            for b in range(3):
                T[i][N + 3 * j + b] = t_qmu(i, j, b)
            for a in range(3):
                T[N + 3 * i + a][j] = t_muq(i, j, a)
                for b in range(3):
                    T[N + 3 * i + a][N + 3 * j + b] = t_mumu(i, j, a, b)
    for f in range(w_ev.size):
        w = w_ev[f] / M.HARTREE_EV
        zq = -w * (w * st.tau + 1j) / (2.0 * st.n * st.tau)
        zmu = -1.0 / aib[0, f]
        A = [[0j] * n4 for _ in range(n4)]
        for i in range(N):      # charge rows: Kbar applied to the charge rows of T
            for c in range(n4):
                A[i][c] = sum(Kb[i][k] * T[k][c] for k in range(N)) - (zq if c == i else 0.0)
        for r in range(N, n4):  # dipole rows: T itself
            for c in range(n4):
                A[r][c] = T[r][c] - (zmu if c == r else 0.0)
        V = [-(e @ p) for p in pos]
        b = [-sum(Kb[i][k] * V[k] for k in range(N)) for i in range(N)]
        b += [e[a] for i in range(N) for a in range(3)]
        x = _gauss_solve_longdouble(A, b)
        q, mu = x[:N], x[N:]
        dip = sum(q[i] * pos[i] for i in range(N)) + sum(
            np.array(mu[3 * i:3 * i + 3]) for i in range(N))
        assert np.allclose(res.alpha[f, :, 0], dip, rtol=1e-7, atol=0)
        assert np.allclose(res.q[f, 0], q, rtol=1e-7, atol=1e-9 * max(abs(v) for v in q))


# ------------------------------------------------------------ invariants

@pytest.fixture(scope="module")
def ag_small():
    st, el = _st(S.sphere("fcc", 4.09, 8.0))
    w = np.linspace(2.0, 6.0, 9)
    return st, el, w


def test_charge_conservation_wfq_and_wfqfmu(ag_small):
    st, el, w = ag_small
    r1 = M.solve(st, "wfq", w, XYZ)
    r2 = M.solve(st, "wfqfmu", w, XYZ, alpha_ib=el.alpha_ib(w)[None, :])
    for r in (r1, r2):
        tot = np.abs(r.q.sum(axis=-1))
        assert np.all(tot <= 1e-12 * np.abs(r.q).sum(axis=-1))


def test_reciprocity_and_passivity(ag_small):
    st, el, w = ag_small
    # break the cubic symmetry so that off-diagonal elements are not zero
    xyz = st.pos * M.BOHR_ANG
    xyz = xyz[xyz[:, 0] + 0.3 * xyz[:, 1] < 5.0]
    st2, _ = _st(xyz)
    for model, aib in (("wfq", None), ("wfqfmu", el.alpha_ib(w)[None, :])):
        r = M.solve(st2, model, w, XYZ, alpha_ib=aib)
        for f in range(len(w)):
            a = r.alpha[f]
            assert np.abs(a - a.T).max() <= 1e-10 * np.abs(a).max()
            assert np.all(np.diag(a).imag > 0)
        assert np.abs(r.alpha[:, 0, 1]).max() > 1e-3 * np.abs(r.alpha[:, 0, 0]).max()


def test_translation_and_rotation_covariance():
    xyz = S.cuboid("fcc", 4.09, 4.5, 4.5, 8.0)
    xyz = xyz[xyz[:, 2] < 5.0]
    st, el = _st(xyz)
    w = np.array([2.8, 3.9])
    aib = el.alpha_ib(w)[None, :]
    a0 = M.solve(st, "wfqfmu", w, XYZ, alpha_ib=aib).alpha
    st_t, _ = _st(xyz + np.array([3.3, -7.1, 2.2]))
    at = M.solve(st_t, "wfqfmu", w, XYZ, alpha_ib=aib).alpha
    assert np.abs(at - a0).max() <= 1e-9 * np.abs(a0).max()
    th = 0.7
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(0.4), -math.sin(0.4)], [0, math.sin(0.4), math.cos(0.4)]])
    Rm = Rx @ Rz
    st_r, _ = _st(xyz @ Rm.T)
    ar = M.solve(st_r, "wfqfmu", w, XYZ, alpha_ib=aib).alpha
    for f in range(2):
        assert np.abs(ar[f] - Rm @ a0[f] @ Rm.T).max() <= 1e-9 * np.abs(a0[f]).max()


def test_cubic_isotropy_of_fcc_sphere(ag_small):
    st, el, w = ag_small
    a = M.solve(st, "wfq", w, XYZ).alpha
    for f in range(len(w)):
        d = np.diag(a[f])
        assert np.abs(d - d[0]).max() <= 1e-10 * abs(d[0])


def test_static_limit_is_perfect_conductor():
    """omega -> 0 (z_q -> 0): Kbar (T q + V) = 0 makes the total potential uniform on a
    connected structure, so alpha = x^T T^-1 x - (1^T T^-1 x)^2 / (1^T T^-1 1),
    independent of Kbar (computed here by Cholesky solves on T alone)."""
    import scipy.linalg as sla
    st, _ = _st(S.sphere("fcc", 4.09, 7.0))
    r = M.solve(st, "wfq", [1e-8], XYZ[:1])
    T = M.tqq(st)
    c = sla.cho_factor(T)
    x = st.pos[:, 0]
    one = np.ones(st.natoms)
    Tx, T1 = sla.cho_solve(c, x), sla.cho_solve(c, one)
    expect = x @ Tx - (one @ Tx) ** 2 / (one @ T1)
    assert r.alpha[0, 0, 0].real == pytest.approx(expect, rel=1e-7)


def test_lu_and_spectral_routes_agree():
    st, _ = _st(S.sphere("fcc", 4.09, 10.0))
    w = np.linspace(1.5, 6.5, 21)
    lu = M.solve(st, "wfq", w, XYZ)
    md = SP.modes(st)
    sp = SP.alpha(st, md, w, XYZ)
    assert np.abs(sp - lu.alpha).max() <= 1e-10 * np.abs(lu.alpha).max()
    qs = SP.charges(st, md, w, XYZ)
    assert np.abs(qs - lu.q).max() <= 1e-10 * np.abs(lu.q).max()


def test_truncation_of_K_is_below_tolerance():
    st, _ = _st(S.sphere("fcc", 4.09, 8.0))
    w = np.linspace(2.0, 6.0, 5)
    a_cut = M.solve(st, "wfq", w, XYZ[:1], kcut_eps=1e-6).alpha[:, 0, 0]
    a_all = M.solve(st, "wfq", w, XYZ[:1], kcut_eps=0.0).alpha[:, 0, 0]
    assert np.abs(a_cut - a_all).max() <= 1e-5 * np.abs(a_all).max()


def _na_band(radius, w):
    """sigma_abs(w) of a Na sphere (x field) by the spectral route; returns (centroid, fwhm)."""
    st, _ = _st(S.sphere("bcc", 4.23, radius), "Na")
    md = SP.modes(st)
    a = SP.alpha(st, md, w, XYZ[:1], out_dirs=XYZ[:1])[:, 0, 0]
    sig = w * a.imag
    cen = float(np.sum(w * sig) / np.sum(sig))
    half = w[sig >= 0.5 * sig.max()]
    return cen, float(half.max() - half.min())


def test_na_sphere_band_approaches_drude_limit():
    """As the radius grows the dipolar band of sigma_abs moves monotonically toward the
    quasistatic Drude-sphere value omega_p / sqrt(3) (Na, 1 e/atom).  Small clusters
    split the band into several modes, so the band position is its centroid over
    2.5-4.8 eV.  With these stand-in parameters the approach is from below."""
    el = S.ELEMENTS["Na"]
    wp = math.sqrt(4 * math.pi * el.drude_n_au) * M.HARTREE_EV
    limit = wp / math.sqrt(3.0)
    w = np.linspace(2.5, 4.8, 461)
    cens = [_na_band(r, w)[0] for r in (20.0, 26.0, 32.0)]
    gaps = [limit - c for c in cens]
    assert all(g > 0 for g in gaps), cens
    assert gaps[0] > gaps[1] > gaps[2], cens
    assert gaps[-1] / limit < 0.05, cens


@pytest.mark.slow
def test_na_sphere_band_sharpens_with_size():
    el = S.ELEMENTS["Na"]
    limit = math.sqrt(4 * math.pi * el.drude_n_au) * M.HARTREE_EV / math.sqrt(3.0)
    w = np.linspace(2.5, 4.8, 1151)
    res = [_na_band(r, w) for r in (26.0, 32.0, 40.0, 46.0)]
    cens = [c for c, _ in res]
    widths = [f for _, f in res]
    assert all(b > a for a, b in zip(cens, cens[1:])), cens
    assert all(b < a for a, b in zip(widths, widths[1:])), widths
    assert (limit - cens[-1]) / limit < 0.02, cens


def test_mode_frequency_link():
    """Each pole of Eq. 1 sits where the real part of lambda_m - z_q vanishes:
    omega_m^2 = -2 n lambda_m; Im alpha peaks at the dominant mode frequency."""
    st, _ = _st(S.sphere("bcc", 4.23, 12.0), "Na")
    md = SP.modes(st)
    c = SP.project(st, md, XYZ[:1])[:, 0]
    weight = md.lam * c * c
    m = int(np.argmin(weight))       # lambda <= 0, so the largest |weight|
    wm = SP.mode_energies_ev(st, md)[m]
    w = np.linspace(wm - 0.3, wm + 0.3, 601)
    a = SP.alpha(st, md, w, XYZ[:1], out_dirs=XYZ[:1])[:, 0, 0]
    assert w[np.argmax(a.imag)] == pytest.approx(wm, abs=0.03)
