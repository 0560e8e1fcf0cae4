"""Dense FP64 assembly and direct solve of the wFQ (Eq. 1) and wFQFmu (Eq. 7) systems.

Test infrastructure (see the package docstring): plain numpy, float64 and
complex128 throughout, no blocking or reordering beyond the equations.

Units: the public inputs are Angstrom and eV (Sec. "Specify the Nanostructure":
geometry is read in Angstrom); everything inside is Hartree atomic units.

Readings of points the paper leaves open (each one is also a parameter, so
oracle/GPU parity never depends on the choice):
  * pair values of r0, d, s for two atom types: arithmetic mean of the two;
  * K is truncated to pairs with 1 - f(r) >= kcut_eps (kcut_eps = 0 keeps every
    pair), i.e. r <= s*r0*(1 + ln((1-eps)/eps)/d);
  * diagonal of T^qq: the r -> 0 limit of Eq. 5, sqrt(2/pi)/R_q (the paper calls
    this diagonal the chemical hardness);
  * T^qmu, T^muq, T^mumu: gradients of the Gaussian kernel of Eq. 5 with pair
    width sqrt(R_a^2 + R_b^2) for the two densities involved; their diagonals are
    zero unless ``mu_self_term`` is set (then T^mumu_ii = 4/(3 sqrt(pi) R^3) I with
    R = sqrt(2) R_mu, the self-field of a Gaussian dipole);
  * the external potential of a uniform field E0*e is V_i = -E0 e.r_i;
  * z_q uses one (n, tau) for the whole structure (Eq. 1 has a scalar shift).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.special import erf

BOHR_ANG = 0.529177210903      # 1 bohr in Angstrom (CODATA 2018)
HARTREE_EV = 27.211386245988   # 1 hartree in eV (CODATA 2018)
C_AU = 137.035999084           # speed of light in atomic units

TWO_OVER_SQRT_PI = 2.0 / np.sqrt(np.pi)


@dataclass
class Structure:
    """A nanostructure in atomic units, one row per atom."""

    pos: np.ndarray          # (N, 3) bohr
    r0: np.ndarray           # (N,) bohr, nearest-neighbour distance of the atom's lattice
    d: np.ndarray            # (N,) Fermi steepness (Eq. 4)
    s: np.ndarray            # (N,) Fermi scale factor (Eq. 4)
    area: np.ndarray         # (N,) effective area A_i, bohr^2 (Eq. 3)
    Rq: np.ndarray           # (N,) Gaussian charge width, bohr (Sec. 2.1)
    Rmu: np.ndarray          # (N,) Gaussian dipole width, bohr (Sec. 2.2)
    n: float                 # Drude density, a.u. (Eq. 6)
    tau: float               # Drude scattering time, a.u. (Eq. 6)
    type_idx: np.ndarray = field(default=None)  # (N,) atom type index

    @property
    def natoms(self) -> int:
        return self.pos.shape[0]


def structure_from_types(xyz_ang, type_idx, types) -> Structure:
    """Build a :class:`Structure` from boundary-style inputs.

    ``types`` is a sequence of dicts with keys r0_ang, d, s, area_bohr2,
    Rq_bohr, Rmu_bohr, drude_n_au, tau_au (the per-type parameters of Eqs. 3-6).
    All atom types must share n and tau (Eq. 1 has a single scalar z_q).
    """
    xyz_ang = np.asarray(xyz_ang, dtype=np.float64).reshape(-1, 3)
    type_idx = np.asarray(type_idx, dtype=np.int64).reshape(-1)
    tt = list(types)
    col = lambda key: np.array([float(t[key]) for t in tt])[type_idx]
    ns = {float(t["drude_n_au"]) for t in tt}
    taus = {float(t["tau_au"]) for t in tt}
    if len(ns) != 1 or len(taus) != 1:
        raise ValueError("all atom types must share drude_n_au and tau_au")
    return Structure(
        pos=xyz_ang / BOHR_ANG,
        r0=col("r0_ang") / BOHR_ANG,
        d=col("d"),
        s=col("s"),
        area=col("area_bohr2"),
        Rq=col("Rq_bohr"),
        Rmu=col("Rmu_bohr"),
        n=ns.pop(),
        tau=taus.pop(),
        type_idx=type_idx,
    )


# ----------------------------------------------------------------------------
# Geometry
# ----------------------------------------------------------------------------

def pair_vectors(pos):
    """r_ij = r_i - r_j (N, N, 3) and |r_ij| (N, N)."""
    rij = pos[:, None, :] - pos[None, :, :]
    dist = np.sqrt(np.sum(rij * rij, axis=-1))
    return rij, dist


# ----------------------------------------------------------------------------
# Conductance operator, Eqs. 2-4
# ----------------------------------------------------------------------------

def fermi(r, r0, d, s):
    """Eq. 4: f(r) = 1 / (1 + exp[-d (r / (s r0) - 1)])."""
    return 1.0 / (1.0 + np.exp(-d * (r / (s * r0) - 1.0)))


def cutoff_radius(r0, d, s, kcut_eps):
    """Distance beyond which 1 - f(r) < kcut_eps (inf when kcut_eps == 0).

    1 - f(r) = 1 / (1 + exp[d (r/(s r0) - 1)]) falls monotonically, so the pairs
    kept are exactly those with r <= s r0 (1 + ln((1 - eps)/eps) / d).
    """
    if kcut_eps <= 0.0:
        return np.full(np.shape(r0), np.inf)
    return s * r0 * (1.0 + np.log((1.0 - kcut_eps) / kcut_eps) / d)


def pair_params(st: Structure):
    """Pair values r0_ij, d_ij, s_ij (arithmetic means of the two atoms' values)."""
    mean = lambda a: 0.5 * (a[:, None] + a[None, :])
    return mean(st.r0), mean(st.d), mean(st.s)


def conductance_K(st: Structure, kcut_eps: float = 1e-6):
    """Eq. 3: K_ij = [1 - f(r_ij)] A_i / r_ij for i != j (kept pairs), K_ii = 0."""
    _, dist = pair_vectors(st.pos)
    r0, d, s = pair_params(st)
    rcut = cutoff_radius(r0, d, s, kcut_eps)
    N = st.natoms
    K = np.zeros((N, N))
    off = ~np.eye(N, dtype=bool)
    keep = off & (dist <= rcut)
    one_minus_f = 1.0 - fermi(dist[keep], r0[keep], d[keep], s[keep])
    A_row = np.broadcast_to(st.area[:, None], (N, N))
    K[keep] = one_minus_f * A_row[keep] / dist[keep]
    return K


def kbar(K):
    """Eq. 2: Kbar_ij = K_ij - delta_ij sum_k K_ik."""
    return K - np.diag(K.sum(axis=1))


# ----------------------------------------------------------------------------
# Gaussian interaction kernels, Eq. 5 and its derivatives (Sec. 2.2)
# ----------------------------------------------------------------------------

def gauss_T(r, R):
    """T(r; R) = erf(r/R)/r (Eq. 5), r > 0."""
    return erf(r / R) / r


def gauss_T1(r, R):
    """dT/dr = (g x - erf x) / r^2 with x = r/R, g = (2/sqrt(pi)) exp(-x^2)."""
    x = r / R
    g = TWO_OVER_SQRT_PI * np.exp(-x * x)
    return (g * x - erf(x)) / (r * r)


def gauss_T2(r, R):
    """d2T/dr2 = (2 erf x - 2 g x - 2 g x^3) / r^3."""
    x = r / R
    g = TWO_OVER_SQRT_PI * np.exp(-x * x)
    return (2.0 * erf(x) - 2.0 * g * x - 2.0 * g * x ** 3) / r ** 3


def tqq(st: Structure):
    """Eq. 5: T^qq_ij = erf(r_ij / R_ij) / r_ij, R_ij = sqrt(Rq_i^2 + Rq_j^2).

    Diagonal: the r -> 0 limit, 2 / (sqrt(pi) R_ii) = sqrt(2/pi) / Rq_i.
    """
    _, dist = pair_vectors(st.pos)
    N = st.natoms
    Rij = np.sqrt(st.Rq[:, None] ** 2 + st.Rq[None, :] ** 2)
    T = np.empty((N, N))
    off = ~np.eye(N, dtype=bool)
    T[off] = gauss_T(dist[off], Rij[off])
    T[np.diag_indices(N)] = np.sqrt(2.0 / np.pi) / st.Rq
    return T


def tqmu(st: Structure):
    """Charge-dipole kernel, (N, N, 3): potential at atom i of a unit dipole at atom j.

    T^qmu_ij = grad_{r_j} T(|r_i - r_j|; R) = -T'(r_ij) rhat_ij,
    R = sqrt(Rq_i^2 + Rmu_j^2), rhat_ij = (r_i - r_j)/r_ij; zero for i == j.
    """
    rij, dist = pair_vectors(st.pos)
    N = st.natoms
    R = np.sqrt(st.Rq[:, None] ** 2 + st.Rmu[None, :] ** 2)
    out = np.zeros((N, N, 3))
    off = ~np.eye(N, dtype=bool)
    rhat = rij[off] / dist[off][:, None]
    out[off] = -gauss_T1(dist[off], R[off])[:, None] * rhat
    return out


def tmuq(st: Structure):
    """Dipole-charge kernel, (N, 3, N): minus the field at atom i of a unit charge at j.

    T^muq_ij = grad_{r_i} T(|r_i - r_j|; R) = +T'(r_ij) rhat_ij,
    R = sqrt(Rmu_i^2 + Rq_j^2); zero for i == j.
    """
    rij, dist = pair_vectors(st.pos)
    N = st.natoms
    R = np.sqrt(st.Rmu[:, None] ** 2 + st.Rq[None, :] ** 2)
    out = np.zeros((N, N, 3))
    off = ~np.eye(N, dtype=bool)
    rhat = rij[off] / dist[off][:, None]
    out[off] = gauss_T1(dist[off], R[off])[:, None] * rhat
    return np.transpose(out, (0, 2, 1))


def tmumu(st: Structure, mu_self_term: bool = False):
    """Dipole-dipole kernel, (N, 3, N, 3): minus the field at i of a unit dipole at j.

    T^mumu_ij = -grad grad T = -[T'' rhat rhat^T + (T'/r)(I - rhat rhat^T)],
    R = sqrt(Rmu_i^2 + Rmu_j^2).  Diagonal 0, or the Gaussian self term
    4/(3 sqrt(pi) R^3) I with R = sqrt(2) Rmu_i when ``mu_self_term``.
    """
    rij, dist = pair_vectors(st.pos)
    N = st.natoms
    R = np.sqrt(st.Rmu[:, None] ** 2 + st.Rmu[None, :] ** 2)
    out = np.zeros((N, N, 3, 3))
    off = ~np.eye(N, dtype=bool)
    r = dist[off]
    rhat = rij[off] / r[:, None]
    rr = rhat[:, :, None] * rhat[:, None, :]
    eye = np.eye(3)[None]
    t1 = gauss_T1(r, R[off])
    t2 = gauss_T2(r, R[off])
    out[off] = -(t2[:, None, None] * rr + (t1 / r)[:, None, None] * (eye - rr))
    if mu_self_term:
        Rs = np.sqrt(2.0) * st.Rmu
        for i in range(N):
            out[i, i] = 4.0 / (3.0 * np.sqrt(np.pi) * Rs[i] ** 3) * np.eye(3)
    return np.transpose(out, (0, 2, 1, 3))


def t_full(st: Structure, mu_self_term: bool = False):
    """The 4N x 4N kernel of Eq. 7, unknown order (q_1..q_N, mu_1x, mu_1y, mu_1z, ...)."""
    N = st.natoms
    T = np.zeros((4 * N, 4 * N))
    T[:N, :N] = tqq(st)
    T[:N, N:] = tqmu(st).reshape(N, 3 * N)
    T[N:, :N] = tmuq(st).reshape(3 * N, N)
    T[N:, N:] = tmumu(st, mu_self_term).reshape(3 * N, 3 * N)
    return T


# ----------------------------------------------------------------------------
# Frequency-dependent shifts, Eqs. 6 and 8
# ----------------------------------------------------------------------------

def z_q(omega, n, tau):
    """Eq. 6: z_q(w) = -w (w tau + i) / (2 n tau)."""
    return -omega * (omega * tau + 1j) / (2.0 * n * tau)


def z_mu(alpha_ib):
    """Eq. 8: z_mu(w) = -1 / alpha^IB(w)."""
    return -1.0 / np.asarray(alpha_ib, dtype=np.complex128)


# ----------------------------------------------------------------------------
# Right-hand sides and system matrices, Eqs. 1 and 7
# ----------------------------------------------------------------------------

def potential_V(st: Structure, e_dir, e0=1.0):
    """External potential of the uniform field E0 e: V_i = -E0 e . r_i."""
    return -e0 * st.pos @ np.asarray(e_dir, dtype=np.float64)


def rhs_wfq(Kb, st, e_dir, e0=1.0):
    """Right-hand side of Eq. 1: -Kbar V."""
    return -(Kb @ potential_V(st, e_dir, e0))


def rhs_wfqfmu(Kb, st, e_dir, e0=1.0):
    """Right-hand side of Eq. 7: diag(Kbar, I_3N) (-V; E)."""
    N = st.natoms
    b = np.empty(4 * N)
    b[:N] = -(Kb @ potential_V(st, e_dir, e0))
    b[N:] = np.tile(e0 * np.asarray(e_dir, dtype=np.float64), N)
    return b


def matrix_wfq(Kb, T, zq):
    """Eq. 1 system matrix: Kbar T^qq - z_q I_N."""
    return (Kb @ T).astype(np.complex128) - zq * np.eye(T.shape[0])


def matrix_wfqfmu(Kb, T4, zq, zmu_atoms):
    """Eq. 7 system matrix: diag(Kbar, I_3N) T - diag(z_q I_N, z_mu I_3N).

    ``zmu_atoms`` holds z_mu for every atom (N,), so several atom types may carry
    their own alpha^IB; each atom's value fills its three dipole rows.
    """
    N = Kb.shape[0]
    P = np.zeros((4 * N, 4 * N))
    P[:N, :N] = Kb
    P[N:, N:] = np.eye(3 * N)
    shift = np.concatenate([np.full(N, zq, dtype=np.complex128),
                            np.repeat(np.asarray(zmu_atoms, dtype=np.complex128), 3)])
    return (P @ T4).astype(np.complex128) - np.diag(shift)


# ----------------------------------------------------------------------------
# Observables, Sec. "Observables"
# ----------------------------------------------------------------------------

def dipole(st: Structure, q, mu=None):
    """d = sum_i q_i r_i (+ sum_i mu_i for wFQFmu); q (N, P), mu (N, 3, P) -> (3, P)."""
    d = st.pos.T @ q
    if mu is not None:
        d = d + mu.sum(axis=0)
    return d


def sigma_abs(omega, alpha_diag_im_sum):
    """sigma_abs = 4 pi w / (3 c) Tr Im alpha (Im alpha summed over x, y, z given)."""
    return 4.0 * np.pi * omega / (3.0 * C_AU) * alpha_diag_im_sum


# ----------------------------------------------------------------------------
# The direct solve ("inversion": one LU factorisation per frequency)
# ----------------------------------------------------------------------------

@dataclass
class Result:
    alpha: np.ndarray        # (F, 3, P) complex, bohr^3
    q: np.ndarray            # (F, P, N) complex
    mu: np.ndarray | None    # (F, P, N, 3) complex (wFQFmu)
    sigma_abs_pol: np.ndarray  # (F, P): 4 pi w / c * Im(e_p . alpha e_p)
    rel_residual: np.ndarray   # (F, P): ||b - A x|| / ||b|| of the LU solution


def solve(st: Structure, model: str, omega_ev, pol_dirs, alpha_ib=None,
          kcut_eps: float = 1e-6, e0: float = 1.0, mu_self_term: bool = False) -> Result:
    """Solve Eq. 1 (model='wfq') or Eq. 7 (model='wfqfmu') by LU for every frequency.

    ``alpha_ib``: complex (n_types, F) interband polarisabilities in a.u. (wFQFmu).
    All polarisations share one factorisation per frequency.
    """
    omega = np.asarray(omega_ev, dtype=np.float64) / HARTREE_EV
    pols = np.asarray(pol_dirs, dtype=np.float64).reshape(-1, 3)
    N, F, P = st.natoms, omega.size, pols.shape[0]
    Kb = kbar(conductance_K(st, kcut_eps))
    if model == "wfq":
        T = tqq(st)
        B = np.stack([rhs_wfq(Kb, st, e, e0) for e in pols], axis=1)
    elif model == "wfqfmu":
        T = t_full(st, mu_self_term)
        B = np.stack([rhs_wfqfmu(Kb, st, e, e0) for e in pols], axis=1)
        alpha_ib = np.asarray(alpha_ib, dtype=np.complex128)
    else:
        raise ValueError(model)
    alpha = np.zeros((F, 3, P), dtype=np.complex128)
    qs = np.zeros((F, P, N), dtype=np.complex128)
    mus = np.zeros((F, P, N, 3), dtype=np.complex128) if model == "wfqfmu" else None
    relres = np.zeros((F, P))
    for f in range(F):
        zq = z_q(omega[f], st.n, st.tau)
        if model == "wfq":
            A = matrix_wfq(Kb, T, zq)
        else:
            zmu_atoms = z_mu(alpha_ib[st.type_idx, f])
            A = matrix_wfqfmu(Kb, T, zq, zmu_atoms)
        X = np.linalg.solve(A, B.astype(np.complex128))
        bn = np.linalg.norm(B, axis=0)
        rn = np.linalg.norm(B - A @ X, axis=0)
        relres[f] = np.where(bn > 0, rn / np.where(bn > 0, bn, 1.0), 0.0)
        q = X[:N]
        mu = X[N:].reshape(N, 3, P) if model == "wfqfmu" else None
        alpha[f] = dipole(st, q, mu) / e0
        qs[f] = q.T
        if mus is not None:
            mus[f] = np.transpose(mu, (2, 0, 1))
    sig = np.zeros((F, P))
    for p in range(P):
        a_pp = np.einsum("k,fkl,l->f", pols[p], alpha, np.eye(P)[p])  # e_p . alpha[:, :, p]
        sig[:, p] = 4.0 * np.pi * omega / C_AU * a_pp.imag
    return Result(alpha=alpha, q=qs, mu=mus, sigma_abs_pol=sig, rel_residual=relres)
