"""Heterogeneous wFQFmu (alloys, core-shell): Eq. 9 with the per-atom interband
polarisability of Eq. 10, assembled densely and solved by LU per frequency.

Test infrastructure (see the package docstring): plain numpy FP64 / complex128.

Readings of points the paper leaves open (each a parameter or a stated choice):
  * z_q is per atom, z_q,i = -w (w tau_i + i) / (2 n_i tau_i) (Eq. 6 with the row
    atom's n, tau; Eq. 9 prints a scalar z_q, which is exact only for equal n, tau).
    With it the bond conductance g_ij = D_i K_ij + D_j K_ji, D = 2 n tau/(1 - i w tau),
    is symmetric, so the induced charge is conserved; the tests check that.
  * H_ij = (n_j tau_j)/(n_i tau_i) (1 - i w tau_i)/(1 - i w tau_j) K_ji, literal (note
    the transposed K); Hbar = H - diag(row sums of H).
  * "nearest neighbours" N_A,i, N_B,i of Eq. 10: atoms j != i within the Fermi
    midpoint of the pair, r_ij <= s_ij r0_ij (the first shell of fcc / bcc lattices
    with s = 1.1).
  * T, K and the Gaussian widths are those of the homogeneous model (pair values of
    r0, d, s are means of the two atoms' types).
"""
from __future__ import annotations

import numpy as np

from . import model as M


def structure(xyz_ang, type_idx, types):
    """A model.Structure with per-atom n, tau arrays (returned separately)."""
    xyz_ang = np.asarray(xyz_ang, dtype=np.float64).reshape(-1, 3)
    type_idx = np.asarray(type_idx, dtype=np.int64).reshape(-1)
    tt = list(types)
    col = lambda key: np.array([float(t[key]) for t in tt])[type_idx]
    st = M.Structure(pos=xyz_ang / M.BOHR_ANG, r0=col("r0_ang") / M.BOHR_ANG, d=col("d"),
                     s=col("s"), area=col("area_bohr2"), Rq=col("Rq_bohr"),
                     Rmu=col("Rmu_bohr"), n=float("nan"), tau=float("nan"),
                     type_idx=type_idx)
    return st, col("drude_n_au"), col("tau_au")


def neighbour_counts(st, n_types):
    """counts[i, t] = atoms of type t within the Fermi midpoint s_ij r0_ij of atom i."""
    _, dist = M.pair_vectors(st.pos)
    r0, _, s = M.pair_params(st)
    near = (dist <= s * r0) & ~np.eye(st.natoms, dtype=bool)
    counts = np.zeros((st.natoms, n_types), dtype=np.int64)
    for t in range(n_types):
        counts[:, t] = (near & (st.type_idx[None, :] == t)).sum(axis=1)
    return counts


def alpha_ib_hetero(type_idx, counts, alpha_ib_types):
    """Eq. 10 for every atom: the own type and its nearest neighbours' types enter the
    inverse polarisability with weights (1 + N_own) and N_other over (1 + sum N).
    alpha_ib_types (n_types,) complex at one frequency; returns (N,) complex."""
    inv = 1.0 / np.asarray(alpha_ib_types, dtype=np.complex128)
    N = len(type_idx)
    out = np.empty(N, dtype=np.complex128)
    for i in range(N):
        w = counts[i].astype(np.float64).copy()
        w[type_idx[i]] += 1.0
        out[i] = 1.0 / ((w * inv).sum() / w.sum())
    return out


def h_matrix(K, n, tau, omega):
    """H_ij = (n_j tau_j)/(n_i tau_i) (1 - i w tau_i)/(1 - i w tau_j) K_ji."""
    ntau = n * tau
    fac = (ntau[None, :] / ntau[:, None]) * ((1.0 - 1j * omega * tau)[:, None]
                                              / (1.0 - 1j * omega * tau)[None, :])
    return fac * K.T


def z_q_atoms(omega, n, tau):
    """Eq. 6 per atom with the atom's own n, tau (reading above)."""
    return -omega * (omega * tau + 1j) / (2.0 * n * tau)


def solve(xyz_ang, type_idx, types, omega_ev, pol_dirs, alpha_ib_types, kcut_eps=1e-6,
          e0=1.0, mu_self_term=False):
    """Eq. 9 by LU per frequency.  alpha_ib_types (n_types, F) complex.
    Returns (alpha (F, 3, P), q (F, P, N), mu (F, P, N, 3), rel_residual (F, P))."""
    st, n, tau = structure(xyz_ang, type_idx, types)
    N = st.natoms
    omega = np.asarray(omega_ev, dtype=np.float64) / M.HARTREE_EV
    pols = np.asarray(pol_dirs, dtype=np.float64).reshape(-1, 3)
    F, P = omega.size, pols.shape[0]
    aib = np.asarray(alpha_ib_types, dtype=np.complex128)
    K = M.conductance_K(st, kcut_eps)
    Kb = M.kbar(K)
    T = M.t_full(st, mu_self_term)
    counts = neighbour_counts(st, aib.shape[0])
    alpha = np.zeros((F, 3, P), dtype=np.complex128)
    qs = np.zeros((F, P, N), dtype=np.complex128)
    mus = np.zeros((F, P, N, 3), dtype=np.complex128)
    rel = np.zeros((F, P))
    for f, w in enumerate(omega):
        H = h_matrix(K, n, tau, w)
        Hb = H - np.diag(H.sum(axis=1))
        C = 0.5 * (Kb + Hb)                          # frequency-dependent conductance block
        Pm = np.zeros((4 * N, 4 * N), dtype=np.complex128)
        Pm[:N, :N] = C
        Pm[N:, N:] = np.eye(3 * N)
        zq = z_q_atoms(w, n, tau)
        zmu = -1.0 / alpha_ib_hetero(st.type_idx, counts, aib[:, f])
        A = Pm @ T - np.diag(np.concatenate([zq, np.repeat(zmu, 3)]))
        B = np.zeros((4 * N, P), dtype=np.complex128)
        for p, e in enumerate(pols):
            V = M.potential_V(st, e, e0)
            rhs = np.concatenate([-V, np.tile(e0 * e, N)])
            B[:, p] = Pm @ rhs
        X = np.linalg.solve(A, B)
        bn = np.linalg.norm(B, axis=0)
        rel[f] = np.linalg.norm(B - A @ X, axis=0) / np.where(bn > 0, bn, 1.0)
        q = X[:N]
        mu = X[N:].reshape(N, 3, P)
        alpha[f] = M.dipole(st, q, mu) / e0
        qs[f] = q.T
        mus[f] = np.transpose(mu, (2, 0, 1))
    return alpha, qs, mus, rel
