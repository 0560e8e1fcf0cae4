"""Second exact route for the wFQ system (Eq. 1): Cholesky of T plus one eigensolve.

Test infrastructure (see the package docstring).

With T^qq = L L^T (T is the Coulomb Gram matrix of Gaussians, hence symmetric
positive definite) and Kbar symmetric (uniform effective area), the matrix
M = Kbar T of Eq. 1 is similar to S = L^T Kbar L:  M = L^-T S L^T.  With
S = U diag(lambda) U^T and y_l = L^-1 r_l (r_l the atom coordinates along the
field direction e_l):

    q_l(w)      = E0 L^-T U diag(lambda / (lambda - z_q(w))) U^T y_l
    alpha_kl(w) = sum_m lambda_m (u_m . y_k)(u_m . y_l) / (lambda_m - z_q(w))

One O(N^3) factorisation then gives every frequency in O(N) per (w, k, l).
This is an exact rewriting of Eq. 1 (no approximation), so it must agree with
the LU route of ``oracle.model.solve`` to rounding.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from . import model


@dataclass
class Modes:
    lam: np.ndarray      # (N,) eigenvalues of S (<= 0)
    U: np.ndarray        # (N, N) eigenvectors of S
    L: np.ndarray        # (N, N) lower Cholesky factor of T^qq
    Kb: np.ndarray       # (N, N) Kbar


def modes(st: model.Structure, kcut_eps: float = 1e-6) -> Modes:
    Kb = model.kbar(model.conductance_K(st, kcut_eps))
    if not np.allclose(Kb, Kb.T, rtol=0, atol=1e-14 * np.abs(Kb).max()):
        raise ValueError("spectral route needs a symmetric Kbar (uniform effective area)")
    T = model.tqq(st)
    L = sla.cholesky(T, lower=True)
    S = L.T @ Kb @ L
    S = 0.5 * (S + S.T)
    lam, U = sla.eigh(S)
    return Modes(lam=lam, U=U, L=L, Kb=Kb)


def project(st: model.Structure, md: Modes, pol_dirs):
    """c[m, l] = u_m . y_l with y_l = L^-1 r_l; r_l = pos . e_l."""
    pols = np.asarray(pol_dirs, dtype=np.float64).reshape(-1, 3)
    R = st.pos @ pols.T                       # (N, P)
    Y = sla.solve_triangular(md.L, R, lower=True)
    return md.U.T @ Y                          # (N, P)


def alpha(st: model.Structure, md: Modes, omega_ev, pol_dirs, out_dirs=None):
    """alpha[f, k, l] for output directions k (default x, y, z) and field directions l."""
    omega = np.asarray(omega_ev, dtype=np.float64) / model.HARTREE_EV
    out_dirs = np.eye(3) if out_dirs is None else np.asarray(out_dirs, dtype=np.float64)
    C_in = project(st, md, pol_dirs)           # (N, P)
    C_out = project(st, md, out_dirs)          # (N, 3)
    zq = model.z_q(omega, st.n, st.tau)        # (F,)
    w = md.lam[None, :] / (md.lam[None, :] - zq[:, None])     # (F, N)
    return np.einsum("mk,fm,ml->fkl", C_out, w, C_in)


def charges(st: model.Structure, md: Modes, omega_ev, pol_dirs, e0: float = 1.0):
    """q[f, p, i] for every frequency and field direction."""
    omega = np.asarray(omega_ev, dtype=np.float64) / model.HARTREE_EV
    C_in = project(st, md, pol_dirs)           # (N, P)
    zq = model.z_q(omega, st.n, st.tau)
    w = md.lam[None, :] / (md.lam[None, :] - zq[:, None])     # (F, N)
    LinvT_U = sla.solve_triangular(md.L.T, md.U, lower=False)  # L^-T U
    return e0 * np.einsum("im,fm,mp->fpi", LinvT_U, w, C_in)


def mode_energies_ev(st: model.Structure, md: Modes):
    """w_m = sqrt(-2 n lambda_m) in eV: the real part of the pole of mode m."""
    lam = np.minimum(md.lam, 0.0)
    return np.sqrt(-2.0 * st.n * lam) * model.HARTREE_EV
