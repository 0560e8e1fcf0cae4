"""Boundary element method in the DPCM form (Sec. 2.3, Eq. 11): the surface charges of a
meshed dielectric or metal particle in a uniform field, solved densely per frequency.

Test infrastructure (see the package docstring): plain numpy FP64 / complex128.

The surface is discretised into tesserae i with barycentre s_i, outward unit normal n_i
and area A_i; the unknowns are the surface charge densities sigma_i (charge A_i sigma_i).

Reading of Eq. 11.  As printed, [2 pi (e2 + e1)/(e2 - e1) A + F] sigma = -E_n with
F_ij = (s_i - s_j).n_j A_j / |s_i - s_j|^3 (i != j), F_ii = 1.0694 sqrt(4 pi A_i) / (2R):
with the area matrix A multiplying the first term the system is not dimensionally
consistent, and a sphere meshed ever more finely does not approach the exact quasistatic
polarisability.  The equation it abbreviates is the normal-field boundary condition of
DPCM: with Lambda(w) = 2 pi (e2 + e1)/(e2 - e1) (e2 the particle's permittivity, e1 the
medium's),
    (Lambda I - Ft) sigma = E . n,
    Ft_ij = A_j (s_i - s_j).n_i / |s_i - s_j|^3  (i != j),   Ft_ii = 1.0694 sqrt(4 pi A_i) / (2R),
i.e. the jump e_in E_n,in = e_out E_n,out across each tessera, E_n,in/out = E_n -/+ 2 pi sigma
for its own sheet, E_n the normal field of the external field and every other charge,
and the printed curvature self term.  It converges to R^3 (e2 - e1)/(e2 + 2 e1) for a
sphere (the tests pin this).  R is the radius of the sphere that encloses the mesh.
Observables (Sec. "Observables"): d = sum_i q_i s_i with the tesserae's charges
q_i = A_i sigma_i, alpha_kl = d_k / E_l.

Reading of Eq. 12 (IEFPCM).  [Lambda I + F] S A^-1 sigma = -(2 pi I + F) V, with sigma
here the tesserae's charges (S A^-1 maps charges to the potential they create at the
barycentres: (S A^-1)_ij = 1/|s_i - s_j|, diagonal 1.0694 sqrt(4 pi / A_i)), V_i = -E0 e.s_i
the external potential, and F_ij = A_j (s_i - s_j).n_j / |s_i - s_j|^3 (the source
tessera's normal, as printed).  With the printed positive diagonal the refined sphere
converges only slowly (0.67 -> 0.80 of the exact value from 800 to 3,200 tesserae at
e2 = -2.5 + 0.3i); the diagonal that continues the off-diagonal sum -- the self part of
the double layer, negative on a convex surface whose off-diagonal entries are negative --
is F_ii = -1.0694 sqrt(4 pi A_i) / (2R), and with it the sphere converges like DPCM.  That
sign is this reading.  Solved in two steps: y = S A^-1 q from (Lambda I + F) y = -(2 pi I +
F) V, then q from (S A^-1) q = y.
"""
from __future__ import annotations

import numpy as np

from . import model as M


def enclosing_radius(pos):
    return float(np.linalg.norm(pos - pos.mean(axis=0), axis=1).max())


def f_matrix(pos, nrm, area, R):
    """Ft of the reading above (bohr units)."""
    d = pos[:, None, :] - pos[None, :, :]
    r = np.linalg.norm(d, axis=-1)
    n = pos.shape[0]
    off = ~np.eye(n, dtype=bool)
    F = np.zeros((n, n))
    F[off] = (np.einsum("ijk,ik->ij", d, nrm)[off] / r[off] ** 3) * np.broadcast_to(area[None, :], (n, n))[off]
    F[np.diag_indices(n)] = 1.0694 * np.sqrt(4.0 * np.pi * area) / (2.0 * R)
    return F


def f_rows(pos, nrm, area, R, rows):
    """Rows `rows` of Ft (bohr units), one at a time, for meshes too large for f_matrix."""
    rows = np.asarray(rows, dtype=np.int64).reshape(-1)
    out = np.zeros((rows.size, pos.shape[0]))
    for k, i in enumerate(rows):
        d = pos[i][None, :] - pos
        r = np.linalg.norm(d, axis=1)
        off = np.arange(pos.shape[0]) != i
        out[k, off] = area[off] * (d[off] @ nrm[i]) / r[off] ** 3
        out[k, i] = 1.0694 * np.sqrt(4.0 * np.pi * area[i]) / (2.0 * R)
    return out


def lam(eps2, eps1):
    """Lambda(w) = 2 pi (e2 + e1) / (e2 - e1)."""
    eps2 = np.asarray(eps2, dtype=np.complex128)
    eps1 = np.asarray(eps1, dtype=np.complex128)
    return 2.0 * np.pi * (eps2 + eps1) / (eps2 - eps1)


def solve(pos_ang, nrm, area_ang2, eps2, eps1, pol_dirs, e0=1.0, radius_ang=None):
    """DPCM by LU per frequency.  eps2, eps1: (F,) complex (or broadcastable scalars).
    Returns alpha (F, 3, P) bohr^3, q (F, P, N) (tessera charges), relative residuals."""
    pos = np.asarray(pos_ang, dtype=np.float64) / M.BOHR_ANG
    area = np.asarray(area_ang2, dtype=np.float64) / M.BOHR_ANG ** 2
    nrm = np.asarray(nrm, dtype=np.float64)
    R = (enclosing_radius(np.asarray(pos_ang)) if radius_ang is None else radius_ang) / M.BOHR_ANG
    pols = np.asarray(pol_dirs, dtype=np.float64).reshape(-1, 3)
    L = np.atleast_1d(lam(eps2, eps1))
    F = f_matrix(pos, nrm, area, R)
    n = pos.shape[0]
    B = e0 * (nrm @ pols.T)                      # E . n for every direction, (n, P)
    Fq = L.size
    alpha = np.zeros((Fq, 3, pols.shape[0]), dtype=np.complex128)
    qs = np.zeros((Fq, pols.shape[0], n), dtype=np.complex128)
    rel = np.zeros((Fq, pols.shape[0]))
    for f in range(Fq):
        A = L[f] * np.eye(n) - F
        sig = np.linalg.solve(A, B.astype(np.complex128))
        rel[f] = np.linalg.norm(B - A @ sig, axis=0) / np.linalg.norm(B, axis=0)
        q = area[:, None] * sig
        alpha[f] = pos.T @ q / e0
        qs[f] = q.T
    return alpha, qs, rel


def f_matrix_ief(pos, nrm, area, R):
    """F of Eq. 12 (bohr units): source normal n_j off the diagonal, and the negative
    self term of the reading above."""
    d = pos[:, None, :] - pos[None, :, :]
    r = np.linalg.norm(d, axis=-1)
    n = pos.shape[0]
    off = ~np.eye(n, dtype=bool)
    F = np.zeros((n, n))
    F[off] = (np.einsum("ijk,jk->ij", d, nrm)[off] / r[off] ** 3) * np.broadcast_to(area[None, :], (n, n))[off]
    F[np.diag_indices(n)] = -1.0694 * np.sqrt(4.0 * np.pi * area) / (2.0 * R)
    return F


def g_matrix(pos, area):
    """S A^-1 of Eq. 12: 1/|s_i - s_j| off the diagonal, 1.0694 sqrt(4 pi / A_i) on it."""
    d = pos[:, None, :] - pos[None, :, :]
    r = np.linalg.norm(d, axis=-1)
    n = pos.shape[0]
    off = ~np.eye(n, dtype=bool)
    G = np.zeros((n, n))
    G[off] = 1.0 / r[off]
    G[np.diag_indices(n)] = 1.0694 * np.sqrt(4.0 * np.pi / area)
    return G


def solve_iefpcm(pos_ang, nrm, area_ang2, eps2, eps1, pol_dirs, e0=1.0, radius_ang=None):
    """IEFPCM (Eq. 12) by LU per frequency.  Returns alpha (F, 3, P) bohr^3, q (F, P, N)
    (tessera charges), and the relative residuals of the two steps (F, P, 2)."""
    pos = np.asarray(pos_ang, dtype=np.float64) / M.BOHR_ANG
    area = np.asarray(area_ang2, dtype=np.float64) / M.BOHR_ANG ** 2
    nrm = np.asarray(nrm, dtype=np.float64)
    R = (enclosing_radius(np.asarray(pos_ang)) if radius_ang is None else radius_ang) / M.BOHR_ANG
    pols = np.asarray(pol_dirs, dtype=np.float64).reshape(-1, 3)
    L = np.atleast_1d(lam(eps2, eps1))
    F = f_matrix_ief(pos, nrm, area, R)
    G = g_matrix(pos, area)
    n = pos.shape[0]
    V = -e0 * (pos @ pols.T)                      # external potential, (n, P)
    c = -(2.0 * np.pi * V + F @ V)                # right-hand side of the first step
    Fq = L.size
    alpha = np.zeros((Fq, 3, pols.shape[0]), dtype=np.complex128)
    qs = np.zeros((Fq, pols.shape[0], n), dtype=np.complex128)
    rel = np.zeros((Fq, pols.shape[0], 2))
    for f in range(Fq):
        A = L[f] * np.eye(n) + F
        y = np.linalg.solve(A, c.astype(np.complex128))
        q = np.linalg.solve(G, y)
        rel[f, :, 0] = np.linalg.norm(c - A @ y, axis=0) / np.linalg.norm(c, axis=0)
        rel[f, :, 1] = np.linalg.norm(y - G @ q, axis=0) / np.linalg.norm(y, axis=0)
        alpha[f] = pos.T @ q / e0
        qs[f] = q.T
    return alpha, qs, rel
