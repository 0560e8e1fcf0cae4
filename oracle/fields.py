"""Induced density, potential and field of a solved structure at probe points
(Sec. "Post-process Analysis": density and field maps at a plasmon resonance).

Test infrastructure (see the package docstring): plain numpy / scipy in float64 and
complex128, one probe point against every atom, no blocking.

The model's charges and dipoles are Gaussian distributions (Secs. 2.1, 2.2): atom i
carries the charge density q_i g(r - r_i; R_q,i) and the dipole density
-mu_i . grad g(r - r_i; R_mu,i), with the normalised Gaussian
    g(x; R) = (pi R^2)^(-3/2) exp(-|x|^2 / R^2),
whose potential is erf(|x| / R) / |x| (the same kernel as Eq. 5, with the single
width R of one density instead of the pair width).  Reading of the paper: it names
the maps but prints no formula; these follow from the model's densities.

    phi(r) = sum_i q_i G(r - r_i; R_q,i) - sum_i mu_i . grad G(r - r_i; R_mu,i)
    E(r)   = -grad phi(r)
with G(x; R) = erf(|x|/R)/|x| (G(0) = 2 / (sqrt(pi) R)).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

SQRT_PI = np.sqrt(np.pi)


def _radial(r, R):
    """G, G' and G'' of G(r) = erf(r/R)/r for r > 0 (derivatives in r)."""
    x = r / R
    e = erf(x)
    gx = 2.0 / SQRT_PI * np.exp(-x * x)       # d erf(x) / dx
    G = e / r
    G1 = (gx / R) / r - e / (r * r)
    G2 = (-2.0 * x * gx / (R * R)) / r - 2.0 * (gx / R) / (r * r) + 2.0 * e / (r ** 3)
    return G, G1, G2


def density(pos, Rq, Rmu, q, mu, points):
    """Induced charge density at points (M, 3) bohr: sum of Gaussian charges and
    Gaussian dipole densities.  q (N,) complex, mu (N, 3) complex or None."""
    pts = np.asarray(points, dtype=np.float64)
    rho = np.zeros(pts.shape[0], dtype=np.complex128)
    for i in range(pos.shape[0]):
        dx = pts - pos[i]
        r2 = np.einsum("mk,mk->m", dx, dx)
        gq = (np.pi * Rq[i] ** 2) ** -1.5 * np.exp(-r2 / Rq[i] ** 2)
        rho += q[i] * gq
        if mu is not None:
            gm = (np.pi * Rmu[i] ** 2) ** -1.5 * np.exp(-r2 / Rmu[i] ** 2)
            # -mu . grad g = (2 / R^2) (mu . x) g
            rho += (2.0 / Rmu[i] ** 2) * (dx @ mu[i]) * gm
    return rho


def potential(pos, Rq, Rmu, q, mu, points):
    """Induced potential phi at points (M, 3) bohr (Hartree atomic units)."""
    pts = np.asarray(points, dtype=np.float64)
    phi = np.zeros(pts.shape[0], dtype=np.complex128)
    for i in range(pos.shape[0]):
        dx = pts - pos[i]
        r = np.sqrt(np.einsum("mk,mk->m", dx, dx))
        at = r == 0.0
        rs = np.where(at, 1.0, r)
        G, G1, _ = _radial(rs, Rq[i])
        phi += q[i] * np.where(at, 2.0 / (SQRT_PI * Rq[i]), G)
        if mu is not None:
            _, G1m, _ = _radial(rs, Rmu[i])
            # -mu . grad G = -(mu . x / r) G'(r); zero at the centre (odd function)
            phi += np.where(at, 0.0, -(dx @ mu[i]) / rs * G1m)
    return phi


def field(pos, Rq, Rmu, q, mu, points):
    """Induced electric field E = -grad phi at points (M, 3) bohr; (M, 3) complex."""
    pts = np.asarray(points, dtype=np.float64)
    E = np.zeros(pts.shape, dtype=np.complex128)
    for i in range(pos.shape[0]):
        dx = pts - pos[i]
        r = np.sqrt(np.einsum("mk,mk->m", dx, dx))
        if np.any(r == 0.0):
            raise ValueError("probe point on an atom centre")
        u = dx / r[:, None]
        _, G1, _ = _radial(r, Rq[i])
        E += -q[i] * G1[:, None] * u                       # -grad (q G)
        if mu is not None:
            _, G1m, G2m = _radial(r, Rmu[i])
            # phi_mu = -(mu . u) G'(r);  E = grad((mu . u) G') =
            #   (mu . u) G'' u + G'/r (mu - (mu . u) u)
            mu_u = u @ mu[i]
            E += (mu_u * G2m)[:, None] * u + (G1m / r)[:, None] * (mu[i][None, :] - mu_u[:, None] * u)
    return E
