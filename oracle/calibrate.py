"""Effective-area calibration for the parameter presets (test infrastructure).

The paper gives A_i of Eq. 3 only as "the effective area of atom i" and prints
no values.  The presets use the area for which the bond network of an infinite
lattice, driven by a uniform field, carries the Drude current of the continuum:
with G_ij = 2 sigma(w) K_ij (the conductance that Eqs. 1 and 6 imply), the
bond currents of a uniform field give

    3D (cubic):    sigma_eff = sigma/(3 Omega)   * A * sum_j (1 - f(r_j)) r_j
    2D (isotropic): sigma_eff = sigma/(2 Omega2) * A * sum_j (1 - f(r_j)) r_j

so A = 3 Omega / S (3D) or A = 2 Omega2 / S (2D), S = sum_j (1 - f(r_j)) r_j over
the neighbours of one atom (Omega: volume per atom, Omega2: area per atom).

Running ``python -m oracle.calibrate`` prints the values that
``paper_2510_12731_gb300/structures.py`` stores as literals; a CPU test checks
that the stored literals equal this computation.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import model


def _lattice_sum(points, r0, d, s):
    r = np.linalg.norm(points, axis=1)
    r = r[(r > 1e-9) & (r < 6.0 * r0)]
    return float(np.sum((1.0 - model.fermi(r, r0, d, s)) * r))


def _cubic_points(a, basis, reach=8):
    rng = range(-reach, reach + 1)
    cells = np.array(list(itertools.product(rng, rng, rng)), dtype=np.float64)
    return (cells[:, None, :] + np.asarray(basis)[None, :, :]).reshape(-1, 3) * a


def area_fcc(a_bohr, d=12.0, s=1.1):
    """A for an fcc lattice of cube edge a (r0 = a/sqrt2, Omega = a^3/4)."""
    pts = _cubic_points(a_bohr, [[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    r0 = a_bohr / np.sqrt(2.0)
    return 3.0 * (a_bohr ** 3 / 4.0) / _lattice_sum(pts, r0, d, s)


def area_bcc(a_bohr, d=12.0, s=1.1):
    """A for a bcc lattice of cube edge a (r0 = a sqrt3/2, Omega = a^3/2)."""
    pts = _cubic_points(a_bohr, [[0, 0, 0], [0.5, 0.5, 0.5]])
    r0 = a_bohr * np.sqrt(3.0) / 2.0
    return 3.0 * (a_bohr ** 3 / 2.0) / _lattice_sum(pts, r0, d, s)


def area_honeycomb(acc_bohr, d=12.0, s=1.1, reach=12):
    """A for a honeycomb sheet of bond length acc (Omega2 = 3 sqrt3/4 acc^2)."""
    a1 = np.array([1.5, np.sqrt(3.0) / 2.0]) * acc_bohr
    a2 = np.array([1.5, -np.sqrt(3.0) / 2.0]) * acc_bohr
    basis = [np.zeros(2), np.array([acc_bohr, 0.0])]
    pts = []
    for i in range(-reach, reach + 1):
        for j in range(-reach, reach + 1):
            for b in basis:
                pts.append(i * a1 + j * a2 + b)
    pts = np.array(pts)
    pts3 = np.concatenate([pts, np.zeros((len(pts), 1))], axis=1)
    omega2 = 3.0 * np.sqrt(3.0) / 4.0 * acc_bohr ** 2
    return 2.0 * omega2 / _lattice_sum(pts3, acc_bohr, d, s)


def preset_areas():
    """Areas (bohr^2) of the four lattices used by the synthetic workloads."""
    B = model.BOHR_ANG
    return {
        "Ag": area_fcc(4.09 / B),
        "Au": area_fcc(4.08 / B),
        "Na": area_bcc(4.23 / B),
        "C": float(area_honeycomb(1.42 / B)),
    }


if __name__ == "__main__":
    for k, v in preset_areas().items():
        print(f"{k}: {v!r}")
