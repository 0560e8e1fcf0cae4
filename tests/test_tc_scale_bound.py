"""The power-of-two scale of the tensor-core pair kernels (FP16 split).

The on-the-fly kernels generate 2^e T in FP32 and cut it into FP16 parts, with e chosen on
the host before any entry exists: 2^e * bound <= 2^14, where the bound on max|T| comes from
the smallest charge and dipole widths alone.  These checks hold that bound against every
entry of the oracle's kernels (Eq. 5 for wFQ; the T^qq / T^qmu / T^muq / T^mumu blocks of
Sec. 2.2 for wFQFmu, with the Gaussian dipole self term), so that no generated entry can
leave the FP16 range, and pin the radial constants the bound is built from.
"""
import math

import numpy as np
import pytest

from oracle import model as M


def _bound(types, model):
    """max|T| bound of the pair kernels' scale: the T^qq diagonal sqrt(2/pi)/R_q; for
    wFQFmu also 0.5 / (R_q^2 + R_mu^2) (T^qmu, T^muq) and 1 / (2 R_mu^2)^(3/2) (T^mumu)."""
    rq = min(t["Rq_bohr"] for t in types)
    rm = min(t["Rmu_bohr"] for t in types)
    b = math.sqrt(2.0 / math.pi) / rq
    if model == "wfqfmu":
        b = max(b, 0.5 / (rq * rq + rm * rm), 1.0 / (2.0 * rm * rm) ** 1.5)
    return b


def _types(rq, rm):
    base = dict(r0_ang=2.88, d=12.0, s=1.1, area_bohr2=5.0, drude_n_au=0.0086, tau_au=3000.0)
    return [dict(base, Rq_bohr=a, Rmu_bohr=b) for a, b in zip(rq, rm)]


def test_radial_constants_of_the_bound():
    """With x = r/R: |d/dx (erf x / x)| <= 0.43, |G'/r| and |G''| <= 0.76 / R^3."""
    R = 1.0
    r = np.linspace(1e-3, 12.0, 240001)
    t1 = M.gauss_T1(r, R)
    t2 = M.gauss_T2(r, R)
    assert np.abs(t1).max() <= 0.43
    # the small-r limit of both is -4 / (3 sqrt(pi)) = -0.752; away from it they are smaller
    assert np.abs(t1 / r).max() <= 0.76
    assert np.abs(t2[r > 1e-2]).max() <= 0.76


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("model", ["wfq", "wfqfmu"])
def test_every_kernel_entry_is_below_the_scale_bound(seed, model):
    """Random clusters of two atom types with unequal charge and dipole widths, spacings
    down to a fifth of the widths (closer than any lattice), the dipole self term on."""
    rng = np.random.default_rng(seed)
    rq = rng.uniform(1.2, 3.5, 2)
    rm = rng.uniform(1.2, 3.5, 2)
    types = _types(rq, rm)
    n = 60
    # a random walk of steps 0.2 .. 2 bohr, so that many pairs are well inside R
    steps = rng.normal(size=(n, 3))
    steps *= (rng.uniform(0.2, 2.0, n) / np.linalg.norm(steps, axis=1))[:, None]
    xyz_ang = np.cumsum(steps, axis=0) * M.BOHR_ANG
    st = M.structure_from_types(xyz_ang, rng.integers(0, 2, n), types)
    T = M.tqq(st) if model == "wfq" else M.t_full(st, mu_self_term=True)
    b = _bound(types, model)
    assert np.isfinite(T).all()
    assert np.abs(T).max() <= b
    # the bound is not loose by more than the margins taken (a factor of about 2)
    assert np.abs(T).max() >= 0.25 * b
