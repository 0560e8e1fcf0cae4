"""GPU parity of the induced density / potential / field maps (px_fields) against the
oracle's maps (oracle/fields.py), on seeded charges and dipoles over a multi-tile
structure (kernel parity), on a solved structure (end to end), and against the exact
single-atom limits at the atom centre (Gaussian charge and dipole densities)."""
import math

import numpy as np
import pytest

from oracle import fields as FL
from oracle import model as M
from paper_2510_12731_gb300 import structures as S

pytestmark = pytest.mark.gpu


def _grid(xyz_ang, n=9, pad=4.0, z=None, shift=0.0):
    lo, hi = xyz_ang.min(axis=0) - pad + shift, xyz_ang.max(axis=0) + pad + shift
    ax = [np.linspace(lo[k], hi[k], n) for k in range(3)]
    if z is not None:
        ax[2] = np.array([z])
    X, Y, Z = np.meshgrid(*ax, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def _maps(w, points, q, mu):
    import torch
    from paper_2510_12731_gb300 import Solver
    dev = torch.device("cuda", 0)
    C = q.shape[0]
    M_ = points.shape[0]
    tq = torch.from_numpy(np.ascontiguousarray(q)).to(dev)
    tmu = torch.from_numpy(np.ascontiguousarray(mu)).to(dev) if mu is not None else None
    rho = torch.zeros((C, M_), dtype=torch.complex128, device=dev)
    phi = torch.zeros((C, M_), dtype=torch.complex128, device=dev)
    E = torch.zeros((C, M_, 3), dtype=torch.complex128, device=dev)
    with Solver(precision="fp32") as s:
        s.set_structure(w.model, w.xyz_ang, w.type_idx, w.types)
        s.fields(points, tq, d_mu=tmu, d_rho=rho, d_phi=phi, d_E=E)
    return rho.cpu().numpy(), phi.cpu().numpy(), E.cpu().numpy()


def _close(a, b, tol=2e-5):
    scale = np.abs(b).max()
    assert np.abs(a - b).max() <= tol * scale, np.abs(a - b).max() / scale


@pytest.mark.parametrize("model", ["wfq", "wfqfmu"])
def test_maps_match_oracle_on_seeded_charges(model):
    """Ag sphere r = 9 A (177 atoms: two 128-atom tiles, the second ragged), 3 columns of
    seeded complex charges (and dipoles), 729 probe points around it (6 blocks of 128,
    the last ragged)."""
    w = S.small_cluster(element="Ag", radius=9.0, model=model, nfreq=1)
    rng = np.random.default_rng(12731)
    N, C = w.natoms, 3
    q = rng.normal(size=(C, N)) + 1j * rng.normal(size=(C, N))
    mu = (rng.normal(size=(C, N, 3)) + 1j * rng.normal(size=(C, N, 3))) if model == "wfqfmu" else None
    pts = _grid(w.xyz_ang, shift=0.37)          # off the atom centres (the oracle's field
    rho, phi, E = _maps(w, pts, q, mu)          # is undefined there)
    st = M.structure_from_types(w.xyz_ang, w.type_idx, w.types)
    pb = pts / M.BOHR_ANG
    for c in range(C):
        m = None if mu is None else mu[c]
        _close(rho[c], FL.density(st.pos, st.Rq, st.Rmu, q[c], m, pb))
        _close(phi[c], FL.potential(st.pos, st.Rq, st.Rmu, q[c], m, pb))
        _close(E[c], FL.field(st.pos, st.Rq, st.Rmu, q[c], m, pb))


def test_maps_of_a_solved_sphere_end_to_end():
    """Charges solved by the library at the plasmon peak; maps in the z = 0 plane through
    the atom centres (the centre atom sits on a probe point) against the oracle's maps of
    the oracle's own LU charges."""
    import torch
    from paper_2510_12731_gb300 import Solver
    w = S.small_cluster(element="Na", radius=12.0, model="wfq", nfreq=1, wmin=3.3, wmax=3.3,
                        pols=S.X_ONLY)
    dev = torch.device("cuda", 0)
    d_q = torch.zeros((1, 1, w.natoms), dtype=torch.complex128, device=dev)
    pts = _grid(w.xyz_ang, n=21, z=0.0)
    pts = pts[np.abs(pts).sum(axis=1) > 0]
    pts = np.concatenate([pts, np.zeros((1, 3))])       # the centre atom
    phi = torch.zeros((1, pts.shape[0]), dtype=torch.complex128, device=dev)
    rho = torch.zeros_like(phi)
    with Solver(precision="fp32", tol_rel=1e-10) as s:
        s.set_structure(w.model, w.xyz_ang, w.type_idx, w.types)
        assert s.solve_device(w.omega_ev, w.pol_dirs, d_q=d_q)
        s.fields(pts, d_q, d_rho=rho, d_phi=phi)
    st = M.structure_from_types(w.xyz_ang, w.type_idx, w.types)
    ref = M.solve(st, "wfq", w.omega_ev, w.pol_dirs)
    pb = pts / M.BOHR_ANG
    _close(phi.cpu().numpy()[0], FL.potential(st.pos, st.Rq, st.Rmu, ref.q[0, 0], None, pb), 1e-4)
    _close(rho.cpu().numpy()[0], FL.density(st.pos, st.Rq, st.Rmu, ref.q[0, 0], None, pb), 1e-4)


def test_single_atom_limits_at_its_centre():
    """At the centre of one Gaussian charge q (width R_q) and dipole mu (width R_mu):
    rho = q / (pi R_q^2)^(3/2), phi = 2 q / (sqrt(pi) R_q), E = -4 mu / (3 sqrt(pi) R_mu^3)
    (the charge's field vanishes there; the dipole's self-field is uniform)."""
    w = S.small_cluster(element="Au", radius=0.5, model="wfqfmu", nfreq=1)
    assert w.natoms == 1
    q = np.array([[0.3 - 0.7j]])
    mu = np.array([[[0.2 + 0.1j, -0.5 + 0.0j, 0.9 - 0.3j]]])
    rho, phi, E = _maps(w, np.zeros((1, 3)), q, mu)
    t = w.types[0]
    Rq, Rm = t["Rq_bohr"], t["Rmu_bohr"]
    assert rho[0, 0] == pytest.approx(q[0, 0] / (math.pi * Rq * Rq) ** 1.5, rel=1e-5)
    assert phi[0, 0] == pytest.approx(2.0 * q[0, 0] / (math.sqrt(math.pi) * Rq), rel=1e-5)
    expect = -4.0 / (3.0 * math.sqrt(math.pi) * Rm ** 3) * mu[0, 0]
    assert np.abs(E[0, 0] - expect).max() <= 1e-5 * np.abs(expect).max()


def test_fields_rejects_dipoles_for_wfq():
    import torch
    from paper_2510_12731_gb300 import PxError, Solver
    w = S.small_cluster(element="Ag", radius=6.0, model="wfq", nfreq=1)
    dev = torch.device("cuda", 0)
    q = torch.zeros((1, w.natoms), dtype=torch.complex128, device=dev)
    mu = torch.zeros((1, w.natoms, 3), dtype=torch.complex128, device=dev)
    with Solver(precision="fp32") as s:
        s.set_structure(w.model, w.xyz_ang, w.type_idx, w.types)
        with pytest.raises(PxError, match="EINVAL"):
            s.fields(np.zeros((2, 3)), q, d_mu=mu)
