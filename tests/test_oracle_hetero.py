"""Pins of the heterogeneous wFQFmu oracle (oracle/hetero.py, Eqs. 9-10): it reduces to
Eq. 7 for one atom type and for two identical types, conserves the induced charge for a
genuinely mixed structure (which fixes the index order of H and the per-atom z_q), keeps
alpha^IB when both types share it, and counts twelve first-shell neighbours inside an
fcc alloy."""
import numpy as np

from oracle import hetero as HT
from oracle import model as M
from paper_2510_12731_gb300 import structures as S

W_EV = np.array([2.7, 3.6])
XYZ = np.eye(3)


def _alloy(n_atoms_radius=6.0, seed=5):
    """Ag/Au fcc sphere (a = 4.09 A) with seeded random substitution."""
    xyz = S.sphere("fcc", 4.09, n_atoms_radius)
    rng = np.random.default_rng(seed)
    tidx = (rng.random(len(xyz)) < 0.4).astype(np.int64)
    return xyz, tidx


def test_single_type_reduces_to_eq7():
    el = S.ELEMENTS["Ag"]
    xyz = S.sphere("fcc", 4.09, 6.0)
    tidx = np.zeros(len(xyz), np.int64)
    t = [el.atom_type()]
    aib = el.alpha_ib(W_EV)[None, :]
    a, q, mu, rel = HT.solve(xyz, tidx, t, W_EV, XYZ, aib)
    ref = M.solve(M.structure_from_types(xyz, tidx, t), "wfqfmu", W_EV, XYZ, alpha_ib=aib)
    assert np.abs(a - ref.alpha).max() <= 1e-11 * np.abs(ref.alpha).max()
    assert np.abs(q - ref.q).max() <= 1e-10 * np.abs(ref.q).max()
    assert rel.max() < 1e-10


def test_two_identical_types_reduce_to_eq7():
    """Two types with the same parameters: H = K^T = K (uniform area), alpha^IB_hetero =
    alpha^IB, so the mixed labelling changes nothing."""
    el = S.ELEMENTS["Ag"]
    xyz, tidx = _alloy()
    t = [el.atom_type(), el.atom_type()]
    aib1 = el.alpha_ib(W_EV)
    a, q, _, _ = HT.solve(xyz, tidx, t, W_EV, XYZ, np.stack([aib1, aib1]))
    ref = M.solve(M.structure_from_types(xyz, np.zeros_like(tidx), t[:1]), "wfqfmu", W_EV,
                  XYZ, alpha_ib=aib1[None, :])
    assert np.abs(a - ref.alpha).max() <= 1e-11 * np.abs(ref.alpha).max()


def test_mixed_structure_conserves_charge():
    """Ag/Au alloy with different n, tau, effective area and alpha^IB: the bond
    conductance D_i K_ij + D_j K_ji is symmetric only with H_ij proportional to K_ji and
    the row atom's z_q, so sum_i q_i = 0 pins both (it fails with K_ij in H, or with one
    type's z_q for all atoms)."""
    ag, au = S.ELEMENTS["Ag"], S.ELEMENTS["Au"]
    t_ag = ag.atom_type()
    t_au = {**au.atom_type(), "tau_au": 0.5 * au.atom_type()["tau_au"],
            "drude_n_au": 1.3 * au.atom_type()["drude_n_au"]}
    xyz, tidx = _alloy()
    aib = np.stack([ag.alpha_ib(W_EV), au.alpha_ib(W_EV)])
    _, q, _, rel = HT.solve(xyz, tidx, [t_ag, t_au], W_EV, XYZ, aib)
    assert rel.max() < 1e-10
    tot = np.abs(q.sum(axis=-1))
    assert np.all(tot <= 1e-10 * np.abs(q).sum(axis=-1))
    # a mis-ordered H (K_ij instead of K_ji) breaks it
    orig = HT.h_matrix
    try:
        HT.h_matrix = lambda K, n, tau, w: orig(K.T, n, tau, w)
        _, q_bad, _, _ = HT.solve(xyz, tidx, [t_ag, t_au], W_EV, XYZ, aib)
    finally:
        HT.h_matrix = orig
    assert np.any(np.abs(q_bad.sum(axis=-1)) > 1e-6 * np.abs(q_bad).sum(axis=-1))
    # so does one z_q (the first atom's n, tau) for every atom
    orig_z = HT.z_q_atoms
    try:
        HT.z_q_atoms = lambda w, n, tau: orig_z(w, np.full_like(n, n[0]), np.full_like(tau, tau[0]))
        _, q_bad, _, _ = HT.solve(xyz, tidx, [t_ag, t_au], W_EV, XYZ, aib)
    finally:
        HT.z_q_atoms = orig_z
    assert np.any(np.abs(q_bad.sum(axis=-1)) > 1e-6 * np.abs(q_bad).sum(axis=-1))


def test_alpha_ib_hetero_invariances():
    """Equal alpha^IB of both types is kept whatever the counts; an atom with no
    neighbours keeps its own type's value."""
    counts = np.array([[3, 9], [0, 0], [12, 0], [0, 12]])
    tidx = np.array([0, 1, 0, 1])
    a = np.array([2.0 + 0.5j, 2.0 + 0.5j])
    assert np.allclose(HT.alpha_ib_hetero(tidx, counts, a), a[0], rtol=1e-15)
    b = np.array([2.0 + 0.5j, 5.0 + 1.0j])
    out = HT.alpha_ib_hetero(tidx, counts, b)
    assert abs(out[1] - b[1]) <= 1e-15 * abs(b[1]) and abs(out[2] - b[0]) <= 1e-15 * abs(b[0])
    # between the two pure values for a mixed neighbourhood (harmonic-type mean)
    assert min(abs(b)) < abs(out[0]) < max(abs(b))


def test_fcc_alloy_bulk_atoms_have_twelve_neighbours():
    xyz, tidx = _alloy(n_atoms_radius=9.0)
    t = [S.ELEMENTS["Ag"].atom_type(), S.ELEMENTS["Au"].atom_type()]
    st, _, _ = HT.structure(xyz, tidx, t)
    counts = HT.neighbour_counts(st, 2)
    inner = np.linalg.norm(st.pos, axis=1) * M.BOHR_ANG < 9.0 - 3.0
    assert inner.sum() > 10
    assert np.all(counts[inner].sum(axis=1) == 12)
