"""GPU parity of the shifted Krylov solver (PX_SOLVER_SHIFTED) against the FP64 oracle.

In Eq. 1 the frequency enters only through the scalar shift z_q(w) I (Eq. 6) and the
right-hand side does not depend on w, so the library runs one real Arnoldi process per
field direction for the whole sweep.  These tests compare its polarisabilities and
charges with the oracle's dense LU, check its relative residuals against an independent
FP64 recomputation from the returned charges (px_relres_device_noalloc), and cover the
edge cases: several direction groups (P > 4), a direction with a zero right-hand side, a
basis limit that hands columns to the batched refinement, wFQFmu (which stays batched),
and agreement with the batched solver.
"""
import numpy as np
import pytest

from oracle import model as M
from paper_2510_12731_gb300 import structures as S

pytestmark = pytest.mark.gpu


def _oracle(w):
    st = M.structure_from_types(w.xyz_ang, w.type_idx, w.types)
    return M.solve(st, w.model, w.omega_ev, w.pol_dirs, alpha_ib=w.alpha_ib)


def _alpha_err(a, ref):
    return np.max(np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1))


def _run(w, want_stats=True, **opts):
    from paper_2510_12731_gb300 import Solver
    with Solver(solver="shifted", **opts) as s:
        s.set_structure(w.model, w.xyz_ang, w.type_idx, w.types)
        out = s.solve(w.omega_ev, w.pol_dirs, w.alpha_ib)
        st = s.stats()
    return out, st


@pytest.mark.parametrize("element,radius,nfreq", [("Ag", 9.0, 12), ("Na", 12.0, 9)])
def test_shifted_small_sphere_parity(element, radius, nfreq):
    w = S.small_cluster(element=element, radius=radius, model="wfq", nfreq=nfreq, wmin=1.8,
                        wmax=5.5)
    ref = _oracle(w)
    out, st = _run(w, precision="fp32", tol_rel=1e-9)
    assert out["ok"] and np.all(out["rel_residual"] <= 1e-9)
    assert _alpha_err(out["alpha"], ref.alpha) <= 1e-7
    qerr = np.abs(out["q"] - ref.q).max() / np.abs(ref.q).max()
    assert qerr <= 1e-6
    assert st["solver_used"] == 1 and st["shift_steps"] > 0 and st["cycles"] == 0
    assert np.all(out["iters"] > 0) and np.all(out["iters"] <= st["shift_steps"])


def test_shifted_multi_tile_sphere_with_ragged_tail():
    """Na sphere r = 17 A: N = 537 atoms (5 row tiles of 128, the last ragged), 30 frequencies."""
    w = S.small_cluster(element="Na", radius=17.0, model="wfq", nfreq=30, wmin=2.0, wmax=4.5)
    assert w.natoms % 128 != 0 and w.natoms > 3 * 128
    ref = _oracle(w)
    out, st = _run(w, precision="fp32", tol_rel=1e-8)
    assert out["ok"]
    assert _alpha_err(out["alpha"], ref.alpha) <= 1e-6
    # sigma_abs of the x, y, z triple: 4 pi w / (3c) Tr Im alpha
    sig = M.sigma_abs(w.omega_ev / M.HARTREE_EV, np.einsum("fkk->f", ref.alpha).imag)
    assert np.allclose(out["sigma_abs"], sig, rtol=1e-6)


def test_shifted_residuals_match_an_independent_fp64_recomputation():
    import torch
    from paper_2510_12731_gb300 import Solver
    w = S.small_cluster(element="Ag", radius=10.0, model="wfq", nfreq=10, wmin=2.0, wmax=5.0)
    F, P, N = w.omega_ev.size, 3, w.natoms
    dev = torch.device("cuda", 0)
    d_q = torch.zeros((F, P, N), dtype=torch.complex128, device=dev)
    d_rr = torch.zeros((F, P), dtype=torch.float64, device=dev)
    d_rr2 = torch.zeros((F, P), dtype=torch.float64, device=dev)
    with Solver(solver="shifted", precision="fp32", tol_rel=1e-9) as s:
        s.set_structure(w.model, w.xyz_ang, w.type_idx, w.types)
        assert s.solve_device(w.omega_ev, w.pol_dirs, d_q=d_q, d_relres=d_rr)
        s.relres_device_noalloc(w.omega_ev, w.pol_dirs, d_q, d_rr2)
    a, b = d_rr.cpu().numpy(), d_rr2.cpu().numpy()
    assert np.all(a <= 1e-9) and np.all(b <= 1e-9)
    assert np.allclose(a, b, rtol=1e-4, atol=1e-12)


def test_shifted_two_direction_groups_and_a_zero_rhs_direction():
    """Five field directions (groups of 4 + 1); on a flat graphene flake the normal
    direction has no bond component, so its right-hand side is zero and x = 0."""
    el = S.ELEMENTS["C"]
    xyz = S.honeycomb_disk(el.a_ang, 20.0)
    pols = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [0.6, 0.8, 0], [0.8, 0, 0.6]], dtype=float)
    w = S.Workload("graphene_flake", "wfq", xyz, np.zeros(len(xyz), np.int32), [el.atom_type()],
                   np.linspace(0.2, 1.2, 8), pols, None)
    ref = _oracle(w)
    out, st = _run(w, precision="fp32", tol_rel=1e-9)
    assert out["ok"]
    assert np.abs(out["q"][:, 2]).max() == 0.0
    ok = np.linalg.norm(ref.alpha, axis=1) > 0
    err = np.linalg.norm(out["alpha"] - ref.alpha, axis=1)[ok] / np.linalg.norm(ref.alpha, axis=1)[ok]
    assert err.max() <= 1e-7


def test_shifted_basis_limit_hands_columns_to_refinement():
    w = S.small_cluster(element="Ag", radius=9.0, model="wfq", nfreq=6, wmin=2.0, wmax=5.0)
    ref = _oracle(w)
    out, st = _run(w, precision="fp32", tol_rel=1e-9, shift_krylov_max=12)
    assert out["ok"]
    assert st["shift_steps"] <= 3 * 12 and st["cycles"] > 0
    assert _alpha_err(out["alpha"], ref.alpha) <= 1e-7


def test_shifted_option_leaves_wfqfmu_batched():
    w = S.small_cluster(element="Ag", radius=7.0, model="wfqfmu", nfreq=4, wmin=2.5, wmax=5.0)
    ref = _oracle(w)
    out, st = _run(w, precision="fp32", tol_rel=1e-9)
    assert out["ok"] and st["solver_used"] == 0 and st["shift_steps"] == 0
    assert _alpha_err(out["alpha"], ref.alpha) <= 1e-7


def test_shifted_and_batched_agree():
    from paper_2510_12731_gb300 import Solver
    w = S.small_cluster(element="Na", radius=14.0, model="wfq", nfreq=20, wmin=2.0, wmax=4.0)
    outs = []
    for solver in ("batched", "shifted"):
        with Solver(solver=solver, precision="fp32", tol_rel=1e-10) as s:
            s.set_structure(w.model, w.xyz_ang, w.type_idx, w.types)
            outs.append(s.solve(w.omega_ev, w.pol_dirs))
    assert _alpha_err(outs[1]["alpha"], outs[0]["alpha"]) <= 1e-8


def test_shifted_after_fp64_structure_needs_new_set_structure():
    from paper_2510_12731_gb300 import PxError, Solver
    w = S.small_cluster(element="Ag", radius=6.0, model="wfq", nfreq=2, wmin=3.0, wmax=4.0)
    with Solver(precision="fp64") as s:
        s.set_structure(w.model, w.xyz_ang, w.type_idx, w.types)
        s.set_options(precision="fp64", solver="shifted")
        with pytest.raises(PxError, match="EINVAL.*before px_set_structure"):
            s.solve(w.omega_ev, w.pol_dirs)
        s.set_structure(w.model, w.xyz_ang, w.type_idx, w.types)
        assert s.solve(w.omega_ev, w.pol_dirs)["ok"]
