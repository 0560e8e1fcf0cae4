"""GPU parity of the boundary-element (DPCM, Sec. 2.3, Eq. 11) path against the FP64 oracle.

The library builds Ft once and solves (Ft - Lambda(w) I) sigma = -E0 e . n for every
frequency as a column shift, through the batched solver at every precision and through the
shifted Krylov solver.  These tests compare polarisabilities and tessera charges with the
oracle's dense LU on meshes spanning several 128-row tiles with a ragged tail, check the
sphere's closed form, the degenerate one- and two-tessera meshes, the error paths, and, on a
large mesh the oracle cannot factorise quickly, the FP64 residual of sampled rows computed
from the oracle's own rows of Ft.
"""
import math

import numpy as np
import pytest

from oracle import bem as BE
from oracle import model as M
from paper_2510_12731_gb300 import structures as S

pytestmark = pytest.mark.gpu


def _alpha_err(a, ref):
    return np.max(np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1))


def _solve(w, formulation="dpcm", **opts):
    from paper_2510_12731_gb300 import Solver
    with Solver(**opts) as s:
        s.set_mesh(w.pos_ang, w.normals, w.area_ang2, w.radius_ang, formulation)
        out = s.solve_bem(w.omega_ev, w.eps2, w.eps1, w.pol_dirs)
        st = s.stats()
    return out, st


CASES = [("fp64", "batched"), ("fp32", "batched"), ("bf16split", "batched"),
         ("fp16split", "batched"), ("fp32", "shifted")]


@pytest.mark.parametrize("precision,solver", CASES)
def test_bem_sphere_parity(precision, solver):
    """Drude sphere, 1000 tesserae (7 full row tiles + a 104-row tail), 12 frequencies
    across the dipolar resonance (condition numbers up to ~40)."""
    w = S.drude_sphere_mesh(1000, nfreq=12, wmin=2.5, wmax=4.5)
    ref_a, ref_q, _ = BE.solve(w.pos_ang, w.normals, w.area_ang2, w.eps2, w.eps1, w.pol_dirs,
                               radius_ang=w.radius_ang)
    out, st = _solve(w, precision=precision, solver=solver, tol_rel=1e-10)
    assert out["ok"] and np.all(out["rel_residual"] <= 1e-10)
    assert _alpha_err(out["alpha"], ref_a) <= 1e-7
    assert np.abs(out["q"] - ref_q).max() <= 1e-6 * np.abs(ref_q).max()
    assert st["solver_used"] == (1 if solver == "shifted" else 0)
    # sigma_abs = 4 pi w / (3c) Im Tr alpha for the x, y, z triple
    sig = M.sigma_abs(w.omega_ev / M.HARTREE_EV, np.einsum("fkk->f", ref_a).imag)
    assert np.allclose(out["sigma_abs"], sig, rtol=1e-6)


def _spheroid():
    pos, nrm, area = S.spheroid_mesh(700, 8.0, 8.0, 16.0)
    wv = np.linspace(2.0, 4.0, 9)
    pols = np.array([[1.0, 0.0, 0.0], [0.0, 0.6, 0.8], [0.0, 0.0, 1.0], [0.48, 0.6, 0.64]])
    return S.MeshWorkload("spheroid", pos, nrm, area, 16.0, wv, S.drude_eps(wv, 6.0, 0.15),
                          np.full(wv.size, 1.77 + 0j), pols)


@pytest.mark.parametrize("precision,solver", CASES)
def test_bem_spheroid_in_a_medium_parity(precision, solver):
    """Prolate spheroid 8 x 8 x 16 A, 700 tesserae, eps1 = 1.77 (water), oblique fields.
    Unlike the sphere's, the spheroid's operator is not symmetric: a matvec that applied
    its transpose would converge to a wrong answer with a small residual."""
    w = _spheroid()
    ref_a, ref_q, _ = BE.solve(w.pos_ang, w.normals, w.area_ang2, w.eps2, w.eps1, w.pol_dirs,
                               radius_ang=16.0)
    out, _ = _solve(w, precision=precision, solver=solver, tol_rel=1e-10)
    assert out["ok"]
    assert _alpha_err(out["alpha"], ref_a) <= 1e-7
    assert np.abs(out["q"] - ref_q).max() <= 1e-6 * np.abs(ref_q).max()
    assert "sigma_abs" not in out   # P = 4: no trace from four directions


@pytest.mark.parametrize("precision,solver", CASES)
def test_iefpcm_parity(precision, solver):
    """IEFPCM (Eq. 12) in two steps on the spheroid (4 oblique directions) and on the Drude
    sphere (x, y, z, sigma_abs), against the oracle's two dense LUs."""
    w = _spheroid()
    ref_a, ref_q, _ = BE.solve_iefpcm(w.pos_ang, w.normals, w.area_ang2, w.eps2, w.eps1,
                                      w.pol_dirs, radius_ang=16.0)
    out, st = _solve(w, "iefpcm", precision=precision, solver=solver, tol_rel=1e-10)
    assert out["ok"] and np.all(out["rel_residual"] <= 1e-10)
    assert _alpha_err(out["alpha"], ref_a) <= 1e-7
    assert np.abs(out["q"] - ref_q).max() <= 1e-6 * np.abs(ref_q).max()
    assert st["solver_used"] == (1 if solver == "shifted" else 0)
    w = S.drude_sphere_mesh(600, nfreq=8, wmin=2.5, wmax=4.5)
    ref_a, ref_q, _ = BE.solve_iefpcm(w.pos_ang, w.normals, w.area_ang2, w.eps2, w.eps1,
                                      w.pol_dirs, radius_ang=w.radius_ang)
    out, _ = _solve(w, "iefpcm", precision=precision, solver=solver, tol_rel=1e-10)
    assert out["ok"]
    assert _alpha_err(out["alpha"], ref_a) <= 1e-7
    sig = M.sigma_abs(w.omega_ev / M.HARTREE_EV, np.einsum("fkk->f", ref_a).imag)
    assert np.allclose(out["sigma_abs"], sig, rtol=1e-6)


def test_bem_sphere_closed_form():
    """3200 tesserae: alpha_xx approaches R^3 (e2 - e1)/(e2 + 2 e1) (as the oracle does)."""
    R = 20.0
    pos, nrm, area = S.sphere_mesh(3200, R)
    eps2 = np.array([-2.5 + 0.3j, 5.0 + 0.0j, -1.0 + 0.5j])
    w = S.MeshWorkload("sphere", pos, nrm, area, R, np.array([1.0, 2.0, 3.0]), eps2,
                       np.ones(3, dtype=np.complex128), np.eye(3))
    out, _ = _solve(w, precision="bf16split", tol_rel=1e-10)
    rb = R / M.BOHR_ANG
    exact = rb ** 3 * (eps2 - 1) / (eps2 + 2)
    assert np.abs(out["alpha"][:, 0, 0] / exact - 1).max() < 6e-3
    assert np.abs(out["alpha"][:, 0, 1]).max() < 1e-5 * np.abs(exact).max()


@pytest.mark.parametrize("n", [1, 2, 129])
def test_bem_degenerate_meshes(n):
    """One tessera (a 1 x 1 system), two, and one row past a full tile."""
    pos, nrm, area = S.sphere_mesh(n, 5.0)
    wv = np.array([2.0, 3.0, 3.5])
    w = S.MeshWorkload("tiny", pos, nrm, area, 5.0, wv, S.drude_eps(wv, 6.0, 0.2),
                       np.ones(3, dtype=np.complex128), np.eye(3))
    ref_a, ref_q, _ = BE.solve(pos, nrm, area, w.eps2, w.eps1, w.pol_dirs, radius_ang=5.0)
    for solver in ("batched", "shifted"):
        out, _ = _solve(w, precision="fp32", solver=solver, tol_rel=1e-10)
        scale = np.abs(ref_q).max()
        assert np.abs(out["q"] - ref_q).max() <= 1e-8 * scale
        assert np.abs(out["alpha"] - ref_a).max() <= 1e-8 * np.abs(ref_a).max()
    # FP64 with at most four real operand columns (the narrowest block matvec)
    w1 = S.MeshWorkload("tiny", pos, nrm, area, 5.0, wv[:2], w.eps2[:2], w.eps1[:2], np.eye(3)[:1])
    out, _ = _solve(w1, precision="fp64", tol_rel=1e-12)
    assert np.abs(out["q"] - ref_q[:2, :1]).max() <= 1e-10 * np.abs(ref_q).max()
    ref_a, ref_q, _ = BE.solve_iefpcm(pos, nrm, area, w.eps2, w.eps1, w.pol_dirs, radius_ang=5.0)
    for solver in ("batched", "shifted"):
        out, _ = _solve(w, "iefpcm", precision="fp32", solver=solver, tol_rel=1e-10)
        assert np.abs(out["q"] - ref_q).max() <= 1e-8 * np.abs(ref_q).max()


def test_bem_large_mesh_sampled_residuals():
    """16,000 tesserae, 60 frequencies: shifted and batched solutions agree, and the FP64
    residual of 64 sampled rows, from the oracle's rows of Ft, meets the tolerance."""
    w = S.drude_sphere_mesh(16000, nfreq=60, wmin=2.5, wmax=4.5)
    tol = 1e-8
    out_s, st = _solve(w, precision="fp32", solver="shifted", tol_rel=tol)
    out_b, _ = _solve(w, precision="bf16split", solver="batched", tol_rel=tol)
    assert out_s["ok"] and out_b["ok"] and st["solver_used"] == 1
    assert _alpha_err(out_s["alpha"], out_b["alpha"]) <= 1e-6
    rng = np.random.default_rng(7)
    rows = np.sort(rng.choice(16000, 64, replace=False))
    pos = w.pos_ang / M.BOHR_ANG
    area = w.area_ang2 / M.BOHR_ANG ** 2
    Fr = BE.f_rows(pos, w.normals, area, w.radius_ang / M.BOHR_ANG, rows)
    lam = BE.lam(w.eps2, w.eps1)
    b = -(w.normals @ w.pol_dirs.T)                               # (n, P)
    sig = out_s["q"] / area[None, None, :]                        # (F, P, n)
    r = b[rows].T[None] - (np.einsum("kn,fpn->fpk", Fr, sig) - lam[:, None, None] * sig[:, :, rows])
    # the row residuals are bounded by the global one times sqrt(n / rows) in the mean
    rel = np.linalg.norm(r, axis=2) / np.linalg.norm(b[rows], axis=0)[None]
    assert rel.max() <= 10 * tol
    # IEFPCM on the same mesh: both solvers for the first step agree
    i_s, st = _solve(w, "iefpcm", precision="fp32", solver="shifted", tol_rel=tol)
    i_b, _ = _solve(w, "iefpcm", precision="bf16split", solver="batched", tol_rel=tol)
    assert i_s["ok"] and i_b["ok"] and st["solver_used"] == 1
    assert _alpha_err(i_s["alpha"], i_b["alpha"]) <= 1e-6
    # DPCM and IEFPCM discretise the same continuum problem: close on a fine sphere
    assert _alpha_err(i_s["alpha"], out_s["alpha"]) <= 5e-3


def test_bem_error_paths():
    from paper_2510_12731_gb300 import PxError, Solver
    from paper_2510_12731_gb300 import _lib as L
    pos, nrm, area = S.sphere_mesh(200, 10.0)
    w = np.array([3.0])
    with Solver(precision="fp32") as s:
        with pytest.raises(PxError):                       # no mesh loaded
            s.solve_bem(w, [-2.0 + 0.2j], 1.0, np.eye(3))
        bad = nrm.copy()
        bad[3] *= 1.1
        with pytest.raises(PxError):                       # non-unit normal
            s.set_mesh(pos, bad, area, 10.0)
        with pytest.raises(PxError):                       # non-positive area
            s.set_mesh(pos, nrm, -area, 10.0)
        with pytest.raises(PxError):
            s.set_mesh(pos, nrm, area, 0.0)
        with pytest.raises(PxError):                       # unknown formulation
            s.set_mesh(pos, nrm, area, 10.0, 7)
        s.set_mesh(pos, nrm, area, 10.0)
        with pytest.raises(PxError):                       # e2 == e1
            s.solve_bem(w, [1.0 + 0j], 1.0, np.eye(3))
        with pytest.raises(PxError):                       # a mesh needs permittivities
            s.solve(w, np.eye(3))
        import torch
        d_q = torch.zeros((1, 3, 200), dtype=torch.complex128, device="cuda:0")
        with pytest.raises(PxError) as e:
            s.fields(np.zeros((4, 3)) + 30.0, d_q)
        assert e.value.status == L.PX_ENOTIMPL
        out = s.solve_bem(w, [-2.0 + 0.2j], 1.0, np.eye(3))
        assert out["ok"]
    with Solver(precision="fp32", mode="matfree") as s:
        with pytest.raises(PxError) as e:
            s.set_mesh(pos, nrm, area, 10.0)
        assert e.value.status == L.PX_ENOTIMPL


def test_bem_fresh_mesh_replaces_an_atomistic_structure():
    from paper_2510_12731_gb300 import PxError, Solver
    cl = S.small_cluster(element="Na", radius=8.0, model="wfq", nfreq=3, wmin=2.0, wmax=4.0)
    pos, nrm, area = S.sphere_mesh(300, 12.0)
    wv = np.array([2.0, 3.0])
    e2 = S.drude_eps(wv, 6.0, 0.2)
    with Solver(precision="fp32") as s:
        s.set_structure(cl.model, cl.xyz_ang, cl.type_idx, cl.types)
        with pytest.raises(PxError):                       # an atomistic structure is loaded
            s.solve_bem(wv, e2, 1.0, np.eye(3))
        a1 = s.solve(cl.omega_ev, cl.pol_dirs)["alpha"]
        s.set_mesh(pos, nrm, area, 12.0)
        out = s.solve_bem(wv, e2, 1.0, np.eye(3))
        s.set_structure(cl.model, cl.xyz_ang, cl.type_idx, cl.types)
        a2 = s.solve(cl.omega_ev, cl.pol_dirs)["alpha"]
    ref_a, _, _ = BE.solve(pos, nrm, area, e2, 1.0, np.eye(3), radius_ang=12.0)
    assert _alpha_err(out["alpha"], ref_a) <= 1e-7
    assert np.allclose(a1, a2, rtol=1e-12, atol=0)
    assert math.isfinite(out["sigma_abs"].sum())
