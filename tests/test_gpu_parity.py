"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Sizes span several 128-row tiles with a ragged tail and ragged column blocks;
edge cases cover the degenerate structures of the method.
"""
import math

import numpy as np
import pytest

from oracle import model as M
from paper_2510_12731_gb300 import structures as S

pytestmark = pytest.mark.gpu

XYZ = np.eye(3)


def _solver(**kw):
    from paper_2510_12731_gb300 import Solver
    return Solver(**kw)


def _oracle(w, **kw):
    st = M.structure_from_types(w.xyz_ang, w.type_idx, w.types)
    return M.solve(st, w.model, w.omega_ev, w.pol_dirs, alpha_ib=w.alpha_ib, **kw), st


def _rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def _run(w, **opts):
    with _solver(**opts) as s:
        s.set_structure(w.model, w.xyz_ang, w.type_idx, w.types)
        out = s.solve(w.omega_ev, w.pol_dirs, w.alpha_ib)
        stats = s.stats()
    return out, stats


def _alpha_err(out, ref):
    """max over (w, pol) of |alpha_gpu - alpha_ref| / |alpha_ref| (the field-direction column)."""
    a, r = out["alpha"], ref.alpha
    num = np.linalg.norm(a - r, axis=1)
    den = np.linalg.norm(r, axis=1)
    return float(np.max(num / den))


@pytest.mark.parametrize("model", ["wfq", "wfqfmu"])
@pytest.mark.parametrize("precision,tol,alpha_tol", [("fp64", 1e-10, 1e-8), ("fp32", 1e-9, 1e-7)])
def test_small_sphere_parity(model, precision, tol, alpha_tol):
    # Ag sphere r = 9 A: N = 225 atoms (2 row tiles, ragged), 7 w x 3 pols = 21 columns
    w = S.small_cluster(element="Ag", radius=9.0, model=model, nfreq=7, wmin=2.0, wmax=5.5)
    ref, st = _oracle(w)
    out, stats = _run(w, precision=precision, tol_rel=tol)
    assert out["ok"], out["rel_residual"]
    assert np.all(out["rel_residual"] <= tol)
    assert _alpha_err(out, ref) <= alpha_tol
    qerr = np.abs(out["q"] - ref.q).max() / np.abs(ref.q).max()
    assert qerr <= 10 * alpha_tol
    if model == "wfqfmu":
        merr = np.abs(out["mu"] - ref.mu).max() / np.abs(ref.mu).max()
        assert merr <= 10 * alpha_tol
    # charge conservation and reciprocity on the GPU outputs
    assert np.all(np.abs(out["q"].sum(axis=-1)) <= 1e-9 * np.abs(out["q"]).sum(axis=-1))
    for f in range(w.omega_ev.size):
        a = out["alpha"][f]
        assert np.abs(a - a.T).max() <= 1e-6 * np.abs(a).max()
    assert stats["kernel_launches"] > 0


def test_ag_sphere_791_fp64_sweep():
    """wFQ Ag fcc sphere r = 15 A (N = 791), 60 w in 2.0-4.5 eV, x-polarised, plain FP64."""
    w = S.ag_sphere_791()
    ref, _ = _oracle(w)
    out, _ = _run(w, precision="fp64", tol_rel=1e-10)
    assert out["ok"]
    assert _alpha_err(out, ref) <= 1e-8
    sig_ref = ref.sigma_abs_pol
    assert np.abs(out["sigma_abs_pol"] - sig_ref).max() <= 1e-8 * np.abs(sig_ref).max()


def test_ag_sphere_791_fp32_meets_1e5():
    w = S.ag_sphere_791()
    ref, _ = _oracle(w)
    out, stats = _run(w, precision="fp32", tol_rel=1e-7)
    assert out["ok"]
    assert _alpha_err(out, ref) <= 1e-5


def test_sigma_abs_three_polarisations():
    w = S.small_cluster(element="Na", radius=10.0, model="wfq", nfreq=5, wmin=2.5, wmax=4.0)
    ref, st = _oracle(w)
    out, _ = _run(w, precision="fp64", tol_rel=1e-11)
    om = w.omega_ev / M.HARTREE_EV
    tr = np.einsum("fkk->f", ref.alpha).imag
    sig = M.sigma_abs(om, tr)
    assert np.allclose(out["sigma_abs"], sig, rtol=1e-8, atol=0)


@pytest.mark.parametrize("model", ["wfq", "wfqfmu"])
def test_sigma_abs_rotated_and_skewed_triples(model):
    """Tr Im alpha from any three linearly independent field directions (alpha = A E^-1):
    a rotated orthonormal triple and a skewed one give the x, y, z orientation average."""
    w = S.small_cluster(element="Ag", radius=8.0, model=model, nfreq=4, wmin=2.5, wmax=5.0)
    ref, st = _oracle(w)
    sig = M.sigma_abs(w.omega_ev / M.HARTREE_EV, np.einsum("fkk->f", ref.alpha).imag)
    a, b = 0.7, -0.4
    Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, np.cos(b), -np.sin(b)], [0, np.sin(b), np.cos(b)]])
    skew = np.array([[1.0, 0.0, 0.0], [0.6, 0.8, 0.0], [0.0, 0.6, 0.8]])
    for E in ((Rz @ Rx).T, skew):
        with _solver(precision="fp64", tol_rel=1e-11) as s:
            s.set_structure(w.model, w.xyz_ang, w.type_idx, w.types)
            out = s.solve(w.omega_ev, E, w.alpha_ib)
        assert out["ok"]
        assert np.allclose(out["sigma_abs"], sig, rtol=1e-8, atol=0)


def test_sigma_abs_rejects_linearly_dependent_triple():
    from paper_2510_12731_gb300 import PxError
    w = S.small_cluster(element="Ag", radius=6.0, model="wfq", nfreq=2, wmin=3.0, wmax=4.0)
    xxy = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    with _solver(precision="fp64") as s:
        s.set_structure(w.model, w.xyz_ang, w.type_idx, w.types)
        with pytest.raises(PxError, match="EINVAL.*linearly independent"):
            s.solve(w.omega_ev, xxy, w.alpha_ib)
        # without sigma_abs the same directions are a valid request
        d = s.solve(w.omega_ev, xxy, w.alpha_ib, out={**s.alloc_outputs(2, 3), "sigma_abs": None})
        assert d["ok"]


# ------------------------------------------------------------------ edge cases

def _single(model, xyz, element="Ag", nfreq=3):
    el = S.ELEMENTS[element]
    om = np.linspace(2.5, 4.0, nfreq)
    aib = el.alpha_ib(om)[None, :] if model == "wfqfmu" else None
    return S.Workload("edge", model, np.asarray(xyz, float), np.zeros(len(xyz), np.int32),
                      [el.atom_type()], om, XYZ, aib)


def test_single_atom_wfq_has_zero_response():
    w = _single("wfq", [[0.0, 0.0, 0.0]])
    out, _ = _run(w, precision="fp64")
    assert out["ok"]
    assert np.abs(out["alpha"]).max() == 0.0


def test_single_atom_wfqfmu_is_interband_polarisability():
    w = _single("wfqfmu", [[0.0, 0.0, 0.0]])
    out, _ = _run(w, precision="fp64", tol_rel=1e-12)
    for f in range(3):
        assert np.allclose(out["alpha"][f], w.alpha_ib[0, f] * np.eye(3), rtol=1e-12, atol=0)


def test_two_atom_closed_form_on_gpu():
    d_ang = 2.892
    w = _single("wfq", [[-d_ang / 2, 0, 0], [d_ang / 2, 0, 0]])
    ref, _ = _oracle(w)
    out, _ = _run(w, precision="fp32", tol_rel=1e-12)
    assert out["ok"]
    axx, rxx = out["alpha"][:, 0, 0], ref.alpha[:, 0, 0]
    assert np.abs(axx - rxx).max() <= 1e-10 * np.abs(rxx).max()
    assert np.abs(out["alpha"][:, 1:, 1:]).max() <= 1e-12 * np.abs(rxx).max()


def test_graphene_field_normal_to_sheet_has_zero_rhs():
    el = S.ELEMENTS["C"]
    xyz = S.honeycomb_disk(1.42, 16.0)
    om = np.linspace(0.2, 0.8, 4)
    w = S.Workload("g", "wfq", xyz, np.zeros(len(xyz), np.int32), [el.atom_type()], om,
                   np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0]]), None)
    ref, _ = _oracle(w)
    out, _ = _run(w, precision="fp64", tol_rel=1e-10)
    assert out["ok"]
    assert np.abs(out["alpha"][:, :, 0]).max() == 0.0
    assert _alpha_err({"alpha": out["alpha"][:, :, 1:]}, type("R", (), {"alpha": ref.alpha[:, :, 1:]})) <= 1e-8


def test_invalid_inputs_are_rejected():
    from paper_2510_12731_gb300 import PxError
    el = S.ELEMENTS["Ag"]
    with _solver() as s:
        with pytest.raises(PxError, match="EINVAL"):
            s.set_structure("wfq", [[0, 0, 0], [0, 0, 0]], [0, 0], [el.atom_type()])
        with pytest.raises(PxError, match="EINVAL"):
            s.set_structure("wfq", [[0, 0, float("nan")]], [0], [el.atom_type()])
        with pytest.raises(PxError, match="EINVAL"):
            s.set_structure("wfq", [[0, 0, 0]], [1], [el.atom_type()])
        s.set_structure("wfq", [[0, 0, 0], [2.9, 0, 0]], [0, 0], [el.atom_type()])
        with pytest.raises(PxError, match="EINVAL"):
            s.solve([-1.0], XYZ)
        with pytest.raises(PxError, match="EINVAL"):
            s.solve([2.0], [[1.0, 1.0, 0.0]])


def test_not_converged_is_reported():
    w = S.small_cluster(element="Ag", radius=9.0, model="wfq", nfreq=3, wmin=2.0, wmax=3.0)
    out, _ = _run(w, precision="fp64", tol_rel=1e-12, max_iter=2, restart_m=2)
    assert not out["ok"]
    assert np.any(out["status"] == 3)


# ------------------------------------------------------------------ tensor-core BF16 split

@pytest.mark.parametrize("model", ["wfq", "wfqfmu"])
def test_bf16split_parity_after_refinement(model):
    # N = 225 (2 row tiles of 128, ragged); 50 w x 3 pols = 150 columns -> 300 real
    # operand columns, padded to 384 -> 3 column tiles of 128 (ragged)
    w = S.small_cluster(element="Ag", radius=9.0, model=model, nfreq=50, wmin=2.0, wmax=5.5)
    ref, _ = _oracle(w)
    out, stats = _run(w, precision="bf16split", tol_rel=1e-9)
    assert out["ok"]
    assert _alpha_err(out, ref) <= 1e-6
    assert stats["used_precision"] == 2


@pytest.mark.parametrize("model", ["wfq", "wfqfmu"])
def test_bf16split_before_refinement_within_1e3(model):
    """One low-precision round (no FP64 refinement): the BF16-split operator alone."""
    w = S.small_cluster(element="Ag", radius=9.0, model=model, nfreq=12, wmin=2.0, wmax=5.5)
    ref, _ = _oracle(w)
    out, _ = _run(w, precision="bf16split", tol_rel=1e-9, inner_tol=1e-8, max_refine=0,
                  restart_m=200, basis="ff32")
    assert _alpha_err(out, ref) <= 1e-3


def test_bf16split_multi_k_tiles_sphere():
    """Na sphere r = 20 A (N = 893: 7 row tiles, 14 K steps), 40 w x 3 pols."""
    w = S.small_cluster(element="Na", radius=20.0, model="wfq", nfreq=40, wmin=2.0, wmax=4.0)
    w.tol = 1e-8
    st = M.structure_from_types(w.xyz_ang, w.type_idx, w.types)
    from oracle import spectral as SP
    md = SP.modes(st)
    a_ref = SP.alpha(st, md, w.omega_ev, w.pol_dirs)
    out, _ = _run(w, precision="bf16split", tol_rel=1e-8)
    assert out["ok"]
    num = np.linalg.norm(out["alpha"] - a_ref, axis=1)
    den = np.linalg.norm(a_ref, axis=1)
    assert np.max(num / den) <= 1e-5


@pytest.mark.parametrize("model", ["wfq", "wfqfmu"])
def test_fp16split_parity(model):
    w = S.small_cluster(element="Ag", radius=9.0, model=model, nfreq=50, wmin=2.0, wmax=5.5)
    ref, _ = _oracle(w)
    out, stats = _run(w, precision="fp16split", tol_rel=1e-9)
    assert out["ok"]
    assert _alpha_err(out, ref) <= 1e-6
    assert stats["used_precision"] == 3


@pytest.mark.parametrize("model", ["wfq", "wfqfmu"])
def test_fp16split_narrow_gaussians(model):
    """The tensor-core operator M = diag(Kbar, I) T gets its fp16 scale from max |M|, so
    narrow Gaussian widths (large T entries, R_q = R_mu = 0.4 bohr) still meet the
    parity bar after refinement."""
    w = S.small_cluster(element="Ag", radius=9.0, model=model, nfreq=12, wmin=2.0, wmax=5.5)
    w.types = [{**t, "Rq_bohr": 0.4, "Rmu_bohr": 0.4} for t in w.types]
    ref, _ = _oracle(w)
    out, _ = _run(w, precision="fp16split", tol_rel=1e-9)
    assert out["ok"]
    assert _alpha_err(out, ref) <= 1e-6


@pytest.mark.parametrize("model", ["wfq", "wfqfmu"])
def test_fp16split_before_refinement_beats_bf16split(model):
    """One low-precision round (no FP64 refinement): the scaled FP16 split keeps ~22
    bits per product against the BF16 split's ~16, so its unrefined alpha is closer to
    the oracle (at least 2x; the operator M = diag(Kbar, I) T is formed in FP64, so
    neither split loses bits to Kbar's neighbour differences), and within 1e-4."""
    w = S.small_cluster(element="Ag", radius=9.0, model=model, nfreq=12, wmin=2.0, wmax=5.5)
    ref, _ = _oracle(w)
    kw = dict(tol_rel=1e-9, inner_tol=1e-8, max_refine=0, restart_m=200, basis="ff32")
    e16 = _alpha_err(_run(w, precision="fp16split", **kw)[0], ref)
    ebf = _alpha_err(_run(w, precision="bf16split", **kw)[0], ref)
    assert e16 <= 1e-4
    assert e16 <= ebf / 2


# ------------------------------------------------------------------ tensor-core tile variants

@pytest.mark.parametrize("precision", ["bf16split", "fp16split"])
def test_gemm_tile_variants_are_bit_identical(precision):
    """128 x 256 and 128 x 128 tiles accumulate every output's K products in the same
    order, so the whole solve (deterministic reductions) gives bit-identical results;
    the autotuned default picks one of them."""
    # Na sphere r = 20 A: N = 893 (7 row tiles, ragged); 64 w x 2 pols = 128 columns ->
    # 256 real operand columns in the first cycle: 1 column tile of 256 or 2 of 128
    w = S.small_cluster(element="Na", radius=20.0, model="wfq", nfreq=64, wmin=2.0, wmax=4.0)
    w.pol_dirs = w.pol_dirs[:2]
    outs = []
    for tiles in (1, 2, 0):
        out, stats = _run(w, precision=precision, tol_rel=1e-8, gemm_tiles=tiles)
        assert out["ok"]
        assert stats["gemm_tiles_used"] in ((tiles,) if tiles else (1, 2))
        outs.append(out)
    for o in outs[1:]:
        assert np.array_equal(o["alpha"], outs[0]["alpha"])
        assert np.array_equal(o["iters"], outs[0]["iters"])


def test_gemm_tiles_fall_back_to_128_columns_when_256_do_not_fit():
    """64 w x 3 pols = 192 columns -> 384 real operand columns, not a multiple of 256:
    asking for 128 x 256 tiles runs 128 x 128 tiles, with results identical to asking
    for those directly."""
    w = S.small_cluster(element="Na", radius=20.0, model="wfq", nfreq=64, wmin=2.0, wmax=4.0)
    a, st_a = _run(w, precision="fp16split", tol_rel=1e-8, gemm_tiles=1)
    b, st_b = _run(w, precision="fp16split", tol_rel=1e-8, gemm_tiles=2)
    assert st_a["gemm_tiles_used"] == 2 and st_b["gemm_tiles_used"] == 2
    assert a["ok"] and np.array_equal(a["alpha"], b["alpha"])


# ------------------------------------------------------------------ restart cycles as graphs

@pytest.mark.parametrize("model,precision", [("wfq", "fp64"), ("wfq", "fp32"),
                                             ("wfq", "bf16split"), ("wfqfmu", "fp16split")])
def test_cycle_graphs_match_eager_launches(model, precision):
    """A restart cycle run as one graph launch (device-side loop over the Krylov steps)
    executes the same kernels on the same data as the eager per-step launches, so the
    results are bit-identical; the eager path runs at most one idle step more."""
    w = S.small_cluster(element="Ag", radius=9.0, model=model, nfreq=20, wmin=2.0, wmax=5.5)
    tol = 1e-10 if precision == "fp64" else 1e-9
    eager, st_e = _run(w, precision=precision, tol_rel=tol, cycle_graphs=0)
    graph, st_g = _run(w, precision=precision, tol_rel=tol, cycle_graphs=1)
    prof, st_p = _run(w, precision=precision, tol_rel=tol, cycle_graphs=1, profile=1)
    assert eager["ok"] and graph["ok"]
    assert st_e["graph_launches"] == 0 and st_p["graph_launches"] == 0
    assert st_g["graph_launches"] == st_g["cycles"] > 0
    for k in ("alpha", "q", "rel_residual", "iters"):
        assert np.array_equal(graph[k], eager[k]), k
        assert np.array_equal(prof[k], eager[k]), k
    assert st_g["total_iters"] <= st_e["total_iters"]


def test_cycle_graph_cache_survives_repeated_solves_and_new_structures():
    """Repeated solves reuse the handle's instantiated graphs (a second identical solve
    captures none); a structure of another size gets its own graphs; results stay those
    of fresh handles."""
    from paper_2510_12731_gb300 import Solver
    w1 = S.small_cluster(element="Ag", radius=9.0, model="wfq", nfreq=10, wmin=2.0, wmax=5.5)
    w2 = S.small_cluster(element="Na", radius=12.0, model="wfq", nfreq=10, wmin=2.0, wmax=4.0)
    ref1, _ = _run(w1, precision="fp32", tol_rel=1e-9)
    ref2, _ = _run(w2, precision="fp32", tol_rel=1e-9)
    with Solver(precision="fp32", tol_rel=1e-9) as s:
        for w, ref in ((w1, ref1), (w1, ref1), (w2, ref2), (w1, ref1)):
            s.set_structure(w.model, w.xyz_ang, w.type_idx, w.types)
            for k in range(2):
                out = s.solve(w.omega_ev, w.pol_dirs, w.alpha_ib)
                assert np.array_equal(out["alpha"], ref["alpha"])
                st = s.stats()
                assert 0 <= st["graphs_built"] <= st["graph_launches"]
                if k == 1:
                    assert st["graphs_built"] == 0


# ------------------------------------------------------------------ structure staging order

@pytest.mark.parametrize("model", ["wfq", "wfqfmu"])
def test_morton_order_is_invisible_to_the_caller(model):
    """Internal Morton order vs the caller's order, and a shuffled input: alpha agrees to
    rounding and per-atom outputs come back in the caller's order."""
    w = S.small_cluster(element="Ag", radius=9.0, model=model, nfreq=6, wmin=2.0, wmax=5.5)
    ref, _ = _run(w, precision="fp64", tol_rel=1e-11, sort_atoms=0)
    srt, _ = _run(w, precision="fp64", tol_rel=1e-11, sort_atoms=1)
    rng = np.random.default_rng(7)
    perm = rng.permutation(w.natoms)
    ws = S.Workload(**{**w.__dict__, "xyz_ang": w.xyz_ang[perm], "type_idx": w.type_idx[perm]})
    shf, _ = _run(ws, precision="fp64", tol_rel=1e-11, sort_atoms=1)
    scale = np.abs(ref["alpha"]).max()
    assert np.abs(srt["alpha"] - ref["alpha"]).max() <= 1e-9 * scale
    assert np.abs(shf["alpha"] - ref["alpha"]).max() <= 1e-9 * scale
    qs = np.abs(ref["q"]).max()
    assert np.abs(srt["q"] - ref["q"]).max() <= 1e-8 * qs
    assert np.abs(shf["q"] - ref["q"][..., perm]).max() <= 1e-8 * qs
    if model == "wfqfmu":
        ms = np.abs(ref["mu"]).max()
        assert np.abs(shf["mu"] - ref["mu"][:, :, perm]).max() <= 1e-8 * ms


# ------------------------------------------------------------------ Krylov basis storage

@pytest.mark.parametrize("model", ["wfq", "wfqfmu"])
@pytest.mark.parametrize("precision", ["fp32", "fp16split"])
@pytest.mark.parametrize("basis", ["fp64", "ff32", "fp32"])
def test_every_basis_reaches_the_fp64_tolerance(model, precision, basis):
    """The basis element type changes only the inner iteration: with the FP64 true
    residual and refinement every choice meets the same per-column tolerance and alpha
    agrees with the oracle."""
    w = S.small_cluster(element="Ag", radius=9.0, model=model, nfreq=30, wmin=2.0, wmax=5.5)
    ref, _ = _oracle(w)
    out, stats = _run(w, precision=precision, tol_rel=1e-9, basis=basis)
    assert out["ok"], out["rel_residual"].max()
    assert np.all(out["rel_residual"] <= 1e-9)
    assert _alpha_err(out, ref) <= 1e-6


def test_fp32_basis_single_round_is_limited_by_fp32_not_by_the_matvec():
    """One round with the FP32 basis and an FP32 matvec, asked for 1e-8: the implicit
    residual no longer follows the true one below a few FP32 ulps, so the unrefined
    alpha is accurate to ~1e-5 but not to 1e-8; refinement rounds close the gap."""
    w = S.small_cluster(element="Ag", radius=9.0, model="wfq", nfreq=12, wmin=2.0, wmax=5.5)
    ref, _ = _oracle(w)
    out1, _ = _run(w, precision="fp32", tol_rel=1e-9, inner_tol=1e-8, max_refine=0,
                   restart_m=200, basis="fp32")
    assert _alpha_err(out1, ref) <= 1e-4
    out2, _ = _run(w, precision="fp32", tol_rel=1e-9, basis="fp32")
    assert out2["ok"] and _alpha_err(out2, ref) <= 1e-7


# ------------------------------------------------------------------ matrix-free (on the fly)

@pytest.mark.parametrize("precision,tol,alpha_tol", [("fp64", 1e-10, 1e-8), ("fp32", 1e-9, 1e-7),
                                                     ("fp16split", 1e-9, 1e-7),
                                                     ("bf16split", 1e-9, 1e-7)])
def test_matfree_parity_small(precision, tol, alpha_tol):
    w = S.small_cluster(element="Ag", radius=9.0, model="wfq", nfreq=9, wmin=2.0, wmax=5.5)
    ref, _ = _oracle(w)
    out, stats = _run(w, precision=precision, tol_rel=tol, mode="matfree")
    assert stats["used_mode"] == 1
    assert out["ok"]
    assert _alpha_err(out, ref) <= alpha_tol


def test_matfree_matches_materialised_on_multi_tile_sphere():
    """Na sphere r = 20 A (N = 893: 7 row tiles, ragged), 40 w x 3 pols: the on-the-fly
    matvec and the materialised one reach the same FP64-refined solution."""
    w = S.small_cluster(element="Na", radius=20.0, model="wfq", nfreq=40, wmin=2.0, wmax=4.0)
    st = M.structure_from_types(w.xyz_ang, w.type_idx, w.types)
    from oracle import spectral as SP
    a_ref = SP.alpha(st, SP.modes(st), w.omega_ev, w.pol_dirs)
    out_mf, _ = _run(w, precision="fp32", tol_rel=1e-8, mode="matfree")
    out_m, _ = _run(w, precision="fp32", tol_rel=1e-8, mode="materialised")
    # the tensor-core pair kernel (T tiles generated in shared memory as fp16 / bf16 planes)
    out_tc, _ = _run(w, precision="fp16split", tol_rel=1e-8, mode="matfree")
    out_tb, _ = _run(w, precision="bf16split", tol_rel=1e-8, mode="matfree")
    for out in (out_mf, out_m, out_tc, out_tb):
        assert out["ok"]
        num = np.linalg.norm(out["alpha"] - a_ref, axis=1)
        assert np.max(num / np.linalg.norm(a_ref, axis=1)) <= 1e-5


@pytest.mark.parametrize("precision,tol,alpha_tol", [("fp32", 1e-9, 1e-7), ("fp64", 1e-10, 1e-8)])
def test_matfree_wfqfmu_parity(precision, tol, alpha_tol):
    """wFQFmu with every 4 x 4 block of T^qq / T^qmu / T^muq / T^mumu generated inside the
    matvec (Sec. 2.2): Ag sphere r = 9 A, N = 177 (6 tiles of 32 atoms, the last ragged;
    K steps of 4 atoms, the last ragged)."""
    w = S.small_cluster(element="Ag", radius=9.0, model="wfqfmu", nfreq=5, wmin=2.5, wmax=5.0)
    assert w.natoms % 32 and w.natoms % 4
    ref, _ = _oracle(w)
    out, stats = _run(w, precision=precision, tol_rel=tol, mode="matfree")
    assert stats["used_mode"] == 1 and out["ok"]
    assert _alpha_err(out, ref) <= alpha_tol
    assert np.abs(out["mu"] - ref.mu).max() <= 1e2 * alpha_tol * np.abs(ref.mu).max()


def test_matfree_wfqfmu_unequal_widths_and_self_term():
    """R_mu != R_q (four distinct pair widths per block) and the Gaussian dipole self
    term on the T^mumu diagonal: matrix-free against the oracle."""
    w = S.small_cluster(element="Au", radius=8.0, model="wfqfmu", nfreq=4, wmin=2.5, wmax=5.0)
    w.types = [{**w.types[0], "Rmu_bohr": 0.8 * w.types[0]["Rq_bohr"]}]
    st = M.structure_from_types(w.xyz_ang, w.type_idx, w.types)
    ref = M.solve(st, w.model, w.omega_ev, w.pol_dirs, alpha_ib=w.alpha_ib, mu_self_term=True)
    out, _ = _run(w, precision="fp32", tol_rel=1e-9, mode="matfree", mu_self_term=1)
    assert out["ok"]
    assert _alpha_err(out, ref) <= 1e-7


def test_matfree_wfqfmu_matches_materialised_rod():
    """Ag rod 18 x 18 x 54 A (N = 1,093: 35 atom tiles, ragged) at 12 frequencies x 3
    directions: on the fly and materialised reach the same refined solution."""
    el = S.ELEMENTS["Ag"]
    xyz = S.cuboid("fcc", el.a_ang, 9.0, 9.0, 27.0)
    w = S.Workload("ag_rod_small", "wfqfmu", xyz, np.zeros(len(xyz), np.int32), [el.atom_type()],
                   np.linspace(2.5, 5.0, 12), np.eye(3), el.alpha_ib(np.linspace(2.5, 5.0, 12))[None, :])
    out_mf, _ = _run(w, precision="fp32", tol_rel=1e-9, mode="matfree")
    out_m, _ = _run(w, precision="fp32", tol_rel=1e-9, mode="materialised")
    # the tensor-core pair kernel (FP16-split blocks generated in shared memory)
    out_tc, _ = _run(w, precision="fp16split", tol_rel=1e-9, mode="matfree")
    assert out_mf["ok"] and out_m["ok"] and out_tc["ok"]
    for out in (out_mf, out_tc):
        num = np.linalg.norm(out["alpha"] - out_m["alpha"], axis=1)
        assert np.max(num / np.linalg.norm(out_m["alpha"], axis=1)) <= 1e-7


def test_wfqfmu_rod_converges_with_dipole_preconditioner():
    """An Ag rod of N = 1,175 atoms (4,700 unknowns), where unpreconditioned GMRES(100)
    stalls above 3.5 eV: the diag(I, alpha^IB) right preconditioner converges every
    column, and alpha matches the oracle's LU."""
    el = S.ELEMENTS["Ag"]
    xyz = S.cuboid("fcc", 4.09, 9.0, 9.0, 30.0)
    w_ev = np.array([2.5, 3.5, 4.5])
    w = S.Workload("rod", "wfqfmu", xyz, np.zeros(len(xyz), np.int32), [el.atom_type()], w_ev,
                   np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0]]), el.alpha_ib(w_ev)[None, :])
    ref, _ = _oracle(w)
    out, stats = _run(w, precision="fp16split", tol_rel=1e-8)
    assert out["ok"]
    assert np.max(out["iters"]) < 3000
    assert _alpha_err(out, ref) <= 1e-5


@pytest.mark.parametrize("model", ["wfq", "wfqfmu"])
def test_system_export_matches_the_oracle_and_solves(model):
    """px_system_device: A0 = diag(Kbar, I) T and b against the oracle's dense assembly;
    a direct LU of A0 - diag(z) in torch reproduces the oracle's alpha."""
    import torch
    w = S.small_cluster(element="Ag", radius=8.0, model=model, nfreq=2, wmin=3.0, wmax=4.0)
    st = M.structure_from_types(w.xyz_ang, w.type_idx, w.types)
    Kb = M.kbar(M.conductance_K(st))
    N = w.natoms
    nu = N if model == "wfq" else 4 * N
    dev = torch.device("cuda", 0)
    A0 = torch.zeros((nu, nu + 5), dtype=torch.float64, device=dev)    # ld > n_u
    b = torch.zeros((nu, 3), dtype=torch.float64, device=dev)
    with _solver(precision="fp64") as s:    # Morton-sorted inside; exported in caller order
        s.set_structure(w.model, w.xyz_ang, w.type_idx, w.types)
        s.system_device(w.pol_dirs, 1.0, d_A0=A0, d_b=b)
    if model == "wfq":
        A_ref = Kb @ M.tqq(st)
        b_ref = np.stack([M.rhs_wfq(Kb, st, e) for e in w.pol_dirs], axis=1)
    else:
        Pm = np.zeros((nu, nu))
        Pm[:N, :N] = Kb
        Pm[N:, N:] = np.eye(3 * N)
        A_ref = Pm @ M.t_full(st)
        b_ref = np.stack([M.rhs_wfqfmu(Kb, st, e) for e in w.pol_dirs], axis=1)
    a = A0[:, :nu].cpu().numpy()
    assert np.abs(a - A_ref).max() <= 1e-12 * np.abs(A_ref).max()
    assert np.abs(b.cpu().numpy() - b_ref).max() <= 1e-12 * np.abs(b_ref).max()
    ref = M.solve(st, w.model, w.omega_ev, w.pol_dirs, alpha_ib=w.alpha_ib)
    om = w.omega_ev / M.HARTREE_EV
    for f in range(2):
        zq = M.z_q(om[f], st.n, st.tau)
        shift = np.full(nu, zq, dtype=np.complex128)
        if model == "wfqfmu":
            shift[N:] = M.z_mu(w.alpha_ib[0, f])
        A = A0[:, :nu].to(torch.complex128) - torch.diag(torch.from_numpy(shift).to(dev))
        x = torch.linalg.solve(A, b.to(torch.complex128)).cpu().numpy()
        q = x[:N]
        mu = x[N:].reshape(N, 3, 3) if model == "wfqfmu" else None
        alpha = M.dipole(st, q, mu)
        assert np.abs(alpha - ref.alpha[f]).max() <= 1e-9 * np.abs(ref.alpha[f]).max()


def test_matfree_tensor_core_matvec_against_the_oracle_operator():
    """One tensor-core pair-kernel step before refinement: with max_refine = 0 and a
    tight inner tolerance, the FP16-split on-the-fly solve reaches the oracle to about the
    split's ~22 bits times the condition number (1e-4), and the BF16 split (~16 bits) to
    1e-2; a wrong swizzle, scale or transposition of the generated tile fails both."""
    w = S.small_cluster(element="Na", radius=17.0, model="wfq", nfreq=6, wmin=2.0, wmax=4.5)
    ref, _ = _oracle(w)
    out16, _ = _run(w, precision="fp16split", tol_rel=1e-9, inner_tol=1e-9, max_refine=0,
                    mode="matfree", restart_m=300)
    assert _alpha_err(out16, ref) <= 1e-4
    outb, _ = _run(w, precision="bf16split", tol_rel=1e-9, inner_tol=1e-9, max_refine=0,
                   mode="matfree", restart_m=300)
    assert _alpha_err(outb, ref) <= 1e-2


@pytest.mark.parametrize("precision", ["fp16split", "bf16split"])
def test_matfree_tensor_core_wfqfmu_parity(precision):
    """wFQFmu on the tensor-core pair kernel: every 4 x 4 block of T^qq / T^qmu / T^muq /
    T^mumu (Sec. 2.2) generated in shared memory as split planes, in the atom-blocked order
    (32-atom row tiles, 16-atom K steps); Ag sphere r = 9 A, N = 177 (6 row tiles and 12 K
    steps, both ragged), refined to the oracle's LU."""
    w = S.small_cluster(element="Ag", radius=9.0, model="wfqfmu", nfreq=5, wmin=2.5, wmax=5.0)
    assert w.natoms % 32 and w.natoms % 16
    ref, _ = _oracle(w)
    out, stats = _run(w, precision=precision, tol_rel=1e-9, mode="matfree")
    assert stats["used_mode"] == 1 and out["ok"]
    assert _alpha_err(out, ref) <= 1e-7
    assert np.abs(out["q"] - ref.q).max() <= 1e-5 * np.abs(ref.q).max()
    assert np.abs(out["mu"] - ref.mu).max() <= 1e-5 * np.abs(ref.mu).max()


def test_matfree_tensor_core_wfqfmu_unequal_widths_and_self_term():
    """R_mu != R_q (four pair widths per close block, and the far-field test over the
    larger of the two) with the Gaussian dipole self term on the T^mumu diagonal, on the
    FP16-split pair kernel."""
    w = S.small_cluster(element="Au", radius=8.0, model="wfqfmu", nfreq=4, wmin=2.5, wmax=5.0)
    w.types = [{**w.types[0], "Rmu_bohr": 0.8 * w.types[0]["Rq_bohr"]}]
    st = M.structure_from_types(w.xyz_ang, w.type_idx, w.types)
    ref = M.solve(st, w.model, w.omega_ev, w.pol_dirs, alpha_ib=w.alpha_ib, mu_self_term=True)
    out, _ = _run(w, precision="fp16split", tol_rel=1e-9, mode="matfree", mu_self_term=1)
    assert out["ok"]
    assert _alpha_err(out, ref) <= 1e-7


def test_matfree_tensor_core_wfqfmu_before_refinement():
    """One low-precision round (max_refine = 0): the unrefined solution carries only the
    generated operator's error, ~22 bits per entry (FP16 split) or ~16 (BF16 split) times
    the conditioning; a misplaced entry of a 4 x 4 block (swizzle, reordering, sign or
    transposition of T^qmu / T^muq) gives O(1) errors instead."""
    w = S.small_cluster(element="Ag", radius=9.0, model="wfqfmu", nfreq=5, wmin=2.5, wmax=5.0)
    ref, _ = _oracle(w)
    kw = dict(tol_rel=1e-9, inner_tol=1e-9, max_refine=0, mode="matfree", restart_m=300)
    out16, _ = _run(w, precision="fp16split", **kw)
    outb, _ = _run(w, precision="bf16split", **kw)
    e16, eb = _alpha_err(out16, ref), _alpha_err(outb, ref)
    assert e16 <= 1e-3 and eb <= 5e-2
    assert e16 < eb


def test_matfree_tensor_core_wfqfmu_single_atom_is_interband_polarisability():
    """One atom: the charge row has no conductance and the dipole row is the interband
    term alone, so alpha = alpha^IB I (Eq. 7) through a tile of 1 real and 31 padding
    atoms and a K step of padding only."""
    w = _single("wfqfmu", [[0.0, 0.0, 0.0]])
    out, stats = _run(w, precision="fp16split", tol_rel=1e-10, mode="matfree")
    assert stats["used_mode"] == 1 and out["ok"]
    for f in range(3):
        assert np.allclose(out["alpha"][f], w.alpha_ib[0, f] * np.eye(3), rtol=1e-10, atol=0)


def test_matfree_tensor_core_wfqfmu_two_atoms():
    d_ang = 2.892
    w = _single("wfqfmu", [[-d_ang / 2, 0, 0], [d_ang / 2, 0, 0]])
    ref, _ = _oracle(w)
    out, _ = _run(w, precision="fp16split", tol_rel=1e-10, mode="matfree")
    assert out["ok"]
    assert _alpha_err(out, ref) <= 1e-8


@pytest.mark.parametrize("n", [16, 32, 33])
def test_matfree_tensor_core_wfqfmu_tile_boundaries(n):
    """N = 16 (one K step of real atoms, one of padding), 32 (exactly one row tile and
    two full K steps) and 33 (one real atom in a second row tile and a third K step):
    the n atoms of an Ag lattice nearest the origin, against the oracle's LU."""
    el = S.ELEMENTS["Ag"]
    xyz = S.sphere("fcc", el.a_ang, 8.0)
    xyz = xyz[np.argsort(np.linalg.norm(xyz, axis=1), kind="stable")[:n]]
    w = _single("wfqfmu", xyz, nfreq=4)
    ref, _ = _oracle(w)
    out, _ = _run(w, precision="fp16split", tol_rel=1e-10, mode="matfree")
    assert out["ok"]
    assert _alpha_err(out, ref) <= 1e-8
