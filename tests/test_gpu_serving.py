"""Continuous-batching server: every request's result in a concurrent mix equals the
same request solved alone, within the solver tolerance, and equals the oracle's (a fixed
mix of 500-5,300-atom wFQ and wFQFmu requests against the values in tests/golden/);
admission respects the budget; repeated structures reuse the device-resident operators."""
import os

import numpy as np
import pytest

from paper_2510_12731_gb300 import structures as S

pytestmark = pytest.mark.gpu

TOL = 1e-9


def _mix():
    ag, na, au = S.ELEMENTS["Ag"], S.ELEMENTS["Na"], S.ELEMENTS["Au"]
    reqs = []
    # (element, shape, model, n_freq, pols)
    spec = [("Ag", S.sphere("fcc", 4.09, 9.0), "wfq", 11, S.XYZ),
            ("Au", S.sphere("fcc", 4.08, 8.0), "wfqfmu", 7, S.X_ONLY),
            ("Na", S.sphere("bcc", 4.23, 14.0), "wfq", 23, S.XYZ),
            ("Ag", S.cuboid("fcc", 4.09, 5.0, 5.0, 12.0), "wfqfmu", 9, S.XYZ),
            ("Ag", S.sphere("fcc", 4.09, 9.0), "wfq", 5, S.X_ONLY),      # same structure again
            ("Na", S.sphere("bcc", 4.23, 10.0), "wfq", 31, S.X_ONLY)]
    for el_name, xyz, model, nf, pols in spec:
        el = S.ELEMENTS[el_name]
        lo, hi = (2.0, 4.0) if el_name == "Na" else (2.0, 5.0)
        w = np.linspace(lo, hi, nf)
        aib = el.alpha_ib(w)[None, :] if model == "wfqfmu" else None
        reqs.append(dict(model=model, xyz_ang=xyz, type_idx=np.zeros(len(xyz), np.int32),
                         types=[el.atom_type()], omega_ev=w, pol_dirs=pols, alpha_ib=aib))
    return reqs


def _alone(r, **opts):
    from paper_2510_12731_gb300 import Solver
    with Solver(**opts) as s:
        s.set_structure(r["model"], r["xyz_ang"], r["type_idx"], r["types"])
        return s.solve(r["omega_ev"], r["pol_dirs"], r["alpha_ib"])


@pytest.mark.parametrize("precision", ["fp32", "fp16split"])
def test_results_alone_equal_results_in_the_mix(precision):
    from paper_2510_12731_gb300 import Server
    reqs = _mix()
    alone = [_alone(r, precision=precision, tol_rel=TOL) for r in reqs]
    with Server(max_slots=3, precision=precision, tol_rel=TOL) as srv:
        ids = [srv.submit(**r) for r in reqs]          # all arrive while others run
        outs = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["p99_latency_ms"] >= st["p50_latency_ms"] > 0
    for a, o in zip(alone, outs):
        assert o["ok"] and a["ok"]
        num = np.linalg.norm(o["alpha"] - a["alpha"], axis=1)
        den = np.linalg.norm(a["alpha"], axis=1)
        assert np.max(num / den) <= 1e-6
        assert np.all(o["rel_residual"] <= TOL)


def test_repeated_structure_reuses_resident_operators():
    """One slot: the second request on the same structure skips the structure set-up
    and still matches its alone result."""
    from paper_2510_12731_gb300 import Server
    reqs = _mix()
    same = [reqs[0], reqs[4]]          # Ag sphere r = 9 A, two different sweeps
    alone = [_alone(r, precision="fp32", tol_rel=TOL) for r in same]
    with Server(max_slots=1, precision="fp32", tol_rel=TOL) as srv:
        ids = [srv.submit(**r) for r in same]
        outs = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert st["structure_reuses"] == 1
    for a, o in zip(alone, outs):
        num = np.linalg.norm(o["alpha"] - a["alpha"], axis=1)
        assert np.max(num / np.linalg.norm(a["alpha"], axis=1)) <= 1e-6


def test_admission_respects_a_small_budget():
    """With a budget that holds one request at a time, requests still all finish (they
    are admitted one by one) and the reserved footprint never exceeds the budget."""
    from paper_2510_12731_gb300 import Server
    reqs = _mix()[:3]
    budget = 160 << 20
    with Server(max_slots=3, hbm_budget_bytes=budget, precision="fp32", tol_rel=1e-8) as srv:
        ids = [srv.submit(**r) for r in reqs]
        outs = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert all(o["ok"] for o in outs)
    assert st["peak_reserved_bytes"] <= budget


def test_poll_and_unknown_ids():
    from paper_2510_12731_gb300 import PxError, Server
    r = _mix()[0]
    with Server(max_slots=1, precision="fp32", tol_rel=1e-8) as srv:
        rid = srv.submit(**r)
        out = None
        import time
        t0 = time.time()
        while out is None and time.time() - t0 < 120:
            out = srv.poll(rid)
            time.sleep(0.01)
        assert out is not None and out["ok"]
        with pytest.raises(KeyError):
            srv.poll(rid)


def _golden(i, P):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", f"serving{i}_alpha.txt")
    if not os.path.exists(path):
        pytest.skip(f"{path} not generated")
    rows = np.loadtxt(path)
    fidx = np.unique(rows[:, 0].astype(int))
    a = np.zeros((len(fidx), 3, P), dtype=np.complex128)
    pos = {f: k for k, f in enumerate(fidx)}
    for fi, _, p, k, re, im in rows:
        a[pos[int(fi)], int(k), int(p)] = re + 1j * im
    return fidx, a


@pytest.mark.parametrize("precision,solver", [("fp16split", "batched"), ("fp32", "batched"),
                                              ("fp32", "shifted")])
def test_served_results_match_the_oracle(precision, solver):
    """Five requests (wFQ and wFQFmu, 893-5,287 atoms) submitted together to three slots
    (with the shifted solver, the wFQ requests run it and the wFQFmu ones stay batched);
    every served alpha within 1e-5 of the oracle (spectral route for wFQ, dense LU at three
    frequencies for wFQFmu), every column at its FP64-class tolerance."""
    from paper_2510_12731_gb300 import Server
    mix = S.serving_check_mix()
    with Server(max_slots=3, precision=precision, tol_rel=1e-7, solver=solver) as srv:
        ids = [srv.submit(w.model, w.xyz_ang, w.type_idx, w.types, w.omega_ev, w.pol_dirs,
                          w.alpha_ib) for w in mix]
        outs = [srv.wait(i, timeout_s=1800) for i in ids]
        st = srv.stats()
    assert st["completed"] == len(mix) and st["failed"] == 0
    assert max(w.natoms for w in mix) > 5000
    for i, (w, o) in enumerate(zip(mix, outs)):
        assert o["ok"] and np.all(o["rel_residual"] <= 1e-7), w.name
        fidx, ref = _golden(i, w.pol_dirs.shape[0])
        err = np.linalg.norm(o["alpha"][fidx] - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert np.max(err) <= 1e-5, (w.name, np.max(err))


@pytest.mark.parametrize("model", ["wfq", "wfqfmu"])
def test_same_structure_requests_merge_into_one_block(model):
    """One slot, busy with another structure: three queued requests on one structure with
    the same field directions and different frequency grids are solved as one block
    (their frequencies appended, alpha_ib rows concatenated per type), and each gets back
    exactly its own columns: equal to its alone result, in its own frequency order."""
    from paper_2510_12731_gb300 import Server
    blocker = _mix()[2]                        # Na sphere r = 14 A, 23 w x 3
    el = S.ELEMENTS["Au"] if model == "wfqfmu" else S.ELEMENTS["Ag"]
    xyz = S.sphere("fcc", 4.08 if model == "wfqfmu" else 4.09, 8.0)
    grids = [np.linspace(2.0, 5.0, 9), np.linspace(2.7, 3.9, 5)[::-1], np.linspace(3.1, 4.6, 13)]
    same = []
    for w in grids:
        same.append(dict(model=model, xyz_ang=xyz, type_idx=np.zeros(len(xyz), np.int32),
                         types=[el.atom_type()], omega_ev=w, pol_dirs=S.XYZ,
                         alpha_ib=el.alpha_ib(w)[None, :] if model == "wfqfmu" else None))
    alone = [_alone(r, precision="fp32", tol_rel=TOL) for r in same]
    with Server(max_slots=1, precision="fp32", tol_rel=TOL) as srv:
        ids = [srv.submit(**blocker)] + [srv.submit(**r) for r in same]
        outs = [srv.wait(i) for i in ids][1:]
        st = srv.stats()
    assert st["merged_requests"] == 2 and st["completed"] == 4 and st["failed"] == 0
    for a, o in zip(alone, outs):
        assert o["ok"] and o["alpha"].shape == a["alpha"].shape
        num = np.linalg.norm(o["alpha"] - a["alpha"], axis=1)
        assert np.max(num / np.linalg.norm(a["alpha"], axis=1)) <= 1e-6
        assert np.all(o["rel_residual"] <= TOL)
        assert np.allclose(o["sigma_abs"], a["sigma_abs"], rtol=1e-6)
