"""Write the oracle's expected polarisabilities for the full-size workloads.

Calls only the CPU oracle (``oracle/``) on the seeded inputs of
``paper_2510_12731_gb300.structures``; the GPU tests compare the library against these
files.  Routes:
  * wFQ workloads: the exact spectral route (Cholesky of T, symmetric eigensolve) gives
    every (frequency, polarisation) column;
  * the wFQFmu rod: one dense LU per sampled frequency (lowest, middle, highest);
  * the fixed serving check mix: each request by the route of its model;
  * the 1,289-atom Ag/Au alloy sphere (Eqs. 9-10): dense LU at three frequencies.
Run:  python tests/golden/make_golden.py [name ...]   (a few minutes to ~30 min each).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import model as M  # noqa: E402
from oracle import spectral as SP  # noqa: E402
from paper_2510_12731_gb300 import structures as S  # noqa: E402


def _write(name, w, idx, alpha, route):
    path = os.path.join(HERE, f"{name}_alpha.txt")
    with open(path, "w") as f:
        f.write(f"# oracle alpha for workload {w.name}: N = {w.natoms}, {route}\n")
        f.write("# written by tests/golden/make_golden.py (CPU oracle only)\n")
        f.write("# columns: freq_index omega_eV pol_index k re(alpha_kp) im(alpha_kp)  [bohr^3]\n")
        for fi_local, fi in enumerate(idx):
            for p in range(w.pol_dirs.shape[0]):
                for k in range(3):
                    a = alpha[fi_local, k, p]
                    f.write(f"{fi} {w.omega_ev[fi]:.12g} {p} {k} {a.real:.17e} {a.imag:.17e}\n")
    print("wrote", path, flush=True)


def spectral_workload(name, w):
    t = time.time()
    st = M.structure_from_types(w.xyz_ang, w.type_idx, w.types)
    md = SP.modes(st)
    alpha = SP.alpha(st, md, w.omega_ev, w.pol_dirs)
    print(name, "spectral route", round(time.time() - t, 1), "s", flush=True)
    _write(name, w, np.arange(w.omega_ev.size), alpha, "spectral route, every column")


def lu_sample(name, w, n_samples=3):
    idx = np.unique(np.linspace(0, w.omega_ev.size - 1, n_samples).round().astype(int))
    st = M.structure_from_types(w.xyz_ang, w.type_idx, w.types)
    t = time.time()
    res = M.solve(st, w.model, w.omega_ev[idx], w.pol_dirs,
                  alpha_ib=None if w.alpha_ib is None else w.alpha_ib[:, idx])
    print(name, "LU", round(time.time() - t, 1), "s, max rel residual", res.rel_residual.max(),
          flush=True)
    _write(name, w, idx, res.alpha, f"dense LU at frequency indices {idx.tolist()}")


def serving_check():
    """Every request of the fixed serving check mix: the spectral route for wFQ, LU at
    three frequencies for wFQFmu."""
    for i, w in enumerate(S.serving_check_mix()):
        name = f"serving{i}"
        if w.model == "wfq":
            spectral_workload(name, w)
        else:
            lu_sample(name, w)


def alloy_lu(name, w, n_samples=3):
    """Heterogeneous wFQFmu (Eqs. 9-10) by the oracle's dense LU at sampled frequencies."""
    from oracle import hetero as HT
    idx = np.unique(np.linspace(0, w.omega_ev.size - 1, n_samples).round().astype(int))
    t = time.time()
    alpha, _, _, rel = HT.solve(w.xyz_ang, w.type_idx, w.types, w.omega_ev[idx], w.pol_dirs,
                                w.alpha_ib[:, idx])
    print(name, "LU", round(time.time() - t, 1), "s, max rel residual", rel.max(), flush=True)
    _write(name, w, idx, alpha, f"dense LU of Eq. 9 at frequency indices {idx.tolist()}")


JOBS = {
    "graphene_disk_20nm": lambda: spectral_workload("graphene_disk_20nm", S.graphene_disk_20nm()),
    "na_icosahedron_19931": lambda: spectral_workload("na_icosahedron_19931",
                                                      S.na_icosahedron_19931()),
    "ag_rod_3x3x10": lambda: lu_sample("ag_rod_3x3x10", S.ag_rod_3x3x10()),
    "serving_check": serving_check,
    "agau_sphere_1289": lambda: alloy_lu("agau_sphere_1289", S.alloy_sphere()),
}

if __name__ == "__main__":
    names = sys.argv[1:] or list(JOBS)
    for n in names:
        JOBS[n]()
