"""Seeded synthetic inputs: lattice-carved nanostructures, parameter presets, sweeps.

This module only prepares inputs (coordinates in Angstrom, per-type parameter
tables, frequency grids, field directions, interband polarisabilities and the
arrival mix of the serving workload).  It contains none of the arithmetic of
the wFQ / wFQFmu method; the library and the independent CPU checker both
consume what it returns.

The paper prints no parameter values and its GEOM structures are not
available, so every structure here is carved from an ideal lattice and every
parameter is a stated stand-in (see ``ELEMENTS``):
  * r0 is the nearest-neighbour distance of the lattice (Eq. 4);
  * d = 12 and s = 1.1 in the Fermi damping (Eq. 4);
  * R_q = R_mu = r0 / 2 (Gaussian widths of Secs. 2.1 and 2.2);
  * n is the free-electron valence density, 1 electron per atom, so that
    n = omega_p^2 / (4 pi) with m* = 1 (Sec. 2.1); for graphene the 2D Drude
    weight E_F / pi with E_F = 0.4 eV;
  * 1/tau = 0.1 eV for metals, 0.01 eV for graphene;
  * A (Eq. 3) is the area for which the bond network of the infinite lattice
    carries the continuum Drude current; the literals below were printed by the
    calibration script of the CPU checker and a CPU test re-derives them;
  * alpha^IB(w) (Eq. 8) is the Clausius-Mossotti polarisability of a one-
    Lorentzian interband permittivity eps_IB = 1 + de w0^2 / (w0^2 - w^2 - i g0 w).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

BOHR_ANG = 0.529177210903      # CODATA 2018
HARTREE_EV = 27.211386245988   # CODATA 2018

# ----------------------------------------------------------------------------
# Parameter presets (all stand-ins; the paper's defaults are not printed)
# ----------------------------------------------------------------------------

# effective areas in bohr^2, printed by the CPU checker's calibration script
_AREA = {
    "Ag": 6.818122713248022,
    "Au": 6.784823018382957,
    "Na": 12.998682769485455,
    "C": 3.089610567125005,
}


@dataclass(frozen=True)
class Element:
    name: str
    lattice: str          # "fcc", "bcc" or "honeycomb"
    a_ang: float          # cube edge (fcc/bcc) or C-C bond length (honeycomb)
    gamma_ev: float       # 1/tau
    drude_n_au: float     # n of Eq. 6
    ib: tuple | None      # (delta_eps, w0_eV, g0_eV) of the interband Lorentzian
    d: float = 12.0
    s: float = 1.1

    @property
    def r0_ang(self) -> float:
        if self.lattice == "fcc":
            return self.a_ang / math.sqrt(2.0)
        if self.lattice == "bcc":
            return self.a_ang * math.sqrt(3.0) / 2.0
        return self.a_ang

    @property
    def volume_bohr3(self) -> float:
        a = self.a_ang / BOHR_ANG
        return a ** 3 / 4.0 if self.lattice == "fcc" else a ** 3 / 2.0

    def atom_type(self) -> dict:
        """Per-type parameter record (same fields as px_atom_type in include/px.h)."""
        r0b = self.r0_ang / BOHR_ANG
        return {
            "r0_ang": self.r0_ang,
            "d": self.d,
            "s": self.s,
            "area_bohr2": _AREA[self.name],
            "Rq_bohr": 0.5 * r0b,
            "Rmu_bohr": 0.5 * r0b,
            "drude_n_au": self.drude_n_au,
            "tau_au": HARTREE_EV / self.gamma_ev,
        }

    def alpha_ib(self, omega_ev) -> np.ndarray:
        """Interband polarisability alpha^IB(w) in a.u. (complex), Clausius-Mossotti."""
        w = np.asarray(omega_ev, dtype=np.float64)
        de, w0, g0 = self.ib
        eps = 1.0 + de * w0 ** 2 / (w0 ** 2 - w ** 2 - 1j * g0 * w)
        return (3.0 * self.volume_bohr3 / (4.0 * math.pi)) * (eps - 1.0) / (eps + 2.0)


def _free_electron_n(lattice, a_ang):
    a = a_ang / BOHR_ANG
    return 1.0 / (a ** 3 / 4.0 if lattice == "fcc" else a ** 3 / 2.0)


ELEMENTS = {
    "Ag": Element("Ag", "fcc", 4.09, 0.1, _free_electron_n("fcc", 4.09), (1.5, 5.0, 1.0)),
    "Au": Element("Au", "fcc", 4.08, 0.1, _free_electron_n("fcc", 4.08), (3.0, 3.0, 1.0)),
    "Na": Element("Na", "bcc", 4.23, 0.1, _free_electron_n("bcc", 4.23), None),
    "C": Element("C", "honeycomb", 1.42, 0.01, (0.4 / HARTREE_EV) / math.pi, None),
}

# ----------------------------------------------------------------------------
# Lattice carving
# ----------------------------------------------------------------------------

_FCC = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]], dtype=np.float64)
_BCC = np.array([[0, 0, 0], [0.5, 0.5, 0.5]], dtype=np.float64)


def cubic_lattice(kind: str, a: float, half_extent: float) -> np.ndarray:
    """All points of an fcc/bcc lattice (atom at the origin) inside the cube |x_k| <= half_extent."""
    basis = _FCC if kind == "fcc" else _BCC
    n = int(math.ceil(half_extent / a)) + 1
    rng = np.arange(-n, n + 1, dtype=np.float64)
    cells = np.array(list(itertools.product(rng, rng, rng)))
    pts = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    keep = np.all(np.abs(pts) <= half_extent + 1e-9, axis=1)
    return pts[keep]


def _sorted(pts):
    """Deterministic order: z, then y, then x (rounded to 1e-6 Angstrom)."""
    key = np.round(pts, 6)
    order = np.lexsort((key[:, 0], key[:, 1], key[:, 2]))
    return np.ascontiguousarray(pts[order])


def sphere(kind: str, a: float, radius: float) -> np.ndarray:
    """Atoms of an fcc/bcc lattice with |r| <= radius (+1e-9), atom at the origin."""
    pts = cubic_lattice(kind, a, radius)
    return _sorted(pts[np.linalg.norm(pts, axis=1) <= radius + 1e-9])


def cuboid(kind: str, a: float, hx: float, hy: float, hz: float) -> np.ndarray:
    """Atoms with |x| <= hx, |y| <= hy, |z| <= hz (+1e-9), atom at the origin."""
    pts = cubic_lattice(kind, a, max(hx, hy, hz))
    h = np.array([hx, hy, hz])
    return _sorted(pts[np.all(np.abs(pts) <= h + 1e-9, axis=1)])


def icosahedron(kind: str, a: float, inradius: float) -> np.ndarray:
    """Solid regular icosahedron of the given inradius (face normals along the
    20 vertex directions of the dual dodecahedron), atom at the origin."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = [np.array(p, dtype=np.float64) for p in itertools.product((-1, 1), repeat=3)]
    for s1, s2 in itertools.product((-1, 1), repeat=2):
        v.append(np.array([0.0, s1 / phi, s2 * phi]))
        v.append(np.array([s1 / phi, s2 * phi, 0.0]))
        v.append(np.array([s1 * phi, 0.0, s2 / phi]))
    normals = np.array(v)
    normals /= np.linalg.norm(normals, axis=1)[:, None]
    circ = 1.2584 * inradius + a       # circumradius / inradius = 1.2584 for an icosahedron
    pts = cubic_lattice(kind, a, circ)
    keep = np.all(pts @ normals.T <= inradius + 1e-9, axis=1)
    return _sorted(pts[keep])


def honeycomb_disk(acc: float, diameter: float, vacancy_frac: float = 0.0,
                   edge_band: float = 5.0, seed: int = 251012731) -> np.ndarray:
    """Graphene disk centred on a hexagon centre, in the z = 0 plane.

    Vacancies: round(vacancy_frac * N) atoms, chosen uniformly (numpy PCG64 with
    ``seed``) among atoms with |r| >= R - edge_band, are removed; afterwards atoms
    left with no neighbour within 1.1 acc are removed too.
    """
    R = diameter / 2.0
    a1 = np.array([1.5, math.sqrt(3.0) / 2.0]) * acc
    a2 = np.array([1.5, -math.sqrt(3.0) / 2.0]) * acc
    n = int(math.ceil(R / acc)) + 2
    ij = np.array(list(itertools.product(range(-n, n + 1), range(-n, n + 1))), dtype=np.float64)
    A = ij[:, :1] * a1 + ij[:, 1:] * a2
    pts = np.concatenate([A, A + np.array([acc, 0.0])], axis=0)
    pts = pts + np.array([acc, 0.0])          # a hexagon centre to the origin
    pts = pts[np.linalg.norm(pts, axis=1) <= R + 1e-9]
    if vacancy_frac > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        r = np.linalg.norm(pts, axis=1)
        cand = np.flatnonzero(r >= R - edge_band)
        nvac = int(round(vacancy_frac * len(pts)))
        drop = rng.choice(cand, size=nvac, replace=False)
        pts = np.delete(pts, drop, axis=0)
        # remove atoms without any neighbour within 1.1 acc
        from scipy.spatial import cKDTree  # input preparation only
        tree = cKDTree(pts)
        cnt = np.array([len(x) for x in tree.query_ball_point(pts, 1.1 * acc)]) - 1
        pts = pts[cnt > 0]
    pts3 = np.concatenate([pts, np.zeros((len(pts), 1))], axis=1)
    return _sorted(pts3)


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    """Everything a solve needs: the structure, its types and the sweep."""

    name: str
    model: str                    # "wfq" or "wfqfmu"
    xyz_ang: np.ndarray           # (N, 3)
    type_idx: np.ndarray          # (N,) int32
    types: list                   # per-type dicts (Element.atom_type())
    omega_ev: np.ndarray          # (F,)
    pol_dirs: np.ndarray          # (P, 3)
    alpha_ib: np.ndarray | None   # (n_types, F) complex, a.u. (wFQFmu)
    precision: str = "fp32"
    mode: str = "auto"
    tol: float = 1e-7
    meta: dict = field(default_factory=dict)

    @property
    def natoms(self) -> int:
        return int(self.xyz_ang.shape[0])

    @property
    def ncols(self) -> int:
        return int(self.omega_ev.size * self.pol_dirs.shape[0])


XYZ = np.eye(3)
X_ONLY = np.array([[1.0, 0.0, 0.0]])


def _one_element(name, el, model, xyz, omega, pols, **kw):
    types = [el.atom_type()]
    aib = el.alpha_ib(omega)[None, :] if model == "wfqfmu" else None
    return Workload(name, model, xyz, np.zeros(len(xyz), dtype=np.int32), types,
                    np.asarray(omega, dtype=np.float64), np.asarray(pols, dtype=np.float64),
                    aib, **kw)


def ag_sphere_791() -> Workload:
    """wFQ, Ag fcc (a = 4.09 A) sphere of radius 15 A on an atom: N = 791; 60 w in
    2.0-4.5 eV, x-polarised; plain FP64."""
    el = ELEMENTS["Ag"]
    return _one_element("ag_sphere_r15A_wfq", el, "wfq", sphere("fcc", el.a_ang, 15.0),
                        np.linspace(2.0, 4.5, 60), X_ONLY, precision="fp64", tol=1e-10)


def na_icosahedron_19931() -> Workload:
    """wFQ, Na bcc (a = 4.23 A) solid icosahedron of inradius 53 A: N = 19,931;
    200 w in 2-4 eV x 3 polarisations; relative residual 1e-7.  Solved by default with
    the FP16-split tensor-core matvec on the materialised T (the FP32 on-the-fly matvec
    reaches the same accuracy: precision "fp32", mode "matfree")."""
    el = ELEMENTS["Na"]
    return _one_element("na_ico_in53A_wfq", el, "wfq", icosahedron("bcc", el.a_ang, 53.0),
                        np.linspace(2.0, 4.0, 200), XYZ, precision="fp16split",
                        mode="materialised", tol=1e-7)


def graphene_disk_20nm() -> Workload:
    """wFQ, graphene disk of diameter 20 nm with 2% edge vacancies (seeded); 300 w
    in 0.1-1.0 eV, x-polarised; materialised T, BF16-split tensor-core matvec."""
    el = ELEMENTS["C"]
    return _one_element("graphene_disk_d20nm_wfq", el, "wfq",
                        honeycomb_disk(el.a_ang, 200.0, vacancy_frac=0.02),
                        np.linspace(0.1, 1.0, 300), X_ONLY, precision="bf16split",
                        mode="materialised", tol=1e-7)


def ag_rod_3x3x10() -> Workload:
    """wFQFmu, Ag fcc cuboid |x|,|y| <= 15 A, |z| <= 50 A: N = 5,513 (22,052
    unknowns); 150 w in 2.5-5.0 eV x 3 polarisations; FP32 matvec."""
    el = ELEMENTS["Ag"]
    return _one_element("ag_rod_3x3x10nm_wfqfmu", el, "wfqfmu",
                        cuboid("fcc", el.a_ang, 15.0, 15.0, 50.0),
                        np.linspace(2.5, 5.0, 150), XYZ, precision="fp32", tol=1e-7)


def na_sphere_r40() -> Workload:
    """wFQ, Na bcc sphere of radius 40 A (N = 7,119), 100 w in 2-4 eV x 3 polarisations:
    a mid-size case whose T (205 MB in FP32) is still larger than L2."""
    el = ELEMENTS["Na"]
    return _one_element("na_sphere_r40A_wfq", el, "wfq", sphere("bcc", el.a_ang, 40.0),
                        np.linspace(2.0, 4.0, 100), XYZ, precision="fp32", tol=1e-7)


def small_cluster(kind="fcc", element="Ag", radius=6.0, model="wfq", nfreq=8,
                  wmin=2.0, wmax=4.5, pols=XYZ) -> Workload:
    """A small sphere for fast parity checks."""
    el = ELEMENTS[element]
    xyz = sphere(el.lattice if el.lattice != "honeycomb" else kind, el.a_ang, radius)
    return _one_element(f"{element}_sphere_r{radius:g}A_{model}", el, model, xyz,
                        np.linspace(wmin, wmax, nfreq), pols, tol=1e-9)


def serving_mix(n_requests=300, seed=12731, rate_hz=1.0, nmin=500, nmax=50000,
                fmin=20, fmax=200):
    """Seeded request mix: Poisson arrivals; wFQ (Ag/Au/Na) or wFQFmu (Ag/Au) with
    p = 1/2; sphere or cuboid rod (aspect 1:1:3); N log-uniform in [nmin, nmax];
    sweep length uniform in [fmin, fmax] over the element's window; 1 or 3
    polarisations.  Returns (arrival_times_s, list of request descriptors)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_requests))
    reqs = []
    for k in range(n_requests):
        model = "wfqfmu" if rng.random() < 0.5 else "wfq"
        element = rng.choice(["Ag", "Au"]) if model == "wfqfmu" else rng.choice(["Ag", "Au", "Na"])
        shape = "sphere" if rng.random() < 0.5 else "rod"
        natoms = float(np.exp(rng.uniform(math.log(nmin), math.log(nmax))))
        nfreq = int(rng.integers(fmin, fmax + 1))
        npol = 1 if rng.random() < 0.5 else 3
        reqs.append({"model": model, "element": str(element), "shape": shape,
                     "natoms_target": natoms, "nfreq": nfreq, "npol": npol})
    return t, reqs


def build_request(desc) -> Workload:
    """Turn a serving-mix descriptor into a workload (structure sized by lattice density)."""
    el = ELEMENTS[desc["element"]]
    vol_ang3 = desc["natoms_target"] * el.volume_bohr3 * BOHR_ANG ** 3
    if desc["shape"] == "sphere":
        radius = (3.0 * vol_ang3 / (4.0 * math.pi)) ** (1.0 / 3.0)
        xyz = sphere(el.lattice, el.a_ang, radius)
    else:
        h = (vol_ang3 / 36.0) ** (1.0 / 3.0)      # box 2h x 2h x 6h
        xyz = cuboid(el.lattice, el.a_ang, h, h, 3.0 * h)
    lo, hi = (2.0, 4.0) if desc["element"] == "Na" else (2.0, 5.0)
    pols = XYZ if desc["npol"] == 3 else X_ONLY
    return _one_element(f"{desc['element']}_{desc['shape']}_{desc['model']}", el, desc["model"],
                        xyz, np.linspace(lo, hi, desc["nfreq"]), pols, tol=1e-7)


def serving_check_mix() -> list:
    """A fixed request mix for checking served results against the oracle: five
    requests of 500-6,000 atoms, wFQ and wFQFmu, Ag / Au / Na, spheres and 1:1:3 rods,
    1 or 3 field directions (the largest, an Ag rod of ~6,000 atoms, is wFQ)."""
    out = []
    spec = [("Na", "sphere", 30.0, "wfq", 40, XYZ),
            ("Ag", "rod", 16.0, "wfq", 30, X_ONLY),
            ("Au", "sphere", 15.5, "wfqfmu", 20, XYZ),
            ("Ag", "rod", 9.0, "wfqfmu", 25, X_ONLY),
            ("Na", "sphere", 20.0, "wfq", 60, X_ONLY)]
    for el_name, shape, size, model, nf, pols in spec:
        el = ELEMENTS[el_name]
        if shape == "sphere":
            xyz = sphere(el.lattice, el.a_ang, size)
        else:
            xyz = cuboid(el.lattice, el.a_ang, size, size, 3.0 * size)
        lo, hi = (2.0, 4.0) if el_name == "Na" else (2.0, 5.0)
        out.append(_one_element(f"{el_name}_{shape}_{len(xyz)}_{model}", el, model, xyz,
                                np.linspace(lo, hi, nf), pols, tol=1e-7))
    return out


def alloy_sphere(radius=17.5, frac_au=0.5, seed=12731, nfreq=251, wmin=2.0, wmax=5.0,
                 pols=XYZ, au_overrides=None) -> Workload:
    """Heterogeneous wFQFmu (Eqs. 9-10): an Ag/Au alloy sphere on the Ag fcc lattice
    (a = 4.09 A); radius 17.5 A (diameter 3.5 nm) gives 1,289 atoms.  A seeded random
    fraction frac_au of the sites (numpy PCG64, ``seed``) carries Au.  Types: Ag, Au with
    their stand-in parameters (``au_overrides`` may replace Au entries, e.g. n or tau);
    alpha^IB per type."""
    xyz = sphere("fcc", 4.09, radius)
    rng = np.random.Generator(np.random.PCG64(seed))
    n_au = int(round(frac_au * len(xyz)))
    tidx = np.zeros(len(xyz), dtype=np.int32)
    if n_au:
        tidx[rng.choice(len(xyz), size=n_au, replace=False)] = 1
    ag, au = ELEMENTS["Ag"], ELEMENTS["Au"]
    t_au = au.atom_type()
    if au_overrides:
        t_au.update(au_overrides)
    w = np.linspace(wmin, wmax, nfreq)
    aib = np.stack([ag.alpha_ib(w), au.alpha_ib(w)])
    return Workload(f"agau_sphere_r{radius:g}A_au{frac_au:g}_wfqfmu_hetero", "wfqfmu_hetero", xyz,
                    tidx, [ag.atom_type(), t_au], w, np.asarray(pols, dtype=np.float64), aib,
                    precision="fp32", tol=1e-7)


# ----------------------------------------------------------------------------
# Boundary-element inputs (Sec. 2.3): meshed particle surfaces and permittivities
# ----------------------------------------------------------------------------

def sphere_mesh(n, radius):
    """n equal-area tesserae on a sphere of the given radius (Angstrom): the points of the
    golden-angle spiral (a Fibonacci lattice) as barycentres, radial outward normals, area
    4 pi R^2 / n each.  Returns (positions (n, 3), normals (n, 3), areas (n,))."""
    i = np.arange(n) + 0.5
    polar = np.arccos(1.0 - 2.0 * i / n)
    azim = np.pi * (1.0 + math.sqrt(5.0)) * i
    u = np.stack([np.cos(azim) * np.sin(polar), np.sin(azim) * np.sin(polar), np.cos(polar)], axis=1)
    return radius * u, u, np.full(n, 4.0 * math.pi * radius * radius / n)


def spheroid_mesh(n, a, b, c):
    """The sphere mesh mapped onto the ellipsoid x^2/a^2 + y^2/b^2 + z^2/c^2 = 1: points
    (a u_x, b u_y, c u_z), normals along (u_x/a, u_y/b, u_z/c), areas scaled by the map's
    area factor a b c |(u_x/a, u_y/b, u_z/c)|."""
    _, u, a0 = sphere_mesh(n, 1.0)
    g = u / np.array([a, b, c])
    gn = np.linalg.norm(g, axis=1)
    return u * np.array([a, b, c]), g / gn[:, None], a0 * a * b * c * gn


def drude_eps(omega_ev, wp_ev, gamma_ev, eps_inf=1.0):
    """Drude permittivity e(w) = e_inf - wp^2 / (w^2 + i gamma w) (a stand-in for the
    tabulated permittivities the paper reads)."""
    w = np.asarray(omega_ev, dtype=np.float64)
    return eps_inf - wp_ev ** 2 / (w * w + 1j * gamma_ev * w)


@dataclass
class MeshWorkload:
    """A boundary-element problem: the meshed surface, the sweep and the permittivities."""

    name: str
    pos_ang: np.ndarray           # (n, 3) tessera barycentres
    normals: np.ndarray           # (n, 3) outward unit normals
    area_ang2: np.ndarray         # (n,) tessera areas
    radius_ang: float             # radius of the sphere enclosing the mesh (F's diagonal)
    omega_ev: np.ndarray          # (F,)
    eps2: np.ndarray              # (F,) complex, the particle
    eps1: np.ndarray              # (F,) complex, the medium
    pol_dirs: np.ndarray          # (P, 3)
    tol: float = 1e-7

    @property
    def ntess(self) -> int:
        return int(self.pos_ang.shape[0])

    @property
    def ncols(self) -> int:
        return int(self.omega_ev.size * self.pol_dirs.shape[0])


def drude_sphere_mesh(n=3200, radius=20.0, nfreq=200, wmin=2.5, wmax=4.5, wp=6.0, gamma=0.1,
                      eps1=1.0, pols=XYZ) -> MeshWorkload:
    """DPCM stand-in workload: a Drude sphere (wp = 6 eV, gamma = 0.1 eV) of radius 20 A
    meshed by n tesserae, in a medium of permittivity eps1, nfreq frequencies around its
    dipolar (Froehlich) resonance wp / sqrt(3 eps1)."""
    pos, nrm, area = sphere_mesh(n, radius)
    w = np.linspace(wmin, wmax, nfreq)
    return MeshWorkload(f"drude_sphere_r{radius:g}A_{n}tess", pos, nrm, area, float(radius), w,
                        drude_eps(w, wp, gamma), np.full(nfreq, eps1, dtype=np.complex128),
                        np.asarray(pols, dtype=np.float64))
