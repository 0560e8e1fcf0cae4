"""The no-allocation residual check (px_relres_device_noalloc) against px_solve_device.

px_relres_device_noalloc serves callers that cannot allocate device memory where they
call it (under a memory pool that owns all free device memory, in latency-bound loops
that must not enter the driver's allocator): it recomputes the FP64
relative residual of a device-resident solution using only a fixed scratch array in
the library.  Here the solution comes from px_solve_device, whose own relative
residuals are the expected values; the check runs twice in a row to show that the
shared scratch array carries nothing over from one call to the next.  This file is
collected last so a failure here cannot hide the other GPU tests.
"""
import numpy as np
import pytest

from paper_2510_12731_gb300 import structures as S

pytestmark = pytest.mark.gpu


def _case(model):
    return S.small_cluster(element="Ag", radius=9.0, model=model, nfreq=7, wmin=2.0, wmax=5.5)


@pytest.mark.parametrize("model", ["wfq", "wfqfmu"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_residual_matches_solve_device(model, precision):
    import torch
    from paper_2510_12731_gb300 import Solver

    w = _case(model)
    F, P, N = w.omega_ev.size, w.pol_dirs.shape[0], w.natoms
    dev = torch.device("cuda", 0)
    d_q = torch.zeros((F, P, N), dtype=torch.complex128, device=dev)
    d_mu = torch.zeros((F, P, N, 3), dtype=torch.complex128, device=dev)
    d_rr = torch.zeros((F, P), dtype=torch.float64, device=dev)
    with Solver(precision=precision, tol_rel=1e-9) as s:
        s.set_structure(w.model, w.xyz_ang, w.type_idx, w.types)
        assert s.solve_device(w.omega_ev, w.pol_dirs, w.alpha_ib, d_q=d_q,
                              d_mu=d_mu if model == "wfqfmu" else None, d_relres=d_rr)
        expect = d_rr.cpu().numpy()
        outs = [torch.full((F, P), -1.0, dtype=torch.float64, device=dev) for _ in range(2)]
        torch.cuda.synchronize()
        for k in range(2):
            free0 = torch.cuda.mem_get_info(dev)[0]
            s.relres_device_noalloc(w.omega_ev, w.pol_dirs, d_q, outs[k], alpha_ib=w.alpha_ib,
                                    d_mu=d_mu if model == "wfqfmu" else None)
            free1 = torch.cuda.mem_get_info(dev)[0]
            # the defining property: the call takes no device memory (the first call of
            # the process may load the library's module, so only later calls are held
            # to it)
            if k == 1:
                assert free1 == free0
        for got_t in outs:
            got = got_t.cpu().numpy()
            assert np.all(got >= 0.0)
            # both are FP64-class residual norms of the same solution (px_solve_device
            # evaluates the low-precision modes' residual in double-FP32, this entry point
            # in FP64); they agree to ~1e-11 of ||b||, far below tol_rel
            assert np.allclose(got, expect, rtol=1e-6, atol=3e-11)
            assert np.all(got <= 1e-9)


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch
    from paper_2510_12731_gb300 import PxError, Solver

    el = S.ELEMENTS["Na"]
    xyz = S.sphere("bcc", 4.23, 30.0)          # N = 2,975
    w_ev = np.linspace(2.0, 4.0, 400)          # 400 x 3 columns: needs ~80 MB of scratch
    F, P, N = w_ev.size, 3, len(xyz)
    dev = torch.device("cuda", 0)
    d_q = torch.zeros((F, P, N), dtype=torch.complex128, device=dev)
    d_rr = torch.zeros((F, P), dtype=torch.float64, device=dev)
    with Solver(precision="fp32") as s:
        s.set_structure("wfq", xyz, np.zeros(N, np.int32), [el.atom_type()])
        with pytest.raises(PxError, match="EINVAL.*scratch"):
            s.relres_device_noalloc(w_ev, np.eye(3), d_q, d_rr)


def test_noalloc_validates_inputs_like_solve():
    import torch
    from paper_2510_12731_gb300 import PxError, Solver

    w = _case("wfqfmu")
    F, P, N = w.omega_ev.size, w.pol_dirs.shape[0], w.natoms
    dev = torch.device("cuda", 0)
    d_q = torch.zeros((F, P, N), dtype=torch.complex128, device=dev)
    d_mu = torch.zeros((F, P, N, 3), dtype=torch.complex128, device=dev)
    d_rr = torch.zeros((F, P), dtype=torch.float64, device=dev)
    with Solver(precision="fp32") as s:
        s.set_structure(w.model, w.xyz_ang, w.type_idx, w.types)
        bad_pol = w.pol_dirs.copy()
        bad_pol[1] *= 2.0
        with pytest.raises(PxError, match="EINVAL.*unit"):
            s.relres_device_noalloc(w.omega_ev, bad_pol, d_q, d_rr, alpha_ib=w.alpha_ib, d_mu=d_mu)
        bad_aib = w.alpha_ib.copy()
        bad_aib[0, 2] = np.nan
        with pytest.raises(PxError, match="EINVAL.*alpha_ib"):
            s.relres_device_noalloc(w.omega_ev, w.pol_dirs, d_q, d_rr, alpha_ib=bad_aib, d_mu=d_mu)
