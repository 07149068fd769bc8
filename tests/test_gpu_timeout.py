"""Failure detection of the bounded device waits, made to happen on purpose without
faulting anything: the causal substitution's CTAs hand values on through progress
counters, and a test hook (swr_test_wait_hook) makes one interface's CTA withhold its
counter, with a short poll limit.  The neighbours' waits then run out, the kernel
raises SWR_ERR_TIMEOUT through the status word and every CTA leaves through the abort
flag; the context stays usable, and with the hook cleared a fresh plan (and the
allocation-free entry point) solves correctly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1503_02564_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def swr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_02564_gb300 import build_ext, swr as S
    build_ext.build()
    yield S
    S.swr_test_wait_hook(0, -1)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def _plan(swr, wl, **kw):
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, p=wl.sigma, precond=swr.SWR_PC_CAUSAL, **kw)
    plan.build_interface(torch.tensor(wl.V, dtype=torch.float64, device="cuda"),
                         torch.tensor(wl.u0, dtype=torch.complex128, device="cuda"))
    return plan


# sweep form (wide subdomains: nothing to resolve in the same step) and window form
# (N = 256 on the scaling grid: the same-step coupling is resolved over H >= 1)
CASES = {"sweeps": lambda: W.config2(nsub=8, nx=8001, nt=64),
         "window": lambda: W.config2(nsub=256, nt=24)}


@pytest.mark.parametrize("case", sorted(CASES))
def test_withheld_progress_times_out_and_the_device_recovers(swr, case):
    wl = CASES[case]()
    y = torch.tensor(W.random_interface(wl.nblk, wl.nt, 5).ravel(), dtype=torch.complex128,
                     device="cuda")
    x = torch.zeros_like(y)
    plan = _plan(swr, wl)
    st = plan.get_stats()
    assert (st["causal_window"] >= 1) == (case == "window"), st
    try:
        swr.swr_test_wait_hook(20000, 3)
        with pytest.raises(swr.SWRError) as e:
            plan.apply_precond(y, x)
        assert e.value.status == swr.SWR_ERR_TIMEOUT
    finally:
        swr.swr_test_wait_hook(0, -1)
        plan.destroy()
    # the context still works: a fresh plan solves to the monodomain solution
    plan = _plan(swr, wl)
    g = torch.zeros(plan.n_interface, dtype=torch.complex128, device="cuda")
    uT = torch.zeros(wl.nx, dtype=torch.complex128, device="cuda")
    info = plan.solve(g, False, uT)
    plan.destroy()
    assert info["status"] == swr.SWR_OK and info["residual"] < 1e-10
    if case == "sweeps":
        P = O.Problem(wl.a0, wl.b0, wl.nx, wl.dt, wl.nt, wl.off.astype(np.int64), wl.u0, wl.V,
                      sigma=wl.sigma)
        gs, uTm = O.mono_interface(P)
        assert rel(uT.cpu().numpy(), uTm) < 1e-9
        assert rel(g.cpu().numpy(), gs.ravel()) < 1e-9


def test_no_alloc_entry_point_reports_the_timeout_then_recovers(swr):
    wl = CASES["sweeps"]()
    plan = _plan(swr, wl, pc_sweeps=1)
    cols = torch.zeros(4 * wl.nsub * wl.nt, dtype=torch.complex128, device="cuda")
    plan.get_interface(None, cols)
    y = torch.tensor(W.random_interface(wl.nblk, wl.nt, 6).ravel(), dtype=torch.complex128,
                     device="cuda")
    x_ref = torch.zeros_like(y)
    plan.apply_precond(y, x_ref)
    plan.destroy()
    x = torch.zeros_like(y)
    try:
        swr.swr_test_wait_hook(20000, 2)
        assert swr.swr_causal_solve_noalloc(wl.nsub, wl.nt, 1, cols, y, x) == \
            swr.SWR_ERR_TIMEOUT
    finally:
        swr.swr_test_wait_hook(0, -1)
    assert swr.swr_causal_solve_noalloc(wl.nsub, wl.nt, 1, cols, y, x) == swr.SWR_OK
    assert rel(x.cpu().numpy(), x_ref.cpu().numpy()) < 1e-10
