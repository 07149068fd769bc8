"""GPU parity for the time-dependent potential V(t,x): both march variants (every
step's factors computed once per build and streamed, and the per-step
refactorising march), matrix-free GMRES of Algorithm 2 preconditioned by
P = I - L_0."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1503_02564_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_MARCH = 1e-10
TOL_SOLVE = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_02564_gb300 import build_ext
    build_ext.build()


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def problem(wl):
    return O.Problem(wl.a0, wl.b0, wl.nx, wl.dt, wl.nt, wl.off.astype(np.int64), wl.u0, wl.V,
                     vkind=wl.vkind, tc=wl.tc, sigma=wl.sigma, nl_coef=wl.nl_coef)


def gpu_plan(wl, streamed=None, chunk=None, **kw):
    """streamed: True / False selects the V(t,x) march variant (None: default);
    chunk: a fixed chunk length."""
    from paper_1503_02564_gb300 import swr
    tuning = {}
    if streamed is not None:
        tuning["tdep_precomp"] = 0 if streamed else -1
    if chunk is not None:
        tuning["chunk_L"] = chunk
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, p=wl.sigma, vkind=wl.vkind, tuning=tuning, **kw)
    V = torch.tensor(np.ascontiguousarray(wl.V).ravel(), dtype=torch.float64, device="cuda")
    u0 = torch.tensor(wl.u0, dtype=torch.complex128, device="cuda")
    plan.build_interface(V, u0)
    if streamed is not None and wl.vkind == swr.SWR_V_TIME:
        want = swr.MARCH_TDEP_STREAMED if streamed else swr.MARCH_TDEP_REFACTOR
        assert plan.get_stats()["march_variant"] == want
    return plan


def ragged_tdep():
    wl = W.config4(nsub=5, nx=401, nt=23)
    wl.off = np.array([0, 2, 90, 201, 260, 400], dtype=np.int32)
    return wl


CASES = {
    "config4_small": lambda: W.config4(nsub=4, nx=2001, nt=40),
    "config4_N16": lambda: W.config4(nsub=16, nx=6001, nt=30),
    "ragged": ragged_tdep,
}


@pytest.mark.parametrize("streamed", [True, False])
@pytest.mark.parametrize("case", sorted(CASES))
def test_tdep_apply_R_matches_oracle(case, streamed):
    wl = CASES[case]()
    plan = gpu_plan(wl, streamed)
    g = W.random_interface(wl.nblk, wl.nt, 31)
    gi = torch.tensor(g.ravel(), dtype=torch.complex128, device="cuda")
    go = torch.zeros_like(gi)
    plan.apply_R(gi, go)
    assert rel(go.cpu().numpy(), O.apply_R(problem(wl), g)) < TOL_MARCH
    d = torch.zeros_like(gi)
    plan.get_interface(d, None)
    assert rel(d.cpu().numpy(), O.build_d(problem(wl))) < TOL_MARCH
    plan.destroy()


@pytest.mark.parametrize("chunk", [4, 8, 12, 16])
def test_tdep_streamed_long_subdomains_match_oracle(chunk):
    """Streamed per-step factors on long subdomains (thread-block clusters): the
    factors are staged in shared memory in full, or only the separator part when
    the chunk factors do not fit (chunk 8 and 16 here), and the result is the same."""
    wl = W.config4(nsub=4, nx=60001, nt=12)
    plan = gpu_plan(wl, True, chunk=chunk)
    g = W.random_interface(wl.nblk, wl.nt, 33)
    gi = torch.tensor(g.ravel(), dtype=torch.complex128, device="cuda")
    go = torch.zeros_like(gi)
    plan.apply_R(gi, go)
    d = torch.zeros_like(gi)
    plan.get_interface(d, None)
    plan.destroy()
    P = problem(wl)
    assert rel(go.cpu().numpy(), O.apply_R(P, g)) < TOL_MARCH
    assert rel(d.cpu().numpy(), O.build_d(P)) < TOL_MARCH


@pytest.mark.parametrize("streamed", [True, False])
def test_tdep_with_constant_potential_equals_static_path(streamed):
    """Fed V(t,x) = V(x) for every t, both V(t,x) marches must give what the
    factor-once march gives."""
    from paper_1503_02564_gb300 import swr
    wl = W.config2(nsub=6, nx=3001, nt=25)
    g = W.random_interface(wl.nblk, wl.nt, 32)
    gi = torch.tensor(g.ravel(), dtype=torch.complex128, device="cuda")
    out_s = torch.zeros_like(gi)
    gpu_plan(wl).apply_R(gi, out_s)
    wl_t = W.config2(nsub=6, nx=3001, nt=25)
    wl_t.V = np.tile(wl.V, (wl.nt + 1, 1))
    wl_t.vkind = swr.SWR_V_TIME
    out_t = torch.zeros_like(gi)
    gpu_plan(wl_t, streamed).apply_R(gi, out_t)
    assert rel(out_t.cpu().numpy(), out_s.cpu().numpy()) < TOL_MARCH


@pytest.mark.parametrize("streamed", [True, False])
@pytest.mark.parametrize("precond", [0, 1, 3])
def test_tdep_gmres_reproduces_monodomain(precond, streamed):
    from paper_1503_02564_gb300 import swr
    wl = CASES["config4_small"]()
    # |g| is about 1e-8 here (the packet barely reaches the interfaces): stop
    # relative to |d| so that the comparison measures the arithmetic
    tol = 1e-13 * np.linalg.norm(O.build_d(problem(wl)))
    plan = gpu_plan(wl, streamed, restart=100, maxit=400, tol_abs=tol,
                    precond=precond)
    g = torch.zeros(plan.n_interface, dtype=torch.complex128, device="cuda")
    uT = torch.zeros(wl.nx, dtype=torch.complex128, device="cuda")
    info = plan.solve(g, False, uT)
    plan.destroy()
    gs, uTm = O.mono_interface(problem(wl))
    assert info["residual"] < tol
    assert rel(uT.cpu().numpy(), uTm) < TOL_SOLVE
    assert rel(g.cpu().numpy(), gs) < TOL_SOLVE


def test_full_size_time_dependent_config_against_monodomain():
    """Full-size time-dependent workload (60001 nodes, 1000 steps, N = 64):
    GMRES preconditioned by the interface operator of the time-averaged
    potential, to the absolute residual 1e-10.  (The zero-potential operator of
    Section 5 stalls here: -x^2/4 reaches -340 at the ends and accumulates
    hundreds of radians of phase over T = 1.)"""
    from paper_1503_02564_gb300 import swr
    wl = W.config4()
    gs, uTm = O.mono_interface(problem(wl))
    tol = 1e-10
    plan = gpu_plan(wl, True, restart=60, maxit=400, tol_abs=tol,
                    precond=swr.SWR_PC_MEAN_POTENTIAL)
    g = torch.zeros(plan.n_interface, dtype=torch.complex128, device="cuda")
    uT = torch.zeros(wl.nx, dtype=torch.complex128, device="cuda")
    info = plan.solve(g, False, uT)
    plan.destroy()
    print("full-size time-dependent solve:", info)
    assert info["residual"] < tol, info
    assert rel(uT.cpu().numpy(), uTm) < TOL_SOLVE
    assert rel(g.cpu().numpy(), gs) < TOL_SOLVE
