"""GPU parity for the order-2 potential-strategy transmission condition S_0^2
(Section 2.2): S-bar v_n = c2 sum_{s<=n} beta_{n-s} v_s, c2 = e^{-i pi/4}
sqrt(2/dt).  The march carries the history sums at the subdomain ends; the
interface algebra (Toeplitz columns, causal preconditioner, GMRES) is the same
as for Robin.  Tolerances as for Robin: 1e-10 per march output, 1e-9 for the
converged solution."""

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


def s02(wl):
    wl.tc = O.TC_S02
    return wl


def problem(wl):
    return O.Problem(wl.a0, wl.b0, wl.nx, wl.dt, wl.nt, wl.off.astype(np.int64), wl.u0, wl.V,
                     vkind=wl.vkind, tc=wl.tc, sigma=wl.sigma, nl_coef=wl.nl_coef)


def gpu_plan(wl, chunk=None, **kw):
    from paper_1503_02564_gb300 import swr
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, tc=swr.SWR_TC_S02, vkind=wl.vkind,
                    tuning=None if chunk is None else {"chunk_L": chunk}, **kw)
    V = torch.tensor(np.ascontiguousarray(wl.V).ravel(), dtype=torch.float64, device="cuda")
    u0 = torch.tensor(wl.u0, dtype=torch.complex128, device="cuda")
    plan.build_interface(V, u0)
    return plan


def gpu_interface(plan):
    d = torch.zeros(plan.n_interface, dtype=torch.complex128, device="cuda")
    cols = torch.zeros(4 * plan.nsub * plan.nt, dtype=torch.complex128, device="cuda")
    plan.get_interface(d, cols)
    return d.cpu().numpy().reshape(plan.nblk, plan.nt), \
        cols.cpu().numpy().reshape(plan.nsub, 4, plan.nt)


def ragged(nx, nt, offs):
    wl = W.config2(nsub=len(offs) - 1, nx=nx, nt=nt)
    wl.off = np.array(offs, dtype=np.int32)
    return s02(wl)


CASES = {
    "config1_small": lambda: s02(W.config1(nx=241, nt=30, nsub=4)),
    "config2_N16_small": lambda: s02(W.config2(nsub=16, nx=4001, nt=40)),
    "ragged_tiny": lambda: ragged(301, 17, [0, 2, 37, 151, 160, 300]),
    "two_long": lambda: s02(W.config2(nsub=2, nx=20001, nt=12)),
    "long_history": lambda: s02(W.config1(nx=241, nt=150, nsub=6)),
}


@pytest.mark.parametrize("chunk", [4, 8, 12, 16])
@pytest.mark.parametrize("case", sorted(CASES))
def test_s02_build_interface_matches_oracle(case, chunk):
    """d = R 0 and the Toeplitz first columns with S_0^2 ends, every chunk
    length (the history sums run in one warp per end, in whichever CTA of a
    cluster holds the end)."""
    wl = CASES[case]()
    plan = gpu_plan(wl, chunk)
    d, cols = gpu_interface(plan)
    plan.destroy()
    P = problem(wl)
    assert rel(d, O.build_d(P)) < TOL_MARCH
    cols_ref = O.build_columns(P)
    assert rel(cols, cols_ref) < TOL_MARCH
    for j in range(wl.nsub):
        for q in range(4):
            nrm = np.linalg.norm(cols_ref[j, q])
            if nrm > 0:
                assert rel(cols[j, q], cols_ref[j, q]) < TOL_MARCH, (j, q)
            else:
                assert np.all(cols[j, q] == 0)


@pytest.mark.parametrize("case", ["config1_small", "config2_N16_small", "ragged_tiny", "two_long"])
def test_s02_apply_R_matches_oracle(case):
    wl = CASES[case]()
    plan = gpu_plan(wl)
    g = W.random_interface(wl.nblk, wl.nt, 41)
    gi = torch.tensor(g.ravel(), dtype=torch.complex128, device="cuda")
    go = torch.zeros_like(gi)
    plan.apply_R(gi, go)
    plan.destroy()
    assert rel(go.cpu().numpy(), O.apply_R(problem(wl), g)) < TOL_MARCH


def _solve(plan, wl):
    g = torch.zeros(plan.n_interface, dtype=torch.complex128, device="cuda")
    uT = torch.zeros(wl.nx, dtype=torch.complex128, device="cuda")
    info = plan.solve(g, False, uT)
    return g.cpu().numpy(), uT.cpu().numpy(), info


@pytest.mark.parametrize("precond", [0, 2])
@pytest.mark.parametrize("case", ["config1_small", "ragged_tiny", "long_history"])
def test_s02_gmres_reproduces_monodomain(case, precond):
    """Converged SWR with S_0^2 equals the monodomain CN solution (S_0^2 is
    invertible: lower-triangular Toeplitz with c2 beta_0 != 0)."""
    wl = CASES[case]()
    plan = gpu_plan(wl, restart=100, maxit=1000, tol_abs=1e-12, precond=precond)
    g, uT, info = _solve(plan, wl)
    plan.destroy()
    gs, uTm = O.mono_interface(problem(wl))
    assert info["residual"] < 1e-12, info
    assert rel(uT, uTm) < TOL_SOLVE
    assert rel(g, gs) < TOL_SOLVE
    assert info["interface_jump"] < 1e-9


def test_s02_classical_iteration_matches_gmres():
    """Algorithm 1 with S_0^2 (the potential strategy converges in few sweeps)
    reaches the GMRES solution."""
    from paper_1503_02564_gb300 import swr
    wl = CASES["config1_small"]()
    pg = gpu_plan(wl, restart=100, tol_abs=1e-12)
    g1, uT1, _ = _solve(pg, wl)
    pg.destroy()
    pc = gpu_plan(wl, solver=swr.SWR_SOLVER_CLASSICAL, maxit=2000, tol_abs=1e-11)
    g2, uT2, info = _solve(pc, wl)
    pc.destroy()
    assert info["status"] == swr.SWR_OK, info
    assert rel(uT2, uT1) < TOL_SOLVE


def test_s02_time_dependent_apply_R_matches_oracle():
    """V(t,x) with S_0^2 ends (streamed per-step factors)."""
    from paper_1503_02564_gb300 import swr
    wl = s02(W.config4(nsub=4, nx=2001, nt=40))
    plan = gpu_plan(wl)
    assert plan.get_stats()["march_variant"] == swr.MARCH_TDEP_STREAMED
    g = W.random_interface(wl.nblk, wl.nt, 42)
    gi = torch.tensor(g.ravel(), dtype=torch.complex128, device="cuda")
    go = torch.zeros_like(gi)
    plan.apply_R(gi, go)
    plan.destroy()
    assert rel(go.cpu().numpy(), O.apply_R(problem(wl), g)) < TOL_MARCH


@pytest.mark.parametrize("nsub,nx", [(4, 801), (2, 20001)])
def test_s02_nonlinear_apply_R_matches_oracle(nsub, nx):
    """|u|^2 nonlinearity with S_0^2 ends (one CTA per system, and a cluster)."""
    from paper_1503_02564_gb300 import swr
    wl = s02(W.config5(nsub=nsub, nx=nx, nt=20))
    plan = gpu_plan(wl, solver=swr.SWR_SOLVER_FIXED_POINT, precond=swr.SWR_PC_ZERO_POTENTIAL)
    g = W.random_interface(wl.nblk, wl.nt, 43) * 1e-2
    gi = torch.tensor(g.ravel(), dtype=torch.complex128, device="cuda")
    go = torch.zeros_like(gi)
    plan.apply_R(gi, go)
    plan.destroy()
    assert rel(go.cpu().numpy(), O.apply_R(problem(wl), g)) < TOL_MARCH


@pytest.mark.parametrize("nsub", [16, 500])
def test_s02_full_size_scaling_config_against_monodomain(nsub):
    """Full-size scaling workload (200001 nodes, 500 steps) with S_0^2:
    converged u(T) and g against the monodomain solution."""
    from paper_1503_02564_gb300 import swr
    wl = s02(W.config2(nsub=nsub))
    plan = gpu_plan(wl, precond=swr.SWR_PC_CAUSAL, restart=30, tol_abs=1e-11)
    g, uT, info = _solve(plan, wl)
    plan.destroy()
    gs, uTm = O.mono_interface(problem(wl))
    assert info["residual"] < 1e-11, info
    assert rel(uT, uTm) < TOL_SOLVE
    assert rel(g, gs) < TOL_SOLVE
