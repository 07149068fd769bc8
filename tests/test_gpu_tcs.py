"""GPU parity for the higher-order transmission conditions of Section 2.2 for V(x):
S_0^3, S_0^4 (potential strategy) and S_1^2, S_1^4 (gauge change strategy), each a
convolution of the end trace with a kernel formed per end from the potential at the end
node and its normal derivative.  Against the oracle, which writes the operators out
from their printed definitions as weight matrices: d, the Toeplitz first columns and
R g per march output (1e-10), converged SWR against the monodomain solution (1e-9)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1503_02564_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_MARCH = 1e-10
TOL_SOLVE = 1e-9
TCS = [O.TC_S03, O.TC_S04, O.TC_S12, O.TC_S14]


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


def problem(wl, tc):
    return O.Problem(wl.a0, wl.b0, wl.nx, wl.dt, wl.nt, wl.off.astype(np.int64), wl.u0, wl.V,
                     vkind=wl.vkind, tc=tc, sigma=wl.sigma)


def gpu_plan(wl, tc, chunk=None, **kw):
    from paper_1503_02564_gb300 import swr
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, tc=tc, tuning=None if chunk is None else {"chunk_L": chunk},
                    **kw)
    plan.build_interface(torch.tensor(wl.V, dtype=torch.float64, device="cuda"),
                         torch.tensor(wl.u0, dtype=torch.complex128, device="cuda"))
    return plan


def ragged(nx, nt, offs):
    wl = W.config2(nsub=len(offs) - 1, nx=nx, nt=nt)
    wl.off = np.array(offs, dtype=np.int32)
    return wl


CASES = {
    "config1_small": lambda: W.config1(nx=241, nt=30, nsub=4),
    "config2_N16_small": lambda: W.config2(nsub=16, nx=4001, nt=40),
    "ragged_tiny": lambda: ragged(301, 17, [0, 2, 37, 151, 160, 300]),
    "two_long": lambda: W.config2(nsub=2, nx=20001, nt=12),
}


@pytest.mark.parametrize("chunk", [4, 12, 16])
@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("tc", TCS)
def test_build_interface_matches_oracle(tc, case, chunk):
    wl = CASES[case]()
    plan = gpu_plan(wl, tc, chunk)
    d = torch.zeros(plan.n_interface, dtype=torch.complex128, device="cuda")
    cols = torch.zeros(4 * plan.nsub * plan.nt, dtype=torch.complex128, device="cuda")
    plan.get_interface(d, cols)
    plan.destroy()
    P = problem(wl, tc)
    assert rel(d.cpu().numpy(), O.build_d(P)) < TOL_MARCH
    cref = O.build_columns(P)
    cg = cols.cpu().numpy().reshape(wl.nsub, 4, wl.nt)
    for j in range(wl.nsub):
        for q in range(4):
            nrm = np.linalg.norm(cref[j, q])
            if nrm > 0:
                assert rel(cg[j, q], cref[j, q]) < TOL_MARCH, (j, q)


@pytest.mark.parametrize("case", ["config1_small", "ragged_tiny", "two_long"])
@pytest.mark.parametrize("tc", TCS)
def test_apply_R_matches_oracle(tc, case):
    wl = CASES[case]()
    plan = gpu_plan(wl, tc)
    g = W.random_interface(wl.nblk, wl.nt, 41)
    gi = torch.tensor(g.ravel(), dtype=torch.complex128, device="cuda")
    go = torch.zeros_like(gi)
    plan.apply_R(gi, go)
    plan.destroy()
    assert rel(go.cpu().numpy(), O.apply_R(problem(wl, tc), g)) < TOL_MARCH


@pytest.mark.parametrize("solver", ["gmres", "bicgstab", "causal", "classical"])
@pytest.mark.parametrize("tc", TCS)
def test_converged_swr_is_the_monodomain_solution(tc, solver):
    from paper_1503_02564_gb300 import swr
    wl = CASES["config1_small"]()
    kw = dict(restart=100, maxit=2000, tol_abs=1e-12, precond=swr.SWR_PC_CAUSAL)
    if solver == "causal":
        kw["solver"] = swr.SWR_SOLVER_CAUSAL
    if solver == "bicgstab":
        kw["solver"] = swr.SWR_SOLVER_BICGSTAB
    if solver == "classical":
        kw = dict(solver=swr.SWR_SOLVER_CLASSICAL, maxit=2000, tol_abs=1e-11)
    plan = gpu_plan(wl, tc, **kw)
    g = torch.zeros(plan.n_interface, dtype=torch.complex128, device="cuda")
    uT = torch.zeros(wl.nx, dtype=torch.complex128, device="cuda")
    info = plan.solve(g, False, uT)
    plan.destroy()
    assert info["status"] == swr.SWR_OK, info
    gs, uTm = O.mono_interface(problem(wl, tc))
    assert rel(uT.cpu().numpy(), uTm) < TOL_SOLVE
    assert rel(g.cpu().numpy(), gs) < TOL_SOLVE
    assert info["interface_jump"] < 1e-8


@pytest.mark.parametrize("tc", [O.TC_S04, O.TC_S14])
def test_full_size_scaling_config_against_monodomain(tc):
    """Full-size scaling workload (200001 nodes, 500 steps, N = 64)."""
    from paper_1503_02564_gb300 import swr
    wl = W.config2(nsub=64)
    plan = gpu_plan(wl, tc, precond=swr.SWR_PC_CAUSAL, restart=30, tol_abs=1e-11)
    g = torch.zeros(plan.n_interface, dtype=torch.complex128, device="cuda")
    uT = torch.zeros(wl.nx, dtype=torch.complex128, device="cuda")
    info = plan.solve(g, False, uT)
    plan.destroy()
    gs, uTm = _mono(wl, tc)
    assert info["residual"] < 1e-11, info
    assert rel(uT.cpu().numpy(), uTm) < TOL_SOLVE
    assert rel(g.cpu().numpy(), gs) < TOL_SOLVE


_MONO = {}


def _mono(wl, tc):
    if tc not in _MONO:
        _MONO[tc] = O.mono_interface(problem(wl, tc))
    return _MONO[tc]


def test_batch_with_higher_order_condition_matches_oracle():
    from paper_1503_02564_gb300 import swr
    wls = [W.config1(nx=241, nt=30, nsub=4), ragged(301, 17, [0, 2, 37, 151, 160, 300])]
    wls[1].dt = wls[0].dt
    wls[1].a0, wls[1].b0 = 0.0, 300 * ((wls[0].b0 - wls[0].a0) / (wls[0].nx - 1))
    insts = [dict(nx=w.nx, a0=w.a0, b0=w.b0, nt=w.nt, nsub=w.nsub, node_off=w.off) for w in wls]
    plan = swr.BatchPlan(insts, dt=wls[0].dt, tc=swr.SWR_TC_S14, restart=60, tol_abs=1e-12,
                         precond=swr.SWR_PC_CAUSAL)
    V = torch.tensor(np.concatenate([w.V for w in wls]), dtype=torch.float64, device="cuda")
    u0 = torch.tensor(np.concatenate([w.u0 for w in wls]), dtype=torch.complex128, device="cuda")
    plan.build_interface(V, u0)
    uT = torch.zeros(plan.nx, dtype=torch.complex128, device="cuda")
    info = plan.solve(None, False, uT)
    plan.destroy()
    assert info["status"] == swr.SWR_OK, info
    u = uT.cpu().numpy()
    k = 0
    for w in wls:
        _, uTm = O.mono_interface(problem(w, O.TC_S14))
        assert rel(u[k:k + w.nx], uTm) < TOL_SOLVE
        k += w.nx


def test_higher_order_conditions_are_refused_where_not_built():
    from paper_1503_02564_gb300 import swr
    wl = W.config4(nsub=4, nx=801, nt=20)
    for kw in (dict(vkind=swr.SWR_V_TIME), dict(precond=swr.SWR_PC_ZERO_POTENTIAL)):
        with pytest.raises(swr.SWRError) as e:
            swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                     node_off=wl.off, tc=swr.SWR_TC_S04, **kw)
        assert e.value.status == swr.SWR_ERR_UNSUPPORTED
