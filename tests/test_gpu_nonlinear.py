"""GPU parity for the nonlinear potential |u|^2 + V0(x) (Durán–Sanz-Serna scheme,
Eq. CNS_NL; inner fixed point of Eq. AvMNL per step; preconditioned outer fixed
point of Section 5)."""
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
                     vkind=wl.vkind, tc=wl.tc, sigma=wl.sigma, nl_coef=wl.nl_coef,
                     nl_tol=1e-13, nl_maxit=50)


def gpu_plan(wl, **kw):
    from paper_1503_02564_gb300 import swr
    kw.setdefault("solver", swr.SWR_SOLVER_FIXED_POINT)
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, p=wl.sigma, vkind=wl.vkind, nl_tol=1e-13, nl_maxit=50,
                    **kw)
    V = torch.tensor(wl.V, dtype=torch.float64, device="cuda")
    u0 = torch.tensor(wl.u0, dtype=torch.complex128, device="cuda")
    plan.build_interface(V, u0)
    return plan


def ragged_nl():
    wl = W.config5(nsub=4, nx=401, nt=20)
    wl.off = np.array([0, 2, 150, 333, 400], dtype=np.int32)
    return wl


CASES = {
    "config5_small": lambda: W.config5(nsub=4, nx=2001, nt=40),
    "config5_N16": lambda: W.config5(nsub=16, nx=4001, nt=30),
    "ragged": ragged_nl,
    "two_long": lambda: W.config5(nsub=2, nx=20001, nt=8),   # one system per cluster
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_nonlinear_apply_R_matches_oracle(case):
    wl = CASES[case]()
    plan = gpu_plan(wl)
    g = 0.05 * W.random_interface(wl.nblk, wl.nt, 41)
    gi = torch.tensor(g.ravel(), dtype=torch.complex128, device="cuda")
    go = torch.zeros_like(gi)
    plan.apply_R(gi, go)
    plan.destroy()
    assert rel(go.cpu().numpy(), O.apply_R(problem(wl), g)) < TOL_MARCH


@pytest.mark.parametrize("case", ["config5_small", "config5_N16", "ragged"])
@pytest.mark.parametrize("L", [2, 4, 8])
def test_nonlinear_apply_R_fixed_chunk_length(case, L):
    """The nonlinear march with each chunk length it is built for, in the modelled launch
    shape: with 2-node chunks config5_small's subdomains (168 separators) spread over
    clusters of two CTAs (two-level separator solve), the others run one per CTA; the
    ragged case has a subdomain of three nodes (one chunk of one node)."""
    wl = CASES[case]()
    plan = gpu_plan(wl, tuning={"chunk_L": L, "autotune": -1})
    g = 0.05 * W.random_interface(wl.nblk, wl.nt, 47)
    gi = torch.tensor(g.ravel(), dtype=torch.complex128, device="cuda")
    go = torch.zeros_like(gi)
    plan.apply_R(gi, go)
    plan.destroy()
    assert rel(go.cpu().numpy(), O.apply_R(problem(wl), g)) < TOL_MARCH


@pytest.mark.parametrize("precond", [0, 1, 3])
def test_nonlinear_solve_reproduces_monodomain(precond):
    """precond 0 is the classical iteration g <- R_nl g, which needs a contracting
    interface map: the paper's Robin form S = -ip with p = 20 (with the complex
    p of the workloads it diverges, as in the linear case)."""
    from paper_1503_02564_gb300 import swr
    wl = CASES["config5_small"]()
    if precond == 0:
        wl.sigma = -20j
    plan = gpu_plan(wl, precond=precond, maxit=500, tol_abs=1e-12)
    g = torch.zeros(plan.n_interface, dtype=torch.complex128, device="cuda")
    uT = torch.zeros(wl.nx, dtype=torch.complex128, device="cuda")
    info = plan.solve(g, False, uT)
    plan.destroy()
    gs, uTm = O.mono_interface(problem(wl))
    assert info["status"] == swr.SWR_OK
    assert rel(uT.cpu().numpy(), uTm) < TOL_SOLVE
    assert rel(g.cpu().numpy(), gs) < TOL_SOLVE


def test_full_size_nonlinear_config_against_monodomain():
    """Full-size nonlinear workload (20001 nodes, 1000 steps, dt = 5e-4, N = 32):
    preconditioned fixed point of Section 5 with P = I - L_V0."""
    from paper_1503_02564_gb300 import swr
    wl = W.config5()
    gs, uTm = O.mono_interface(problem(wl))
    plan = gpu_plan(wl, precond=swr.SWR_PC_MEAN_POTENTIAL, maxit=200, tol_abs=1e-10)
    g = torch.zeros(plan.n_interface, dtype=torch.complex128, device="cuda")
    uT = torch.zeros(wl.nx, dtype=torch.complex128, device="cuda")
    info = plan.solve(g, False, uT)
    plan.destroy()
    print("full-size nonlinear solve:", info)
    assert rel(uT.cpu().numpy(), uTm) < TOL_SOLVE
    assert rel(g.cpu().numpy(), gs) < TOL_SOLVE


@pytest.mark.parametrize("vkind", [0, 2])
def test_cluster_path_is_bit_reproducible(vkind):
    """A subdomain spread over a thread-block cluster (one system per cluster) gives
    bit-identical outputs on repeated calls (its cross-CTA reductions are ordered)."""
    from paper_1503_02564_gb300 import swr
    wl = W.config5(nsub=2, nx=20001, nt=8)
    wl.vkind = vkind
    plan = gpu_plan(wl, solver=swr.SWR_SOLVER_FIXED_POINT if vkind == 2 else swr.SWR_SOLVER_GMRES)
    g = 0.05 * W.random_interface(wl.nblk, wl.nt, 41)
    gi = torch.tensor(g.ravel(), dtype=torch.complex128, device="cuda")
    outs = []
    for _ in range(6):
        go = torch.zeros_like(gi)
        plan.apply_R(gi, go)
        outs.append(go.cpu().numpy().tobytes())
    plan.destroy()
    assert len(set(outs)) == 1



def _nl_cluster_case(name):
    if name == "c7_empty_cta":      # 501 separators on 7 CTAs of 96 threads: the last has none
        return W.config5(nsub=8, nx=20001, nt=12)
    if name == "c6":                # 401 separators on 6 CTAs
        return W.config5(nsub=2, nx=4001, nt=12)
    wl = W.config5(nsub=4, nx=5121, nt=12)   # uneven: 145, 257, 301, 325 separators on 5 CTAs
    wl.off = np.array([0, 720, 2000, 3500, 5120], dtype=np.int32)
    return wl


@pytest.mark.parametrize("name", ["c7_empty_cta", "c6", "ragged_c5"])
def test_nonlinear_two_level_cluster_march_matches_oracle(name):
    """The nonlinear march of systems spread over a cluster with the two-level separator
    solve (warp-shuffle PCR in blocks of 32 and a reduced system of the super-separators,
    in the modelled launch shape with 4-node chunks), against the oracle's nonlinear R g
    and against the same launch with the cluster-wide PCR."""
    wl = _nl_cluster_case(name)
    g = 0.05 * W.random_interface(wl.nblk, wl.nt, 43)
    gi = torch.tensor(g.ravel(), dtype=torch.complex128, device="cuda")
    outs = []
    for tl in (0, -1):
        plan = gpu_plan(wl, tuning={"autotune": -1, "two_level": tl})
        go = torch.zeros_like(gi)
        plan.apply_R(gi, go)
        plan.destroy()
        outs.append(go.cpu().numpy())
    assert rel(outs[0], O.apply_R(problem(wl), g)) < TOL_MARCH
    assert rel(outs[0], outs[1]) < 1e-11
