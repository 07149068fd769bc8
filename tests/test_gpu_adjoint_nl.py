"""GPU gradient dJ/dV0 of the final-time misfit through the nonlinear scheme
(Eq. CNS_NL with f(v) = c|v|^2, static V0; swr_adjoint on a nonlinear plan):
against the oracle's discrete adjoint of the monodomain scheme (the inner
fixed points and the linearised adjoint steps solved exactly there) on small
grids, on the one-system cluster of the 20001-node grid and on the full-size
workload (stored oracle gradient); against central differences of the GPU
forward SWR solve in 16 seeded directions (1e-6); invariance under the
checkpoint interval."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1503_02564_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


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


def problem(wl, V=None):
    return O.Problem(wl.a0, wl.b0, wl.nx, wl.dt, wl.nt, wl.off.astype(np.int64), wl.u0,
                     wl.V if V is None else V, vkind=wl.vkind, tc=wl.tc, sigma=wl.sigma,
                     nl_coef=wl.nl_coef, nl_tol=1e-13, nl_maxit=50)


CASES = {
    "small": lambda: W.config5(nsub=4, nx=801, nt=30),
    "N16": lambda: W.config5(nsub=16, nx=4001, nt=24),
    "one_cluster_20001": lambda: W.config5(nsub=4, nx=20001, nt=10),
}


LAST_ADJOINT_STATS = {}


def gpu_gradient(wl, tgt, K=16, V=None, tc=None, tuning=None):
    from paper_1503_02564_gb300 import swr
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, p=wl.sigma, vkind=swr.SWR_V_NONLINEAR,
                    tc=swr.SWR_TC_ROBIN if tc is None else tc,
                    solver=swr.SWR_SOLVER_FIXED_POINT, precond=swr.SWR_PC_MEAN_POTENTIAL,
                    maxit=500, tol_abs=1e-12, nl_tol=1e-13, nl_maxit=50, tuning=tuning)
    Vt = torch.tensor(wl.V if V is None else V, dtype=torch.float64, device="cuda")
    plan.build_interface(Vt, torch.tensor(wl.u0, dtype=torch.complex128, device="cuda"))
    uT = torch.empty(wl.nx, dtype=torch.complex128, device="cuda")
    plan.solve(None, False, uT)
    ubar = torch.empty_like(uT)
    J = plan.misfit(uT, torch.tensor(tgt, dtype=torch.complex128, device="cuda"), ubar)
    grad = torch.empty(wl.nx, dtype=torch.float64, device="cuda")
    if K is not None:
        plan.get_stats(reset=True)
        plan.adjoint(ubar, grad, K)
        LAST_ADJOINT_STATS.clear()
        LAST_ADJOINT_STATS.update(plan.get_stats())
    plan.destroy()
    return J, grad.cpu().numpy()


@pytest.mark.parametrize("case", sorted(CASES))
def test_nonlinear_adjoint_gradient_matches_oracle(case):
    wl = CASES[case]()
    tgt = W.misfit_target(wl)
    J, g = gpu_gradient(wl, tgt)
    Jo, go = O.adjoint_gradient_nl(problem(wl), tgt)
    assert abs(J - Jo) <= 1e-10 * Jo
    assert rel(g, go) < 1e-8


@pytest.mark.parametrize("case", ["small", "N16", "one_cluster_20001"])
@pytest.mark.parametrize("K", [None, 4])
def test_nonlinear_gradient_two_level_matches_cluster_pcr(case, K):
    """The gradient's monodomain marches with the two-level separator solve (warp blocks
    of 32 and a reduced system of the super-separators: 6 and 26 of them on clusters of 2
    and 12 CTAs, solved by one warp; 126 on 16 CTAs of the 20001-node grid, solved by PCR
    over each CTA) against the same marches with the cluster-wide PCR (two_level -1):
    one segment about the solve's record (the adjoint march), and segments of 4 steps
    (the forward march from checkpoints, its record, the adjoint march)."""
    wl = CASES[case]()
    tgt = W.misfit_target(wl)
    Kr = wl.nt if K is None else K
    _, g_tl = gpu_gradient(wl, tgt, K=Kr)
    _, g_pcr = gpu_gradient(wl, tgt, K=Kr, tuning={"two_level": -1})
    assert rel(g_tl, g_pcr) < 1e-11
    _, go = O.adjoint_gradient_nl(problem(wl), tgt)
    assert rel(g_tl, go) < 1e-8


def test_nonlinear_adjoint_with_s02_plan():
    """The gradient is the monodomain one whatever transmission condition the
    forward SWR solve used."""
    from paper_1503_02564_gb300 import swr
    wl = CASES["small"]()
    tgt = W.misfit_target(wl)
    _, g = gpu_gradient(wl, tgt, tc=swr.SWR_TC_S02)
    _, go = O.adjoint_gradient_nl(problem(wl), tgt)
    assert rel(g, go) < 1e-8


def test_nonlinear_checkpoint_interval_does_not_change_the_gradient():
    """Checkpointed segments (the forward trajectory recomputed by the monodomain march
    from checkpoints of u) give the same gradient for every interval."""
    wl = CASES["small"]()
    tgt = W.misfit_target(wl)
    ref = gpu_gradient(wl, tgt, K=15)[1]
    for K in (1, 7, 29):
        assert rel(gpu_gradient(wl, tgt, K=K)[1], ref) < 1e-11, K


@pytest.mark.parametrize("case", ["small", "N16", "one_cluster_20001"])
def test_nonlinear_adjoint_from_the_solves_record(case):
    """With one segment (K = nt) the adjoint march runs about the v_n that the solve's
    final march recorded (the converged SWR trajectory, from the subdomain marches in
    their tuned shapes); with two segments the monodomain march recomputes them.  The SWR
    trajectory equals the monodomain one to the solve's tolerance (interface residual
    below 1e-12 here), so the two gradients agree far below the oracle tolerance, and
    both match the oracle's discrete adjoint."""
    wl = CASES[case]()
    tgt = W.misfit_target(wl)
    J, g_rec = gpu_gradient(wl, tgt, K=wl.nt)
    assert LAST_ADJOINT_STATS["nl_march_launches"] == 1      # the adjoint march alone
    _, g_seg = gpu_gradient(wl, tgt, K=(wl.nt + 1) // 2)
    assert LAST_ADJOINT_STATS["nl_march_launches"] == 5      # 1 + 2 x (record, adjoint)
    _, go = O.adjoint_gradient_nl(problem(wl), tgt)
    assert rel(g_rec, g_seg) < 1e-10
    assert rel(g_rec, go) < 1e-8
    assert rel(g_seg, go) < 1e-8


def test_nonlinear_adjoint_against_central_differences():
    """16 seeded directions, J from the GPU forward SWR solve alone."""
    wl = CASES["small"]()
    tgt = W.misfit_target(wl)
    J, g = gpu_gradient(wl, tgt)
    rng = np.random.default_rng(16)
    eps = 1e-4
    for _ in range(16):
        d = rng.standard_normal(wl.nx)
        jp = gpu_gradient(wl, tgt, K=None, V=wl.V + eps * d)[0]
        jm = gpu_gradient(wl, tgt, K=None, V=wl.V - eps * d)[0]
        fd = (jp - jm) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-6 * abs(fd)


def test_nonlinear_adjoint_full_size_against_oracle_and_differences():
    """Full-size nonlinear workload (20001 nodes, 1000 steps, N = 32, checkpoints
    every 50 steps), the misfit target being u(T) for the seeded perturbed potential
    (computed by the oracle).  (1) The gradient against the oracle's, stored by
    tests/golden/make_nl_gradient.py (1e-9 relative).  (2) Central differences
    of the GPU forward SWR solve in 16 seeded directions d, fourth order,
    (8 (J(+e) - J(-e)) - (J(+2e) - J(-2e))) / (12 e) with e = 1e-3, to 1e-6
    relative to max(|fd|, |g|): for Gaussian d the directional derivative g.d
    has the size |g|.  The SWR value of J differs from the monodomain one by
    about 1e-12 relative (the outer iteration stops at residual 4e-11), and
    that difference moves smoothly with V: its derivative, about 1e-9, is what
    bounds the agreement, so a direction with a small derivative is measured
    against the gradient's own scale."""
    import os
    from paper_1503_02564_gb300 import swr
    wl = W.config5()
    gold = np.load(os.path.join(os.path.dirname(__file__), "golden", "nl_gradient_config5.npz"))
    tgt = gold["u_target"]     # the oracle's u(T) for the seeded perturbed potential

    def run(V, K):
        plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                        node_off=wl.off, p=wl.sigma, vkind=swr.SWR_V_NONLINEAR,
                        solver=swr.SWR_SOLVER_FIXED_POINT, precond=swr.SWR_PC_MEAN_POTENTIAL,
                        maxit=200, tol_abs=1e-10, nl_tol=1e-13, nl_maxit=50)
        plan.build_interface(torch.tensor(V, dtype=torch.float64, device="cuda"),
                             torch.tensor(wl.u0, dtype=torch.complex128, device="cuda"))
        uT = torch.empty(wl.nx, dtype=torch.complex128, device="cuda")
        plan.solve(None, False, uT)
        ubar = torch.empty_like(uT)
        J = plan.misfit(uT, torch.tensor(tgt, dtype=torch.complex128, device="cuda"), ubar)
        grad = torch.empty(wl.nx, dtype=torch.float64, device="cuda")
        if K:
            plan.adjoint(ubar, grad, K)
        plan.destroy()
        return J, grad.cpu().numpy()

    J, g = run(wl.V, 50)
    assert abs(J - float(gold["J"])) <= 1e-10 * J
    assert rel(g, gold["grad"]) < 1e-9
    rng = np.random.default_rng(17)
    eps = 1e-3
    scale = np.linalg.norm(g)
    for _ in range(16):
        d = rng.standard_normal(wl.nx)
        j1 = run(wl.V + eps * d, 0)[0] - run(wl.V - eps * d, 0)[0]
        j2 = run(wl.V + 2 * eps * d, 0)[0] - run(wl.V - 2 * eps * d, 0)[0]
        fd = (8.0 * j1 - j2) / (12.0 * eps)
        assert abs(fd - g @ d) <= 1e-6 * max(abs(fd), scale)


def test_nonlinear_adjoint_requires_a_solved_plan():
    from paper_1503_02564_gb300 import swr
    wl = W.config5(nsub=4, nx=401, nt=10)
    ubar = torch.zeros(wl.nx, dtype=torch.complex128, device="cuda")
    grad = torch.empty(wl.nx, dtype=torch.float64, device="cuda")
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, p=wl.sigma, vkind=swr.SWR_V_NONLINEAR,
                    solver=swr.SWR_SOLVER_FIXED_POINT)
    plan.build_interface(torch.tensor(wl.V, dtype=torch.float64, device="cuda"),
                         torch.tensor(wl.u0, dtype=torch.complex128, device="cuda"))
    with pytest.raises(swr.SWRError) as e:
        plan.adjoint(ubar, grad)
    assert e.value.status == swr.SWR_ERR_STATE
    plan.destroy()
