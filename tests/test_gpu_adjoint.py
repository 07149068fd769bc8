"""GPU gradient of the final-time misfit J(V) = ||u(T) - u_target||_M^2 through
the converged SWR solution (swr_adjoint): against the oracle's discrete adjoint
of the monodomain scheme, against central differences of the GPU forward solve
(16 seeded directions, 1e-6 relative), invariance under the checkpoint interval,
and the torch.autograd.Function wrapper; with Robin and with S_0^2 transmission
(the segment marches then carry the ends' trace histories across checkpoints;
the gradient is the monodomain one whatever the condition)."""
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
                     wl.V if V is None else V, vkind=wl.vkind, tc=wl.tc, sigma=wl.sigma)


def target(wl, seed=5):
    rng = np.random.default_rng(seed)
    return (wl.u0 * np.exp(0.4j) + 0.05 * (rng.standard_normal(wl.nx)
                                           + 1j * rng.standard_normal(wl.nx)))


CASES = {
    "config1_small": lambda: W.config1(nx=241, nt=60, nsub=4),
    "config2_N16_small": lambda: W.config2(nsub=16, nx=4001, nt=40),
    "two_long": lambda: W.config2(nsub=2, nx=20001, nt=12),
}


def gpu_gradient(wl, tgt, K=16, V=None, tc=None, tuning=None):
    from paper_1503_02564_gb300 import swr
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, p=wl.sigma, restart=100, maxit=1000, tol_abs=1e-13,
                    precond=swr.SWR_PC_CAUSAL, tc=swr.SWR_TC_ROBIN if tc is None else tc,
                    tuning=tuning)
    Vt = torch.tensor(wl.V if V is None else V, dtype=torch.float64, device="cuda")
    plan.build_interface(Vt, torch.tensor(wl.u0, dtype=torch.complex128, device="cuda"))
    uT = torch.empty(wl.nx, dtype=torch.complex128, device="cuda")
    plan.solve(None, False, uT)
    ubar = torch.empty_like(uT)
    J = plan.misfit(uT, torch.tensor(tgt, dtype=torch.complex128, device="cuda"), ubar)
    grad = torch.empty(wl.nx, dtype=torch.float64, device="cuda")
    if K is not None:
        plan.adjoint(ubar, grad, K)
    plan.destroy()
    return J, grad.cpu().numpy()


@pytest.mark.parametrize("tc", [O.TC_ROBIN, O.TC_S02])
@pytest.mark.parametrize("case", sorted(CASES))
def test_adjoint_gradient_matches_oracle(case, tc):
    wl = CASES[case]()
    tgt = target(wl)
    J, g = gpu_gradient(wl, tgt, tc=tc)
    Jo, go = O.adjoint_gradient(problem(wl), tgt)
    assert abs(J - Jo) <= 1e-10 * Jo
    assert rel(g, go) < 1e-8


@pytest.mark.parametrize("case", ["eight_2500", "config2_N16_small"])
def test_adjoint_two_level_record_and_gradient_marches(case):
    """The record and gradient marches in the two-level form (k_march_tl modes 1 and 2:
    eight 2501-node subdomains on clusters of seven CTAs, 500 separators each; sixteen
    251-node subdomains alone in their CTAs), in the modelled launch shapes, against the
    same marches with the cluster-wide or CTA-wide PCR (two_level -1), with checkpoints
    every 5 steps, and against the oracle's discrete adjoint."""
    wl = W.config2(nsub=8, nx=20001, nt=12) if case == "eight_2500" else CASES[case]()
    tgt = target(wl)
    J1, g1 = gpu_gradient(wl, tgt, K=5, tuning={"autotune": -1})
    J2, g2 = gpu_gradient(wl, tgt, K=5, tuning={"autotune": -1, "two_level": -1})
    assert rel(g1, g2) < 1e-11
    Jo, go = O.adjoint_gradient(problem(wl), tgt)
    assert abs(J1 - Jo) <= 1e-10 * Jo
    assert rel(g1, go) < 1e-8


@pytest.mark.parametrize("tc", [O.TC_ROBIN, O.TC_S02])
def test_adjoint_checkpoint_interval_does_not_change_the_gradient(tc):
    wl = CASES["config1_small"]()
    tgt = target(wl)
    ref = gpu_gradient(wl, tgt, K=60, tc=tc)[1]
    for K in (1, 7, 16, 59):
        assert rel(gpu_gradient(wl, tgt, K=K, tc=tc)[1], ref) < 1e-12, K


@pytest.mark.parametrize("tc", [O.TC_ROBIN, O.TC_S02])
def test_adjoint_gradient_against_central_differences(tc):
    """16 seeded directions, J from the GPU forward solve alone."""
    wl = CASES["config1_small"]()
    tgt = target(wl)
    J, g = gpu_gradient(wl, tgt, tc=tc)
    rng = np.random.default_rng(16)
    eps = 1e-4
    for _ in range(16):
        d = rng.standard_normal(wl.nx)
        jp = gpu_gradient(wl, tgt, K=None, V=wl.V + eps * d, tc=tc)[0]
        jm = gpu_gradient(wl, tgt, K=None, V=wl.V - eps * d, tc=tc)[0]
        fd = (jp - jm) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-6 * abs(fd)


def test_zero_target_gives_zero_gradient():
    """J = ||u(T)||_M^2 = ||u_0||_M^2 for every real V: the gradient vanishes."""
    wl = CASES["config1_small"]()
    _, g = gpu_gradient(wl, target(wl))
    _, g0 = gpu_gradient(wl, np.zeros(wl.nx, np.complex128))
    assert np.max(np.abs(g0)) <= 1e-9 * np.max(np.abs(g))


def test_autograd_function_backward_is_the_adjoint():
    from paper_1503_02564_gb300 import swr
    wl = CASES["config1_small"]()
    tgt = target(wl)
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, p=wl.sigma, restart=100, maxit=1000, tol_abs=1e-13,
                    precond=swr.SWR_PC_CAUSAL)
    V = torch.tensor(wl.V, dtype=torch.float64, device="cuda", requires_grad=True)
    u0 = torch.tensor(wl.u0, dtype=torch.complex128, device="cuda")
    ut = torch.tensor(tgt, dtype=torch.complex128, device="cuda")
    J = swr.SWRMisfit.apply(V, plan, u0, ut, 16)
    (3.0 * J).backward()
    plan.destroy()
    Jo, go = O.adjoint_gradient(problem(wl), tgt)
    assert abs(J.item() - Jo) <= 1e-10 * Jo
    assert rel(V.grad.cpu().numpy(), 3.0 * go) < 1e-8


def test_adjoint_requires_a_solved_supported_plan():
    from paper_1503_02564_gb300 import swr
    wl = W.config1(nx=241, nt=20, nsub=4)
    ubar = torch.zeros(wl.nx, dtype=torch.complex128, device="cuda")
    grad = torch.empty(wl.nx, dtype=torch.float64, device="cuda")
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, p=wl.sigma)
    with pytest.raises(swr.SWRError) as e:
        plan.adjoint(ubar, grad)
    assert e.value.status == swr.SWR_ERR_STATE
    plan.destroy()
    # the per-end-kernel conditions (S_0^3 and up) are not differentiated
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, tc=swr.SWR_TC_S03)
    plan.build_interface(torch.tensor(wl.V, dtype=torch.float64, device="cuda"),
                         torch.tensor(wl.u0, dtype=torch.complex128, device="cuda"))
    plan.solve(None, False, None)
    with pytest.raises(swr.SWRError) as e:
        plan.adjoint(ubar, grad)
    assert e.value.status == swr.SWR_ERR_UNSUPPORTED
    plan.destroy()
