"""GPU gradient of the final-time misfit with respect to a tabulated time-dependent
potential, dJ/dV(t_m, x) (swr_adjoint on a V(t,x) plan: the adjoint's SWR problem is
the forward one with the time axis reversed, its marches walk the per-step factors
backwards): against the oracle's discrete adjoint of the monodomain scheme
(oracle.adjoint_gradient_tdep), against fourth-order central differences of the GPU
forward solve, under a change of the checkpoint interval, with Robin and S_0^2 ends,
and the exact zero gradient of the conserved norm."""
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


def case(nsub=4, nx=1201, nt=30):
    wl = W.config4(nsub=nsub, nx=nx, nt=nt)
    rng = np.random.default_rng(21)
    tgt = wl.u0 * np.exp(0.3j) + 0.05 * (rng.standard_normal(wl.nx)
                                         + 1j * rng.standard_normal(wl.nx))
    return wl, tgt


def gpu_gradient(wl, tgt, K=7, V=None, tc=None):
    from paper_1503_02564_gb300 import swr
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, p=wl.sigma, vkind=swr.SWR_V_TIME, restart=60, maxit=400,
                    tol_abs=1e-13, precond=swr.SWR_PC_MEAN_POTENTIAL,
                    tc=swr.SWR_TC_ROBIN if tc is None else tc)
    Vt = torch.tensor(np.ascontiguousarray(wl.V if V is None else V).ravel(),
                      dtype=torch.float64, device="cuda")
    plan.build_interface(Vt, torch.tensor(wl.u0, dtype=torch.complex128, device="cuda"))
    assert plan.get_stats()["march_variant"] == swr.MARCH_TDEP_STREAMED
    uT = torch.empty(wl.nx, dtype=torch.complex128, device="cuda")
    plan.solve(None, False, uT)
    ubar = torch.empty_like(uT)
    J = plan.misfit(uT, torch.tensor(tgt, dtype=torch.complex128, device="cuda"), ubar)
    grad = torch.empty((wl.nt + 1) * wl.nx, dtype=torch.float64, device="cuda")
    if K is not None:
        plan.adjoint(ubar, grad, K)
    plan.destroy()
    return J, grad.cpu().numpy().reshape(wl.nt + 1, wl.nx)


def problem(wl, V=None):
    return O.Problem(wl.a0, wl.b0, wl.nx, wl.dt, wl.nt, wl.off.astype(np.int64), wl.u0,
                     wl.V if V is None else V, vkind=wl.vkind, sigma=wl.sigma)


@pytest.mark.parametrize("tc", [O.TC_ROBIN, O.TC_S02])
def test_tdep_adjoint_gradient_matches_oracle(tc):
    wl, tgt = case()
    J, g = gpu_gradient(wl, tgt, tc=tc)
    Jo, go = O.adjoint_gradient_tdep(problem(wl), tgt)
    assert abs(J - Jo) <= 1e-10 * Jo
    assert rel(g, go) < 1e-8


def test_tdep_adjoint_checkpoint_interval_does_not_change_the_gradient():
    wl, tgt = case()
    ref = gpu_gradient(wl, tgt, K=30)[1]
    for K in (1, 4, 13):
        assert rel(gpu_gradient(wl, tgt, K=K)[1], ref) < 1e-12, K


def test_tdep_adjoint_against_central_differences():
    """Four seeded directions of the whole (nt + 1) x nx table, J from the GPU forward
    solve alone, fourth-order differences."""
    wl, tgt = case()
    J, g = gpu_gradient(wl, tgt)
    rng = np.random.default_rng(22)
    eps = 1e-2
    for _ in range(4):
        d = rng.standard_normal(wl.V.shape)
        Jp = [gpu_gradient(wl, tgt, K=None, V=wl.V + k * eps * d)[0] for k in (1, -1, 2, -2)]
        fd = (8.0 * (Jp[0] - Jp[1]) - (Jp[2] - Jp[3])) / (12.0 * eps)
        assert abs(fd - np.sum(g * d)) <= 1e-6 * abs(fd)


def test_tdep_zero_target_gives_zero_gradient():
    """J = ||u(T)||_M^2 is conserved for every real V(t, x): the gradient vanishes."""
    wl, tgt = case()
    _, g = gpu_gradient(wl, tgt)
    _, g0 = gpu_gradient(wl, np.zeros(wl.nx, np.complex128))
    assert np.max(np.abs(g0)) <= 1e-9 * np.max(np.abs(g))
