"""GPU parity of the FFT form of the causal substitution's history sums.

The substitution x = (I - L)^{-1} y adds, at every step, the lags > 3 of the four Toeplitz
blocks feeding an interface.  By default (nt >= 64, single instance) it splits them at
blocks of 32 steps: the last two blocks summed as the values arrive, the older ones as
64-point FFT convolutions.  Checked here against the direct sums of the same launch
(tuning.history_fft = -1) to rounding, and against the oracle's interface operator:
(I - L) x = y to 1e-12 on wide subdomains, where the same-step corner couplings vanish and
the substitution is exact.  The step counts put block boundaries and partial last blocks
at every place that matters: nt = 64 (two full blocks, no far part used), 65, 95, 96, 97
(the far part of block 2 starts), 200, 500 and 1000."""
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
    return S


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def substitute(swr, wl, history_fft, seed=3):
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, p=wl.sigma, precond=swr.SWR_PC_CAUSAL,
                    tuning={"history_fft": history_fft})
    plan.build_interface(torch.tensor(wl.V, dtype=torch.float64, device="cuda"),
                         torch.tensor(wl.u0, dtype=torch.complex128, device="cuda"))
    cols = torch.zeros(4 * wl.nsub * wl.nt, dtype=torch.complex128, device="cuda")
    plan.get_interface(None, cols)
    y = torch.tensor(W.random_interface(wl.nblk, wl.nt, seed).ravel(), dtype=torch.complex128,
                     device="cuda")
    x = torch.full_like(y, complex("nan"))
    plan.apply_precond(y, x)
    st = plan.get_stats()
    plan.destroy()
    return x.cpu().numpy(), y.cpu().numpy(), cols.cpu().numpy(), st


@pytest.mark.parametrize("nt", [64, 65, 95, 96, 97, 200, 500, 1000])
def test_fft_history_matches_direct_and_the_oracle(swr, nt):
    wl = W.config2(nsub=8, nx=8001, nt=nt)
    xf, y, cols, st = substitute(swr, wl, 0)
    xd, _, _, _ = substitute(swr, wl, -1)
    assert st["causal_window"] == 0
    assert rel(xf, xd) < 1e-12
    P = O.Problem(wl.a0, wl.b0, wl.nx, wl.dt, wl.nt, wl.off.astype(np.int64), wl.u0, wl.V,
                  sigma=wl.sigma)
    # the library's own columns in the oracle's operator: this isolates the substitution
    cols = cols.reshape(wl.nsub, 4, wl.nt)
    assert rel(O.apply_I_minus_L(P, cols, xf).ravel(), y) < 1e-12


@pytest.mark.parametrize("nsub,nt", [(256, 500), (500, 200), (64, 130)])
def test_fft_history_window_and_sweep_free_forms(swr, nsub, nt):
    """The scaling grid: windows H = 3 and H = 6 (same-step coupling solved) and H = 0."""
    wl = W.config2(nsub=nsub, nt=nt)
    xf, _, _, st = substitute(swr, wl, 0, seed=11)
    xd, _, _, _ = substitute(swr, wl, -1, seed=11)
    assert (st["causal_window"] > 0) == (nsub >= 256)
    assert rel(xf, xd) < 1e-12


def test_fft_history_solves_to_the_monodomain_solution(swr):
    """A full solve (GMRES preconditioned by the substitution with the FFT history)."""
    wl = W.config2(nsub=16, nx=16001, nt=300)
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, p=wl.sigma, precond=swr.SWR_PC_CAUSAL)
    plan.build_interface(torch.tensor(wl.V, dtype=torch.float64, device="cuda"),
                         torch.tensor(wl.u0, dtype=torch.complex128, device="cuda"))
    g = torch.zeros(plan.n_interface, dtype=torch.complex128, device="cuda")
    uT = torch.zeros(wl.nx, dtype=torch.complex128, device="cuda")
    info = plan.solve(g, False, uT)
    plan.destroy()
    P = O.Problem(wl.a0, wl.b0, wl.nx, wl.dt, wl.nt, wl.off.astype(np.int64), wl.u0, wl.V,
                  sigma=wl.sigma)
    gs, uTm = O.mono_interface(P)
    assert info["residual"] < 1e-10
    assert rel(uT.cpu().numpy(), uTm) < 1e-9
    assert rel(g.cpu().numpy(), gs.ravel()) < 1e-9


@pytest.mark.parametrize("nt", [100, 300])
def test_fft_history_for_the_mean_potential_preconditioner(swr, nt):
    """V(t,x) with the mean-potential preconditioner: the substitution runs on the
    operator L_0 of the time-averaged potential, whose spectra are formed at each build."""
    wl = W.config4(nsub=8, nx=8001, nt=nt)
    out = []
    for hf in (0, -1):
        plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                        node_off=wl.off, p=wl.sigma, vkind=swr.SWR_V_TIME,
                        precond=swr.SWR_PC_MEAN_POTENTIAL, tuning={"history_fft": hf})
        plan.build_interface(torch.tensor(np.ascontiguousarray(wl.V).ravel(),
                                          dtype=torch.float64, device="cuda"),
                             torch.tensor(wl.u0, dtype=torch.complex128, device="cuda"))
        y = torch.tensor(W.random_interface(wl.nblk, wl.nt, 4).ravel(),
                         dtype=torch.complex128, device="cuda")
        x = torch.full_like(y, complex("nan"))
        plan.apply_precond(y, x)
        plan.destroy()
        out.append(x.cpu().numpy())
    assert np.all(np.isfinite(out[0]))
    assert rel(out[0], out[1]) < 1e-12
