"""swr_causal_solve_noalloc: the causal substitution for callers that cannot
allocate device memory (applications that reserve all device memory in their own
pool, or latency-critical loops that cannot take cudaMalloc's implicit device
synchronisation).  Its output must match the plan-based swr_apply_precond on the
same inputs, on two calls in a row (the second reuses the library array left
over from the first), and solve (I - L) x = y for the oracle's own L."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1503_02564_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-10   # same relative L2 tolerance as the march-level parity tests


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def swr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_02564_gb300 import build_ext, swr as S
    build_ext.build()
    return S


@pytest.mark.parametrize("sweeps", [0, 2, 5])
def test_no_alloc_causal_solve_matches_plan(swr, sweeps):
    wl = W.config2(nsub=8, nx=8001, nt=64)
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, p=wl.sigma, precond=swr.SWR_PC_CAUSAL, pc_sweeps=sweeps)
    V = torch.tensor(wl.V, dtype=torch.float64, device="cuda")
    u0 = torch.tensor(wl.u0, dtype=torch.complex128, device="cuda")
    plan.build_interface(V, u0)
    cols = torch.zeros(4 * wl.nsub * wl.nt, dtype=torch.complex128, device="cuda")
    plan.get_interface(None, cols)
    # the oracle's interface operator on the same problem: subdomains 12.5 wide, so the
    # same-step corner couplings (exp(-width / sqrt(dt)) ~ 1e-170) vanish and the
    # substitution is (I - L)^{-1} to rounding whatever the number of sweeps
    P = O.Problem(wl.a0, wl.b0, wl.nx, wl.dt, wl.nt, wl.off.astype(np.int64), wl.u0, wl.V,
                  sigma=wl.sigma)
    cols_or = O.build_columns(P)
    for call in range(2):
        y = torch.tensor(W.random_interface(wl.nblk, wl.nt, 20 + call).ravel(),
                         dtype=torch.complex128, device="cuda")
        x_ref = torch.zeros_like(y)
        plan.apply_precond(y, x_ref)
        x = torch.full_like(y, complex("nan"))
        st = swr.swr_causal_solve_noalloc(wl.nsub, wl.nt, sweeps, cols, y, x)
        torch.cuda.synchronize()
        assert st == swr.SWR_OK, swr.swr_status_string(st)
        xn, yn = x.cpu().numpy(), y.cpu().numpy()
        assert rel(xn, x_ref.cpu().numpy()) < TOL, call
        assert rel(O.apply_I_minus_L(P, cols_or, xn).ravel(), yn) < 1e-12, call
    plan.destroy()


def test_no_alloc_refuses_aliased_and_oversized_calls(swr):
    """x == y is refused; so is a call with more interfaces than one cooperative launch
    holds resident (N = 1024: 1023 CTAs of the substitution, above 152 SMs x 5)."""
    n, nt = 8, 4
    cols = torch.zeros(4 * n * nt, dtype=torch.complex128, device="cuda")
    y = torch.zeros((2 * n - 2) * nt, dtype=torch.complex128, device="cuda")
    assert swr.swr_causal_solve_noalloc(n, nt, 0, cols, y, y) == swr.SWR_ERR_ARG
    n_big = 1024
    cols = torch.zeros(4 * n_big * nt, dtype=torch.complex128, device="cuda")
    y = torch.zeros((2 * n_big - 2) * nt, dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(y)
    assert swr.swr_causal_solve_noalloc(n_big, nt, 0, cols, y, x) == swr.SWR_ERR_UNSUPPORTED


def test_no_alloc_rejects_sizes_beyond_its_array(swr):
    n_big = 1025
    nt = 2
    cols = torch.zeros(4 * n_big * nt, dtype=torch.complex128, device="cuda")
    y = torch.zeros((2 * n_big - 2) * nt, dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(y)
    assert swr.swr_causal_solve_noalloc(n_big, nt, 0, cols, y, x) == swr.SWR_ERR_ARG
    assert swr.swr_causal_solve_noalloc(4, nt, 17, cols[:4 * 4 * nt], y[:6 * nt],
                                        x[:6 * nt]) == swr.SWR_ERR_ARG
