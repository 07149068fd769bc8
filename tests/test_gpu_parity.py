"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (from the accuracy targets of the solver): relative L2 error at most
1e-10 per march output (d, Toeplitz columns, R g) and at most 1e-9 for the
converged SWR solution (interface vector and u(T)).  Both sides compute in
IEEE binary64; the GPU contracts multiply-adds and reorders sums, the oracle
does not, which with the condition numbers here (about 2 dt / h^2 <= 1e4)
leaves three orders of magnitude of margin.
"""

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


def gpu_plan(wl, chunk=None, autotune=True, tuning=None, **kw):
    from paper_1503_02564_gb300 import swr
    tuning = dict(tuning or {})
    if chunk is not None:
        tuning["chunk_L"] = chunk
    if not autotune:
        tuning["autotune"] = -1
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, p=wl.sigma, vkind=wl.vkind, tuning=tuning, **kw)
    V = torch.tensor(wl.V, dtype=torch.float64, device="cuda")
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
    return wl


CASES = {
    "config1_small": lambda: W.config1(nx=241, nt=30, nsub=4),
    "config1_full": lambda: W.config1(),
    "config2_N16_small": lambda: W.config2(nsub=16, nx=4001, nt=40),
    "ragged_tiny": lambda: ragged(301, 17, [0, 2, 37, 151, 160, 300]),
    "two_long": lambda: W.config2(nsub=2, nx=20001, nt=12),
}


@pytest.mark.parametrize("chunk", [4, 8, 12, 16])
@pytest.mark.parametrize("case", sorted(CASES))
def test_build_interface_matches_oracle(case, chunk):
    wl = CASES[case]()
    if case == "two_long" and chunk == 16:
        pytest.skip("covered by chunk 4/8 (cluster path)")
    plan = gpu_plan(wl, chunk)
    d, cols = gpu_interface(plan)
    P = problem(wl)
    d_ref = O.build_d(P)
    cols_ref = O.build_columns(P)
    assert rel(d, d_ref) < TOL_MARCH
    assert rel(cols, cols_ref) < TOL_MARCH
    for j in range(wl.nsub):
        for q in range(4):
            nrm = np.linalg.norm(cols_ref[j, q])
            if nrm > 0:
                assert rel(cols[j, q], cols_ref[j, q]) < TOL_MARCH, (j, q)
            else:
                assert np.all(cols[j, q] == 0)
    plan.destroy()


@pytest.mark.parametrize("case", ["config2_N16_small", "ragged_tiny", "two_long"])
def test_autotuned_shapes_match_modelled_shapes(case):
    """The measured launch shapes (first build) and the modelled ones
    (tuning.autotune = -1) partition the same systems differently; both give the
    oracle's d and columns, and agree with each other to rounding, also after
    a second build on the tuned plan."""
    wl = CASES[case]()
    pt = gpu_plan(wl)
    d1, c1 = gpu_interface(pt)
    V = torch.tensor(wl.V, dtype=torch.float64, device="cuda")
    u0 = torch.tensor(wl.u0, dtype=torch.complex128, device="cuda")
    pt.build_interface(V, u0)
    d2, c2 = gpu_interface(pt)
    pt.destroy()
    pm = gpu_plan(wl, autotune=False)
    dm, cm = gpu_interface(pm)
    pm.destroy()
    assert np.array_equal(d1, d2) and np.array_equal(c1, c2)
    assert rel(d1, dm) < 1e-12 and rel(c1, cm) < 1e-12
    d_ref = O.build_d(problem(wl))
    assert rel(d1, d_ref) < TOL_MARCH


@pytest.mark.parametrize("case", ["config1_small", "config2_N16_small", "ragged_tiny", "two_long"])
def test_apply_R_matches_oracle(case):
    wl = CASES[case]()
    plan = gpu_plan(wl)
    g = W.random_interface(wl.nblk, wl.nt, 5)
    gi = torch.tensor(g.ravel(), dtype=torch.complex128, device="cuda")
    go = torch.zeros_like(gi)
    plan.apply_R(gi, go)
    ref = O.apply_R(problem(wl), g)
    assert rel(go.cpu().numpy(), ref) < TOL_MARCH
    plan.destroy()


@pytest.mark.parametrize("case", ["config1_small", "config1_full", "ragged_tiny"])
def test_apply_interface_matches_oracle(case):
    wl = CASES[case]()
    plan = gpu_plan(wl)
    P = problem(wl)
    cols = O.build_columns(P)
    x = W.random_interface(wl.nblk, wl.nt, 9)
    xi = torch.tensor(x.ravel(), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(xi)
    plan.apply_interface(xi, y)
    assert rel(y.cpu().numpy(), O.apply_I_minus_L(P, cols, x)) < TOL_MARCH
    plan.destroy()


def _solve(plan, wl):
    g = torch.zeros(plan.n_interface, dtype=torch.complex128, device="cuda")
    uT = torch.zeros(wl.nx, dtype=torch.complex128, device="cuda")
    info = plan.solve(g, False, uT)
    return g.cpu().numpy().reshape(wl.nblk, wl.nt), uT.cpu().numpy(), info


@pytest.mark.parametrize("precond", [0, 2])
@pytest.mark.parametrize("case", ["config1_small", "config1_full", "ragged_tiny"])
def test_gmres_solve_reproduces_monodomain(case, precond):
    from paper_1503_02564_gb300 import swr
    wl = CASES[case]()
    plan = gpu_plan(wl, restart=200, maxit=5000, tol_abs=1e-12,
                    precond=swr.SWR_PC_CAUSAL if precond == 2 else swr.SWR_PC_NONE)
    g, uT, info = _solve(plan, wl)
    gs, uTm = O.mono_interface(problem(wl))
    assert info["residual"] < 1e-12
    assert rel(uT, uTm) < TOL_SOLVE
    assert rel(g, gs) < TOL_SOLVE
    assert info["interface_jump"] < 1e-8
    if precond == 2:
        assert info["iterations"] <= 40, info
    plan.destroy()


def test_causal_preconditioner_is_near_inverse():
    """x = P^{-1} y with P = I - L: (I - L) x reproduces y up to the dropped
    lag-0 couplings across subdomains (corner entries of the subdomain inverse)."""
    from paper_1503_02564_gb300 import swr
    wl = W.config2(nsub=8, nx=8001, nt=64)
    plan = gpu_plan(wl, precond=swr.SWR_PC_CAUSAL)
    P = problem(wl)
    cols = O.build_columns(P)
    y = W.random_interface(wl.nblk, wl.nt, 11)
    yi = torch.tensor(y.ravel(), dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(yi)
    plan.apply_precond(yi, x)
    back = O.apply_I_minus_L(P, cols, x.cpu().numpy())
    assert rel(back, y) < 1e-6
    plan.destroy()


def test_fixed_point_and_classical_agree_with_gmres():
    """Algorithm 1 (g <- R g with full marches), Algorithm 3 with the fixed point
    (g <- L g + d) and GMRES converge to the same solution.  The fixed point
    needs a contracting L: the paper's Robin form S = -ip with p = 20."""
    from paper_1503_02564_gb300 import swr
    wl = W.config2(nsub=3, nx=2001, nt=40)
    wl.sigma = -20j
    ref = None
    for solver in (swr.SWR_SOLVER_GMRES, swr.SWR_SOLVER_FIXED_POINT, swr.SWR_SOLVER_CLASSICAL):
        plan = gpu_plan(wl, solver=solver, maxit=400)
        g, uT, info = _solve(plan, wl)
        plan.destroy()
        if ref is None:
            ref = uT
        assert rel(uT, ref) < TOL_SOLVE, (solver, info)
    _, uTm = O.mono_interface(problem(wl))
    assert rel(ref, uTm) < TOL_SOLVE


@pytest.mark.parametrize("nsub", [16, 64, 500])
def test_full_size_scaling_config_against_monodomain(nsub):
    """Full-size scaling workload (200001 nodes, 500 steps) in the benchmark's
    launch configuration: converged u(T) and g against the monodomain CN
    solution and the interface vector it implies (computed by the oracle)."""
    from paper_1503_02564_gb300 import swr
    wl = W.config2(nsub=nsub)
    plan = gpu_plan(wl, precond=swr.SWR_PC_CAUSAL, restart=30, tol_abs=1e-11)
    g, uT, info = _solve(plan, wl)
    plan.destroy()
    gs, uTm = _mono_cache(nsub, wl)
    assert info["residual"] < 1e-11, info
    assert rel(uT, uTm) < TOL_SOLVE
    assert rel(g, gs) < TOL_SOLVE


_MONO = {}


def _mono_cache(nsub, wl):
    if nsub not in _MONO:
        _MONO[nsub] = O.mono_interface(problem(wl))
    return _MONO[nsub]


@pytest.mark.parametrize("vkind", [0, 1])
def test_solve_with_null_outputs(vkind):
    """g and uT may be NULL in swr_solve (include/swr.h): nothing is written
    through them and the solve still reports its residual."""
    from paper_1503_02564_gb300 import swr
    wl = W.config1(nx=241, nt=30, nsub=4) if vkind == 0 else W.config4(nsub=4, nx=801, nt=20)
    plan = gpu_plan(wl, restart=100, maxit=400)
    info = plan.solve(None, False, None, allow_not_converged=True)
    plan.destroy()
    assert info["status"] in (swr.SWR_OK, swr.SWR_ERR_NOT_CONVERGED)
    assert np.isfinite(info["residual"])


@pytest.mark.parametrize("case", ["config2_N16_small", "two_long"])
def test_repeated_builds_replay_the_captured_build(case):
    """The second build is captured into a CUDA graph and later builds replay it:
    d and the first columns are bitwise those of a direct build, a replay reads
    the new V, and every build counts the same kernel launches."""
    from paper_1503_02564_gb300 import swr
    wl = CASES[case]()
    plan = gpu_plan(wl)                      # first build (direct, tuned)
    d1, c1 = gpu_interface(plan)
    V = torch.tensor(wl.V, dtype=torch.float64, device="cuda")
    u0 = torch.tensor(wl.u0, dtype=torch.complex128, device="cuda")
    counts = []
    for _ in range(3):                       # capture, then two replays
        k0 = swr.swr_kernel_launch_count()
        plan.build_interface(V, u0)
        counts.append(swr.swr_kernel_launch_count() - k0)
        d, c = gpu_interface(plan)
        assert np.array_equal(d, d1) and np.array_equal(c, c1)
    assert counts[0] == counts[1] == counts[2] > 0
    V2 = torch.tensor(wl.V * 0.5, dtype=torch.float64, device="cuda")
    plan.build_interface(V2, u0)             # replay with a different potential
    d3, _ = gpu_interface(plan)
    plan.destroy()
    wl2 = CASES[case]()
    wl2.V = wl.V * 0.5
    fresh = gpu_plan(wl2)
    d4, _ = gpu_interface(fresh)
    fresh.destroy()
    assert np.array_equal(d3, d4)
    assert rel(d3, O.build_d(problem(wl2))) < TOL_MARCH


def _solve_with(wl, superpose, **kw):
    from paper_1503_02564_gb300 import swr
    if "tc" in kw:
        wl.tc = kw["tc"]
    plan = gpu_plan(wl, tuning={"superpose": 0 if superpose else -1}, **kw)
    assert plan.get_stats()["superposed"] == (1 if superpose else 0)
    g, uT, info = _solve(plan, wl)
    plan.destroy()
    return g, uT, info


@pytest.mark.parametrize("tc", [0, 1, 3, 5])
@pytest.mark.parametrize("case", ["config1_small", "ragged_tiny", "config2_N16_small", "two_long"])
def test_superposed_final_state_matches_final_march(case, tc):
    """u(T) as the superposition of the build marches' recorded states (static V,
    Robin) against the final march with the same converged fluxes, and the
    interface mismatch from the final residual against the one from the final
    march's traces."""
    from paper_1503_02564_gb300 import swr
    wl = CASES[case]()
    kw = dict(precond=swr.SWR_PC_CAUSAL, restart=100, maxit=1000, tol_abs=1e-12, tc=tc)
    g1, u1, i1 = _solve_with(wl, True, **kw)
    g0, u0, i0 = _solve_with(wl, False, **kw)
    assert np.array_equal(g1, g0)          # the solve itself does not change
    assert rel(u1, u0) < 1e-12
    assert abs(i1["interface_jump"] - i0["interface_jump"]) <= 1e-12 + 1e-3 * i0["interface_jump"]
    assert i1["march_point_steps"] == 0 and i0["march_point_steps"] > 0
    _, uTm = O.mono_interface(problem(wl))
    assert rel(u1, uTm) < TOL_SOLVE


def test_superposed_final_state_null_uT_and_unconverged():
    """uT may be NULL; with an iteration cap the superposition still reproduces
    the final march of the (unconverged) fluxes, and the mismatch is nonzero."""
    from paper_1503_02564_gb300 import swr
    wl = CASES["config2_N16_small"]()
    out = []
    for sp in (True, False):
        plan = gpu_plan(wl, maxit=3, restart=30, tuning={"superpose": 0 if sp else -1})
        info = plan.solve(None, False, None, allow_not_converged=True)
        assert info["status"] == swr.SWR_ERR_NOT_CONVERGED
        uT = torch.zeros(wl.nx, dtype=torch.complex128, device="cuda")
        info = plan.solve(None, False, uT, allow_not_converged=True)
        out.append((uT.cpu().numpy(), info["interface_jump"]))
        plan.destroy()
    assert rel(out[0][0], out[1][0]) < 1e-12
    assert out[0][1] > 1e-6 and abs(out[0][1] - out[1][1]) <= 1e-9 * out[1][1]


@pytest.mark.parametrize("fft", [True, False])
@pytest.mark.parametrize("case", ["config1_small", "ragged_tiny", "config2_N16_small", "long_nt"])
def test_toeplitz_apply_fft_and_direct_match_oracle(case, fft):
    """(I - L) x and L x + d from the first columns, by the FFT (transform length
    the power of two >= 2 nt - 1) and by the direct causal sums, against the
    oracle's (I - L) x; nt = 1500 takes the largest transform (4096)."""
    from paper_1503_02564_gb300 import swr
    wl = W.config1(nx=241, nt=1500, nsub=4) if case == "long_nt" else CASES[case]()
    plan = gpu_plan(wl, tuning={"toeplitz_fft": 0 if fft else -1})
    M = plan.get_stats()["toeplitz_fft_length"]
    if fft:
        assert M >= 2 * wl.nt - 1 and M & (M - 1) == 0 and M < 4 * wl.nt
    else:
        assert M == 0
    P = problem(wl)
    cols = O.build_columns(P)
    x = W.random_interface(wl.nblk, wl.nt, 9)
    xi = torch.tensor(x.ravel(), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(xi)
    plan.apply_interface(xi, y)
    plan.destroy()
    assert rel(y.cpu().numpy(), O.apply_I_minus_L(P, cols, x)) < TOL_MARCH


def narrow(nsub=500, nx=20001, nt=40):
    """0.2-wide subdomains (40 intervals at h = 0.005, dt = 1e-3): the same-step
    coupling of neighbouring interfaces (lag-0 corner entries ~3e-4) matters."""
    return W.config2(nsub=nsub, nx=nx, nt=nt)


@pytest.mark.parametrize("pc_sweeps", [-1, 0, 1])
def test_causal_window_makes_the_preconditioner_exact(pc_sweeps):
    """pc_sweeps < 0 on narrow subdomains picks the window form (causal_window >= 1):
    P^{-1} is (I - L)^{-1} to rounding, so right-preconditioned GMRES converges in
    one iteration; 0 or 1 sweeps converge to the same solution in more."""
    from paper_1503_02564_gb300 import swr
    wl = narrow()
    plan = gpu_plan(wl, precond=swr.SWR_PC_CAUSAL, restart=30, tol_abs=1e-11,
                    pc_sweeps=pc_sweeps)
    st = plan.get_stats()
    g, uT, info = _solve(plan, wl)
    plan.destroy()
    if pc_sweeps < 0:
        assert st["causal_window"] >= 1 and st["causal_sweeps"] == 0, st
        assert info["iterations"] == 1, info
    else:
        assert st["causal_window"] == 0 and st["causal_sweeps"] == pc_sweeps
        assert info["iterations"] > 1, info
    gs, uTm = _narrow_mono(wl)
    assert info["residual"] < 1e-11
    assert rel(uT, uTm) < TOL_SOLVE
    assert rel(g, gs) < TOL_SOLVE


_NARROW = {}


def _narrow_mono(wl):
    if "m" not in _NARROW:
        _NARROW["m"] = O.mono_interface(problem(wl))
    return _NARROW["m"]


def test_causal_window_precondition_is_near_identity():
    """(I - L) P^{-1} y = y to ~1e-13 with the window form (the same check with
    no same-step coupling resolved stays at the size of the dropped corners)."""
    from paper_1503_02564_gb300 import swr
    wl = narrow(nt=24)
    P = problem(wl)
    cols = O.build_columns(P)
    y = W.random_interface(wl.nblk, wl.nt, 12)
    yi = torch.tensor(y.ravel(), dtype=torch.complex128, device="cuda")
    errs = []
    for sw in (-1, 0):
        plan = gpu_plan(wl, precond=swr.SWR_PC_CAUSAL, pc_sweeps=sw)
        x = torch.zeros_like(yi)
        plan.apply_precond(yi, x)
        plan.destroy()
        errs.append(rel(O.apply_I_minus_L(P, cols, x.cpu().numpy()), y))
    assert errs[0] < 1e-12, errs
    assert errs[1] > 1e-8, errs


@pytest.mark.parametrize("case", ["config1_small", "ragged_tiny", "config2_N16_small", "narrow"])
def test_direct_causal_solver_reproduces_monodomain(case):
    """SWR_SOLVER_CAUSAL: (I - L) g = d by block forward substitution in time, no
    Krylov iteration; one or two substitutions reach the tolerance."""
    from paper_1503_02564_gb300 import swr
    wl = narrow() if case == "narrow" else CASES[case]()
    plan = gpu_plan(wl, solver=swr.SWR_SOLVER_CAUSAL, maxit=20, tol_abs=1e-11)
    g, uT, info = _solve(plan, wl)
    plan.destroy()
    assert info["status"] == swr.SWR_OK, info
    assert info["iterations"] <= 2, info
    gs, uTm = _narrow_mono(wl) if case == "narrow" else O.mono_interface(problem(wl))
    assert rel(uT, uTm) < TOL_SOLVE
    assert rel(g, gs) < TOL_SOLVE


def test_direct_causal_solver_rejects_time_dependent_potential():
    from paper_1503_02564_gb300 import swr
    wl = W.config4(nsub=4, nx=801, nt=20)
    with pytest.raises(swr.SWRError) as e:
        swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                 node_off=wl.off, vkind=swr.SWR_V_TIME, solver=swr.SWR_SOLVER_CAUSAL)
    assert e.value.status == swr.SWR_ERR_ARG


@pytest.mark.parametrize("precond", [0, 2])
@pytest.mark.parametrize("case", ["config1_small", "ragged_tiny", "config2_N16_small"])
def test_bicgstab_reproduces_monodomain(case, precond):
    """Right-preconditioned BiCGStab on (I - L) g = d (the alternative Krylov method of
    Section 6) reaches the monodomain solution."""
    from paper_1503_02564_gb300 import swr
    wl = CASES[case]()
    plan = gpu_plan(wl, solver=swr.SWR_SOLVER_BICGSTAB, maxit=2000, tol_abs=1e-12,
                    precond=swr.SWR_PC_CAUSAL if precond == 2 else swr.SWR_PC_NONE)
    g, uT, info = _solve(plan, wl)
    plan.destroy()
    assert info["status"] == swr.SWR_OK, info
    gs, uTm = O.mono_interface(problem(wl))
    assert rel(uT, uTm) < TOL_SOLVE
    assert rel(g, gs) < TOL_SOLVE


def test_bicgstab_time_dependent_matches_gmres():
    """V(t,x): matrix-free BiCGStab preconditioned by the mean-potential operator
    reaches the GMRES solution (and the monodomain one)."""
    from paper_1503_02564_gb300 import swr
    wl = W.config4(nsub=8, nx=2001, nt=40)
    out = []
    for solver in (swr.SWR_SOLVER_GMRES, swr.SWR_SOLVER_BICGSTAB):
        plan = gpu_plan(wl, solver=solver, restart=60, maxit=400, tol_abs=1e-11,
                        precond=swr.SWR_PC_MEAN_POTENTIAL)
        g, uT, info = _solve(plan, wl)
        plan.destroy()
        assert info["status"] == swr.SWR_OK, info
        out.append(uT)
    assert rel(out[1], out[0]) < TOL_SOLVE
    _, uTm = O.mono_interface(problem(wl))
    assert rel(out[1], uTm) < TOL_SOLVE


@pytest.mark.parametrize("nt,want_M", [(15, 0), (16, 32), (2048, 4096), (2049, 0)])
def test_toeplitz_fft_eligibility_edges(nt, want_M):
    """The library's own choice at the edges of the FFT apply (16 <= nt <= 2048, transform
    the power of two >= 2 nt - 1): the transform length it reports, and (I - L) x against
    the oracle on either side of each edge."""
    wl = W.config1(nx=121, nt=nt, nsub=3)
    plan = gpu_plan(wl)
    assert plan.get_stats()["toeplitz_fft_length"] == want_M
    P = problem(wl)
    cols = O.build_columns(P)
    x = W.random_interface(wl.nblk, wl.nt, 19)
    xi = torch.tensor(x.ravel(), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(xi)
    plan.apply_interface(xi, y)
    plan.destroy()
    assert rel(y.cpu().numpy(), O.apply_I_minus_L(P, cols, x)) < TOL_MARCH


@pytest.mark.parametrize("nt,superposed", [(4259, 1), (4260, 0)])
def test_s02_superposition_limit(nt, superposed):
    """S_0^2 ends: u(T) is superposed, and the interface mismatch found by the Toeplitz
    forward substitution with the trace, kernel and data in shared memory, up to
    nt = 4259; beyond it the final march takes over.  Both against the monodomain
    solution."""
    from paper_1503_02564_gb300 import swr
    wl = W.config1(nx=121, nt=nt, nsub=3)
    wl.tc = swr.SWR_TC_S02
    plan = gpu_plan(wl, tc=swr.SWR_TC_S02, precond=swr.SWR_PC_CAUSAL, restart=50, maxit=500,
                    tol_abs=1e-11)
    assert plan.get_stats()["superposed"] == superposed
    g, uT, info = _solve(plan, wl)
    plan.destroy()
    assert info["residual"] < 1e-11
    gs, uTm = O.mono_interface(problem(wl))
    assert rel(uT, uTm) < TOL_SOLVE
    assert rel(g, gs) < TOL_SOLVE
    assert info["interface_jump"] < 1e-9


@pytest.mark.parametrize("where", ["V", "u0"])
def test_device_status_reports_bad_inputs(where):
    """The kernels' status word, read by the host after the build: a NaN in the potential
    makes a pivot non-finite in the chunk factorisation (SWR_ERR_SINGULAR); a NaN in the
    initial state reaches the marched state (SWR_ERR_NONFINITE).  Neither traps; the plan
    is destroyed normally and a fresh plan on the same device then solves correctly."""
    from paper_1503_02564_gb300 import swr
    wl = CASES["config1_small"]()
    V = np.array(wl.V, dtype=np.float64)
    u0 = np.array(wl.u0, dtype=np.complex128)
    if where == "V":
        V[wl.nx // 3] = np.nan
        want = swr.SWR_ERR_SINGULAR
    else:
        u0[wl.nx // 2] = complex(np.nan, 0.0)
        want = swr.SWR_ERR_NONFINITE
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, p=wl.sigma, vkind=wl.vkind)
    with pytest.raises(swr.SWRError) as e:
        plan.build_interface(torch.tensor(V, device="cuda"), torch.tensor(u0, device="cuda"))
    assert e.value.status == want
    plan.destroy()
    plan = gpu_plan(wl)
    g, uT, info = _solve(plan, wl)
    plan.destroy()
    _, uTm = O.mono_interface(problem(wl))
    assert rel(uT, uTm) < TOL_SOLVE
