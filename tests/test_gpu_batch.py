"""GPU parity for batched plans (swr_plan_batch): independent instances with
uneven partitions and step counts in one plan, against the oracle instance by
instance and against one plan per instance."""
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
                     vkind=wl.vkind, tc=wl.tc, sigma=wl.sigma)


def small_batch(count=5, tc=W.TC_ROBIN, **kw):
    args = dict(count=count, nsub_range=(3, 6), size_range=(40, 120), total_range=(200, 600),
                nt_range=(10, 30))
    args.update(kw)
    wls = W.config3(**args)
    for w in wls:
        w.tc = tc
    return wls


def batch_plan(wls, autotune=True, **kw):
    """autotune=False: the modelled launch shapes, which pack the uneven systems
    of a batch by size (ragged packing) instead of padding them."""
    import os
    from paper_1503_02564_gb300 import swr
    insts = [dict(nx=w.nx, a0=w.a0, b0=w.b0, nt=w.nt, nsub=w.nsub, node_off=w.off) for w in wls]
    kw.setdefault("p", wls[0].sigma)
    kw.setdefault("tc", wls[0].tc)
    plan = swr.BatchPlan(insts, dt=wls[0].dt, tuning=None if autotune else {"autotune": -1},
                         **kw)
    V = torch.tensor(np.concatenate([w.V for w in wls]), dtype=torch.float64, device="cuda")
    u0 = torch.tensor(np.concatenate([w.u0 for w in wls]), dtype=torch.complex128, device="cuda")
    plan.build_interface(V, u0)
    return plan


def split(arr, lengths):
    out, k = [], 0
    for n in lengths:
        out.append(arr[k:k + n])
        k += n
    return out


@pytest.mark.parametrize("autotune", [True, False])
@pytest.mark.parametrize("tc", [W.TC_ROBIN, W.TC_S02])
def test_batch_build_matches_oracle_per_instance(tc, autotune):
    wls = small_batch(tc=tc)
    plan = batch_plan(wls, autotune)
    d = torch.zeros(plan.n_interface, dtype=torch.complex128, device="cuda")
    cols = torch.zeros(plan.n_cols, dtype=torch.complex128, device="cuda")
    plan.get_interface(d, cols)
    plan.destroy()
    ds = split(d.cpu().numpy(), [w.nblk * w.nt for w in wls])
    cs = split(cols.cpu().numpy(), [4 * w.nsub * w.nt for w in wls])
    for w, di, ci in zip(wls, ds, cs):
        P = problem(w)
        assert rel(di, O.build_d(P)) < TOL_MARCH
        assert rel(ci, O.build_columns(P)) < TOL_MARCH


@pytest.mark.parametrize("autotune", [True, False])
def test_batch_apply_R_matches_oracle_per_instance(autotune):
    wls = small_batch(count=6)
    plan = batch_plan(wls, autotune)
    gs = [W.random_interface(w.nblk, w.nt, 50 + i) for i, w in enumerate(wls)]
    gi = torch.tensor(np.concatenate([g.ravel() for g in gs]), dtype=torch.complex128,
                      device="cuda")
    go = torch.zeros_like(gi)
    plan.apply_R(gi, go)
    plan.destroy()
    for w, g, o in zip(wls, gs, split(go.cpu().numpy(), [w.nblk * w.nt for w in wls])):
        assert rel(o, O.apply_R(problem(w), g)) < TOL_MARCH


@pytest.mark.parametrize("autotune", [True, False])
@pytest.mark.parametrize("tc", [W.TC_ROBIN, W.TC_S02])
def test_batch_solve_reproduces_each_monodomain_solution(tc, autotune):
    from paper_1503_02564_gb300 import swr
    wls = small_batch(tc=tc)
    plan = batch_plan(wls, autotune, precond=swr.SWR_PC_CAUSAL, restart=100, tol_abs=1e-12)
    g = torch.zeros(plan.n_interface, dtype=torch.complex128, device="cuda")
    uT = torch.zeros(plan.nx, dtype=torch.complex128, device="cuda")
    info = plan.solve(g, False, uT)
    plan.destroy()
    assert info["residual"] < 1e-12
    gsp = split(g.cpu().numpy(), [w.nblk * w.nt for w in wls])
    usp = split(uT.cpu().numpy(), [w.nx for w in wls])
    for w, gi, ui in zip(wls, gsp, usp):
        gm, um = O.mono_interface(problem(w))
        assert rel(ui, um) < TOL_SOLVE
        assert rel(gi, gm) < TOL_SOLVE


def test_batch_across_several_cooperative_launches_matches_single_plans():
    """Enough instances that the causal substitution needs several cooperative
    launches; each instance agrees with its own one-instance plan.  (Subdomains
    are kept much wider than sqrt(dt): the substitution drops the same-step
    coupling of neighbouring interfaces, which is O(1) for subdomains of a few
    dozen nodes and then makes P^{-1} unstable.)"""
    from paper_1503_02564_gb300 import swr
    wls = W.config3(count=48, nsub_range=(20, 40), size_range=(200, 300),
                    total_range=(2000, 12000), nt_range=(10, 40))
    assert sum(w.nsub - 1 for w in wls) > 760
    plan = batch_plan(wls, precond=swr.SWR_PC_CAUSAL, restart=60, tol_abs=1e-12)
    uT = torch.zeros(plan.nx, dtype=torch.complex128, device="cuda")
    info = plan.solve(None, False, uT)
    plan.destroy()
    assert info["residual"] < 1e-12
    usp = split(uT.cpu().numpy(), [w.nx for w in wls])
    for w, ub in list(zip(wls, usp))[::7]:
        p1 = swr.Plan(nx=w.nx, a0=w.a0, b0=w.b0, nt=w.nt, dt=w.dt, nsub=w.nsub, node_off=w.off,
                      p=w.sigma, precond=swr.SWR_PC_CAUSAL, restart=60, tol_abs=1e-13)
        p1.build_interface(torch.tensor(w.V, dtype=torch.float64, device="cuda"),
                           torch.tensor(w.u0, dtype=torch.complex128, device="cuda"))
        u1 = torch.zeros(w.nx, dtype=torch.complex128, device="cuda")
        p1.solve(None, False, u1)
        p1.destroy()
        assert rel(ub, u1.cpu().numpy()) < TOL_SOLVE


def test_batch_rejects_mismatched_shared_fields():
    from paper_1503_02564_gb300 import swr
    wls = small_batch(count=2)
    insts = [dict(nx=w.nx, a0=w.a0, b0=w.b0, nt=w.nt, nsub=w.nsub, node_off=w.off) for w in wls]
    insts[1]["b0"] = insts[1]["b0"] * 1.5          # a different grid step
    with pytest.raises(swr.SWRError) as e:
        swr.BatchPlan(insts, dt=1e-3, p=wls[0].sigma)
    assert e.value.status == swr.SWR_ERR_ARG
