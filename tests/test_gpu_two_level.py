"""GPU parity of the two-level separator solve (k_march_tl): systems spread over a
thread-block cluster solve their separators in warp blocks of 32 (super-chunks by
warp-shuffle PCR, a reduced system over the super-separators solved by one warp),
one cluster barrier per time step.  Against the oracle per march output (d, the
Toeplitz first columns, R g: 1e-10) and against the cluster-wide PCR of the same
launch shape (tuning.two_level = -1) to rounding, on ragged partitions whose
separator counts end on every residue class that matters (P_j = 0, 1, 31 and other
values mod 32), and with 4-node chunks whose > 993 separators keep the cluster-wide
PCR."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1503_02564_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_MARCH = 1e-10


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


def ragged(L):
    """Five subdomains whose separator counts P_j = ceil((n_j - 1) / (L + 1)) are
    32 m, 32 m + 1, 32 m + 31, a middle value and a short one (n_j nodes)."""
    per = L + 1
    pj = [320, 321, 351, 300, 150] if L >= 8 else [1000, 97, 127, 100, 50]
    sizes = [p * per + 1 for p in pj]            # n_j - 1 = P_j (L + 1): P_j exactly
    sizes[3] -= 4                                # ... and one with shorter chunks
    nx = sum(sizes) - (len(sizes) - 1)
    wl = W.config2(nsub=5, nx=nx, nt=14)
    off = [0]
    for n in sizes:
        off.append(off[-1] + n - 1)
    wl.off = np.array(off, dtype=np.int32)
    # initial data of size one at every interface (the seeded packets sit in (-30, 30),
    # and at an interface outside them d would be an exponentially small tail)
    x = wl.x
    wl.u0 = np.exp(2j * x) * (1.0 + 0.3 * np.sin(0.7 * x))
    return wl


def build(wl, tc, chunk, two_level):
    from paper_1503_02564_gb300 import swr
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, p=wl.sigma, tc=tc,
                    tuning={"chunk_L": chunk, "autotune": -1, "two_level": two_level})
    plan.build_interface(torch.tensor(wl.V, dtype=torch.float64, device="cuda"),
                         torch.tensor(wl.u0, dtype=torch.complex128, device="cuda"))
    d = torch.zeros(plan.n_interface, dtype=torch.complex128, device="cuda")
    cols = torch.zeros(plan.n_cols, dtype=torch.complex128, device="cuda")
    plan.get_interface(d, cols)
    g = W.random_interface(wl.nblk, wl.nt, 51)
    gi = torch.tensor(g.ravel(), dtype=torch.complex128, device="cuda")
    go = torch.zeros_like(gi)
    plan.apply_R(gi, go)
    st = plan.get_stats()
    plan.destroy()
    return d.cpu().numpy(), cols.cpu().numpy(), go.cpu().numpy(), g, st


@pytest.mark.parametrize("tc", [O.TC_ROBIN, O.TC_S02, O.TC_S14])
@pytest.mark.parametrize("chunk", [8, 12, 16, 4])
def test_two_level_march_matches_oracle_and_cluster_pcr(chunk, tc):
    wl = ragged(chunk)
    d1, c1, r1, g, st1 = build(wl, tc, chunk, 0)
    d0, c0, r0, _, st0 = build(wl, tc, chunk, -1)
    # 4-node chunks: more than 993 separators in the longest subdomain, cluster-wide PCR
    assert (st1["two_level_launches"] > 0) == (chunk != 4), st1
    assert st0["two_level_launches"] == 0
    P = O.Problem(wl.a0, wl.b0, wl.nx, wl.dt, wl.nt, wl.off.astype(np.int64), wl.u0, wl.V,
                  tc=tc, sigma=wl.sigma)
    assert rel(d1, O.build_d(P)) < TOL_MARCH
    assert rel(c1, O.build_columns(P)) < TOL_MARCH
    assert rel(r1, O.apply_R(P, g)) < TOL_MARCH
    assert rel(d1, d0) < 1e-12 and rel(c1, c0) < 1e-12 and rel(r1, r0) < 1e-12


@pytest.mark.parametrize("tc", [O.TC_S02, O.TC_S14])
@pytest.mark.parametrize("chunk", [4, 8])
def test_two_level_short_systems_with_both_ends_in_one_warp(chunk, tc):
    """Systems of at most 32 separators (61-node subdomains: 13 or 7 separators) alone in
    their CTAs, with history terms at both ends: both ends sit in warp 0, which forms
    both ends' history sums every step.  Against the oracle's d, columns and R g."""
    wl = W.config2(nsub=6, nx=6 * 60 + 1, nt=20)
    x = wl.x
    wl.u0 = np.exp(2j * x) * (1.0 + 0.3 * np.sin(0.7 * x))
    d1, c1, r1, g, st1 = build(wl, tc, chunk, 0)
    assert st1["two_level_launches"] > 0, st1
    P = O.Problem(wl.a0, wl.b0, wl.nx, wl.dt, wl.nt, wl.off.astype(np.int64), wl.u0, wl.V,
                  tc=tc, sigma=wl.sigma)
    assert rel(d1, O.build_d(P)) < TOL_MARCH
    assert rel(c1, O.build_columns(P)) < TOL_MARCH
    assert rel(r1, O.apply_R(P, g)) < TOL_MARCH


@pytest.mark.parametrize("tc", [O.TC_ROBIN, O.TC_S02])
def test_two_level_one_system_per_cta(tc):
    """About a hundred systems (the build of 34 subdomains): the modelled shape puts one
    system in each CTA (no cluster), and the two-level solve runs there too (its
    cluster is the CTA itself)."""
    wl = W.config2(nsub=34, nx=34 * 700 + 1, nt=14)
    x = wl.x
    wl.u0 = np.exp(2j * x) * (1.0 + 0.3 * np.sin(0.7 * x))
    d1, c1, r1, g, st1 = build(wl, tc, 12, 0)
    d0, c0, r0, _, st0 = build(wl, tc, 12, -1)
    assert st1["two_level_launches"] > 0 and st0["two_level_launches"] == 0
    P = O.Problem(wl.a0, wl.b0, wl.nx, wl.dt, wl.nt, wl.off.astype(np.int64), wl.u0, wl.V,
                  tc=tc, sigma=wl.sigma)
    assert rel(d1, O.build_d(P)) < TOL_MARCH
    assert rel(c1, O.build_columns(P)) < TOL_MARCH
    assert rel(r1, O.apply_R(P, g)) < TOL_MARCH
    assert rel(d1, d0) < 1e-12 and rel(c1, c0) < 1e-12 and rel(r1, r0) < 1e-12


def test_two_level_solve_reproduces_monodomain():
    """A full solve (causal preconditioner, u(T) by superposition) on the ragged
    partition with the two-level marches."""
    from paper_1503_02564_gb300 import swr
    wl = ragged(12)
    plan = swr.Plan(nx=wl.nx, a0=wl.a0, b0=wl.b0, nt=wl.nt, dt=wl.dt, nsub=wl.nsub,
                    node_off=wl.off, p=wl.sigma, precond=swr.SWR_PC_CAUSAL,
                    tuning={"chunk_L": 12, "autotune": -1})
    plan.build_interface(torch.tensor(wl.V, dtype=torch.float64, device="cuda"),
                         torch.tensor(wl.u0, dtype=torch.complex128, device="cuda"))
    g = torch.zeros(plan.n_interface, dtype=torch.complex128, device="cuda")
    uT = torch.zeros(wl.nx, dtype=torch.complex128, device="cuda")
    info = plan.solve(g, False, uT)
    assert plan.get_stats()["two_level_launches"] > 0
    plan.destroy()
    P = O.Problem(wl.a0, wl.b0, wl.nx, wl.dt, wl.nt, wl.off.astype(np.int64), wl.u0, wl.V,
                  sigma=wl.sigma)
    gs, uTm = O.mono_interface(P)
    assert info["residual"] < 1e-10
    assert rel(uT.cpu().numpy(), uTm) < 1e-9
    assert rel(g.cpu().numpy(), gs) < 1e-9
