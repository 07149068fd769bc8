"""Seeded synthetic inputs for the SWR solver (grid, partition, potential, initial data).

This module only draws inputs; it holds none of the method's arithmetic.  The
test-suite feeds the same arrays to the CUDA library and to the CPU oracle.
Every generator uses ``numpy.random.default_rng(20150309 + config_id)``.

The paper's own experiments (Section 6) use analytic potentials and initial
data on (-21, 21) with dx = 1e-5; these workloads have the same kind of inputs
(smooth real potentials, Gaussian packets or a soliton, Neumann ends, equal
subdomains) at the sizes of the five benchmark workloads below.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20150309

V_STATIC, V_TIME, V_NONLINEAR = 0, 1, 2
TC_ROBIN, TC_S02 = 0, 1


@dataclass
class Workload:
    name: str
    a0: float
    b0: float
    nx: int
    dt: float
    nt: int
    off: np.ndarray            # int32, nsub+1 node offsets (subdomain j = nodes off[j]..off[j+1])
    V: np.ndarray              # float64: (nx,) static / V0, or (nt+1, nx) time dependent
    u0: np.ndarray             # complex128, (nx,)
    vkind: int = V_STATIC
    tc: int = TC_ROBIN
    sigma: complex = complex(math.sqrt(5.0) * np.exp(-1j * math.pi / 4))
    nl_coef: float = 1.0
    meta: dict = field(default_factory=dict)

    @property
    def x(self):
        return np.linspace(self.a0, self.b0, self.nx)

    @property
    def nsub(self):
        return len(self.off) - 1

    @property
    def nblk(self):
        return 2 * self.nsub - 2


def equal_offsets(nx: int, nsub: int) -> np.ndarray:
    """N subdomains of nx-1 elements in total: floor(E/N) elements each, the
    first E mod N subdomains one more (input recipe for 'N equal subdomains')."""
    E = nx - 1
    base, extra = divmod(E, nsub)
    sizes = np.full(nsub, base, dtype=np.int64)
    sizes[:extra] += 1
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)


def gaussian_packets(x, rng, count, centre_range, width_range, k_range):
    u = np.zeros_like(x, dtype=np.complex128)
    xc = rng.uniform(*centre_range, size=count)
    sg = rng.uniform(*width_range, size=count)
    kk = rng.uniform(*k_range, size=count)
    ph = rng.uniform(0.0, 2.0 * math.pi, size=count)
    for k in range(count):
        u += np.exp(-(x - xc[k]) ** 2 / (2.0 * sg[k] ** 2) + 1j * kk[k] * x + 1j * ph[k])
    return u


def config1(nx=1001, nt=200, nsub=4, dt=1e-3) -> Workload:
    """Plain SWR, V(x) = -x^2/4 on (-12, 12), u0 = exp(-x^2/2 + 5ix) with a
    +-1e-3 uniform phase noise per node, Robin p = sqrt(5) exp(-i pi/4)."""
    rng = np.random.default_rng(SEED_BASE + 1)
    a0, b0 = -12.0, 12.0
    x = np.linspace(a0, b0, nx)
    theta = rng.uniform(-1e-3, 1e-3, size=nx)
    u0 = np.exp(-x ** 2 / 2 + 5j * x) * np.exp(1j * theta)
    return Workload("config1_plain_N%d" % nsub, a0, b0, nx, dt, nt, equal_offsets(nx, nsub),
                    -x ** 2 / 4.0, u0)


def config2(nsub=16, nx=200001, nt=500, dt=1e-3) -> Workload:
    """Scaling case: (-50, 50), V = -5 sum of 8 seeded Gaussians (centres in
    (-40, 40), widths 0.5-3), u0 = sum of 4 seeded Gaussian packets
    (centres in (-30, 30), widths 0.5-2, wavenumbers in (-10, 10), random phase)."""
    rng = np.random.default_rng(SEED_BASE + 2)
    a0, b0 = -50.0, 50.0
    x = np.linspace(a0, b0, nx)
    c = rng.uniform(-40.0, 40.0, size=8)
    w = rng.uniform(0.5, 3.0, size=8)
    V = np.zeros(nx)
    for k in range(8):
        V -= 5.0 * np.exp(-(x - c[k]) ** 2 / (2.0 * w[k] ** 2))
    u0 = gaussian_packets(x, rng, 4, (-30.0, 30.0), (0.5, 2.0), (-10.0, 10.0))
    return Workload("config2_scaling_N%d" % nsub, a0, b0, nx, dt, nt,
                    equal_offsets(nx, nsub), V, u0)


def config3(count=128, nsub_range=(4, 64), size_range=(200, 2000), total_range=(2000, 40000),
            nt_range=(100, 400), h=1e-3, dt=1e-3):
    """Batch of independent SWR instances.  Each: N ~ U{nsub_range} subdomains
    whose sizes (nodes, shared ends included) are ~ U{size_range}, redrawn until
    the instance's node count lies in total_range; nt ~ U{nt_range}; grid step h
    on a domain centred at 0; V = sum of 4 Gaussian bumps (amplitudes U(-10, 10),
    widths U(0.5, 3), centres inside the domain); u0 one Gaussian packet (width
    U(0.5, 2), wavenumber U(-10, 10)).  Returns a list of Workloads."""
    rng = np.random.default_rng(SEED_BASE + 3)
    out = []
    for i in range(count):
        while True:
            N = int(rng.integers(nsub_range[0], nsub_range[1] + 1))
            elems = rng.integers(size_range[0] - 1, size_range[1], size=N)   # nodes - 1
            nx = int(elems.sum()) + 1
            if total_range[0] <= nx <= total_range[1]:
                break
        nt = int(rng.integers(nt_range[0], nt_range[1] + 1))
        half = 0.5 * (nx - 1) * h
        a0, b0 = -half, half
        x = a0 + h * np.arange(nx)
        amp = rng.uniform(-10.0, 10.0, size=4)
        w = rng.uniform(0.5, 3.0, size=4)
        c = rng.uniform(a0, b0, size=4)
        V = np.zeros(nx)
        for k in range(4):
            V += amp[k] * np.exp(-(x - c[k]) ** 2 / (2.0 * w[k] ** 2))
        u0 = gaussian_packets(x, rng, 1, (0.5 * a0, 0.5 * b0), (0.5, 2.0), (-10.0, 10.0))
        off = np.concatenate([[0], np.cumsum(elems)]).astype(np.int32)
        out.append(Workload("config3_batch_%d" % i, a0, b0, nx, dt, nt, off, V, u0))
    return out


def config4(nsub=64, nx=60001, nt=1000, dt=1e-3) -> Workload:
    """Time-dependent V(t,x) = -x^2/4 (1 + 0.5 sin 4t) - 10 exp(-(x - 5 sin t)^2)
    on (-30, 30); u0 = exp(-(x-x0)^2/2 + i k0 x), x0 ~ U(-10,10), k0 ~ U(-5,5).
    V is tabulated at t_n = n dt, n = 0..nt."""
    rng = np.random.default_rng(SEED_BASE + 4)
    a0, b0 = -30.0, 30.0
    x = np.linspace(a0, b0, nx)
    x0 = rng.uniform(-10.0, 10.0)
    k0 = rng.uniform(-5.0, 5.0)
    u0 = np.exp(-(x - x0) ** 2 / 2 + 1j * k0 * x)
    t = (np.arange(nt + 1) * dt)[:, None]
    V = -x[None, :] ** 2 / 4.0 * (1.0 + 0.5 * np.sin(4.0 * t)) \
        - 10.0 * np.exp(-(x[None, :] - 5.0 * np.sin(t)) ** 2)
    return Workload("config4_timedep_N%d" % nsub, a0, b0, nx, dt, nt,
                    equal_offsets(nx, nsub), np.ascontiguousarray(V), u0, vkind=V_TIME)


def config5(nsub=32, nx=20001, nt=1000, dt=5e-4) -> Workload:
    """Nonlinear V = |u|^2 + V0(x) on (-20, 20), V0 = -sum of 6 seeded Gaussian
    wells (depths 2-10, centres in (-15, 15), widths 0.5-2), u0 = sech(x) e^{2ix}."""
    rng = np.random.default_rng(SEED_BASE + 5)
    a0, b0 = -20.0, 20.0
    x = np.linspace(a0, b0, nx)
    dep = rng.uniform(2.0, 10.0, size=6)
    c = rng.uniform(-15.0, 15.0, size=6)
    w = rng.uniform(0.5, 2.0, size=6)
    V0 = np.zeros(nx)
    for k in range(6):
        V0 -= dep[k] * np.exp(-(x - c[k]) ** 2 / (2.0 * w[k] ** 2))
    u0 = (1.0 / np.cosh(x)) * np.exp(2j * x)
    wl = Workload("config5_nonlinear_N%d" % nsub, a0, b0, nx, dt, nt,
                  equal_offsets(nx, nsub), V0, u0.astype(np.complex128), vkind=V_NONLINEAR)
    wl.meta["V0_params"] = (dep, c, w)
    return wl


def config5_target_potential(wl: Workload, seed: int = 9) -> np.ndarray:
    """The perturbed potential whose final state is the misfit target of the nonlinear
    workload: V0 with every well depth d_k multiplied by (1 + 0.05 xi_k), xi ~ N(0, 1)
    seeded.  (The target state itself is u(T) of the nonlinear problem with this
    potential; whoever needs it marches it.)"""
    rng = np.random.default_rng(SEED_BASE + 300 + seed)
    dep, c, w = wl.meta["V0_params"]
    dep = dep * (1.0 + 0.05 * rng.standard_normal(len(dep)))
    V = np.zeros(wl.nx)
    for k in range(len(dep)):
        V -= dep[k] * np.exp(-(wl.x - c[k]) ** 2 / (2.0 * w[k] ** 2))
    return V


def tc_comparison(nsub=2, nx=4200001, nt=500, dt=1e-3) -> Workload:
    """The setting of the paper's comparison of transmission conditions (Section 6):
    (a0, b0) = (-21, 21), dx = 1e-5 (4200001 nodes), T = 0.5 with dt = 1e-3,
    V(x) = -x^2, u0 = exp(-(x+10)^2 + 20 i (x+10)), N equal subdomains."""
    a0, b0 = -21.0, 21.0
    x = np.linspace(a0, b0, nx)
    V = -x * x
    u0 = np.exp(-(x + 10.0) ** 2 + 20j * (x + 10.0))
    return Workload("tc_comparison_N%d" % nsub, a0, b0, nx, dt, nt, equal_offsets(nx, nsub),
                    V, u0.astype(np.complex128))


def random_interface(nblk: int, nt: int, seed: int = 7) -> np.ndarray:
    """A seeded random interface vector (the paper's 'random g^0', Section 6)."""
    rng = np.random.default_rng(SEED_BASE + 100 + seed)
    return (rng.standard_normal((nblk, nt)) + 1j * rng.standard_normal((nblk, nt)))


def misfit_target(wl: Workload, seed: int = 9) -> np.ndarray:
    """A seeded final-time target for the misfit ||u(T) - u_target||_M^2: the
    initial data with a phase shift plus 5 % complex noise."""
    rng = np.random.default_rng(SEED_BASE + 200 + seed)
    noise = rng.standard_normal(wl.nx) + 1j * rng.standard_normal(wl.nx)
    return wl.u0 * np.exp(0.4j) + 0.05 * noise
