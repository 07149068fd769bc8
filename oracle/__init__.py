"""Plain FP64 CPU oracle for the SWR hot path of Besse & Xing (arXiv 1503.02564).

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  Nothing here is imported
by the CUDA library or its Python binding, and nothing here imports them.

The time loops live in ``swr_oracle.c`` (built by ``oracle/build.py``); this
module writes the paper's algorithms out step by step on top of them with NumPy:

* subdomain operator R (Eq. interfacepbR) with the flux update of
  Eq. TransmisionCond / TransmissionCond_disc;
* the interface vector g (Section 3), d = R 0 (Section 4.1) and the first
  columns of the blocks X^{j,p} (Section 4.1, Props. 3-4);
* (I - L) g from the Toeplitz first columns (the block structure of Props. 3-4);
* the classical fixed point (Algorithm 1), GMRES(m) (Saad, "Iterative methods
  for sparse linear systems", Alg. 6.9 with modified Gram-Schmidt and Givens
  rotations; the paper cites it for Algorithms 2-3), the preconditioned
  iterations of Section 5 (Eqs. chp2_algopd_L, chp2_algopd_Lpf,
  chp2_algopd_NL) with P = I - L_0 applied by an inner GMRES from a zero start
  (Eq. Pxg);
* the interface vector implied by the monodomain solution, which converged SWR
  must reproduce;
* brute-force dense L on tiny grids.

Readings of points the paper leaves open:
  Robin S-bar v = sigma v with complex sigma; generalised mass by exact P1
  quadrature; equal partitions give the first E mod N subdomains one extra
  element; stopping on the absolute Euclidean norm of the true residual; the
  nonlinear outer iteration read as g <- g - P^{-1}(g - R_nl g).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .build import build_oracle

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = build_oracle()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.or_march.restype = ctypes.c_int
        L.or_march.argtypes = [
            ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
            dp, ctypes.c_long, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp,
            ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, dp, ip, ctypes.c_int, ip, dp, dp, dp]
        L.or_thomas.restype = ctypes.c_int
        L.or_thomas.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp]
        L.or_p1_matrices.restype = None
        L.or_p1_matrices.argtypes = [ctypes.c_int, ctypes.c_double, dp] + [dp] * 6
        L.or_causal_conv.restype = None
        L.or_causal_conv.argtypes = [ctypes.c_int, dp, dp, dp]
        vp = ctypes.c_void_p
        L.or_march_ext.restype = ctypes.c_int
        L.or_march_ext.argtypes = [
            ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, ctypes.c_int,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp,
            ctypes.c_int, ctypes.c_int, dp, dp, dp, vp, vp, vp, dp, dp]
        _LIB = L
    return _LIB


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


# --------------------------------------------------------------------------
# Elementary pieces
# --------------------------------------------------------------------------
def p1_matrices(n, h, W=None):
    """P1 mass, stiffness and generalised-mass matrices (Eq. AvML) as
    (diag, offdiag) pairs: returns md, mo, sd, so, wd, wo."""
    out = [np.zeros(n), np.zeros(max(n - 1, 1)), np.zeros(n), np.zeros(max(n - 1, 1)),
           np.zeros(n), np.zeros(max(n - 1, 1))]
    Wc = None if W is None else np.ascontiguousarray(W, dtype=np.float64)
    lib().or_p1_matrices(n, h, _p(Wc), *[_p(o) for o in out])
    return out[0], out[1][: n - 1], out[2], out[3][: n - 1], out[4], out[5][: n - 1]


def thomas(lo, dg, up, rhs):
    """Textbook Thomas solve (no pivoting) of a complex tridiagonal system."""
    n = len(dg)
    lo = np.ascontiguousarray(lo, dtype=np.complex128)
    up = np.ascontiguousarray(up, dtype=np.complex128)
    dg = np.ascontiguousarray(dg, dtype=np.complex128)
    x = np.array(rhs, dtype=np.complex128)
    work = np.zeros(n, dtype=np.complex128)
    st = lib().or_thomas(n, _p(lo), _p(dg), _p(up), _p(x), _p(work))
    if st != 0:
        raise ZeroDivisionError(f"zero pivot at row {-st - 1}")
    return x


def alpha_coefficients(n):
    """alpha_0..alpha_n of Section 2.2: (1, 1, 1/2, 1/2, 3/8, 3/8, 15/48, ...):
    alpha_{2k} = alpha_{2k+1} = (1*3*...*(2k-1)) / (2*4*...*(2k))."""
    a = np.zeros(n + 1)
    val = 1.0
    for s in range(n + 1):
        k = s // 2
        if s % 2 == 0 and k > 0:
            val *= (2 * k - 1) / (2 * k)
        a[s] = val
    return a


def beta_coefficients(n):
    """beta_s = (-1)^s alpha_s (Section 2.2)."""
    a = alpha_coefficients(n)
    return a * np.where(np.arange(n + 1) % 2 == 0, 1.0, -1.0)


def gamma_coefficients(n):
    """gamma_0..gamma_n of Section 2.2: (1, 2, 2, 2, ...)."""
    g = np.full(n + 1, 2.0)
    g[0] = 1.0
    return g


def s02_c2(dt):
    """c_2 = e^{-i pi/4} sqrt(2/dt) (S_0^2, Section 2.2)."""
    return np.exp(-1j * math.pi / 4) * math.sqrt(2.0 / dt)


def partition_equal(nx, nsub):
    """Node offsets of N equal non-overlapping subdomains: E = nx-1 elements,
    floor(E/N) each and one more for the first E mod N (reading of 'equal' when
    N does not divide E).  Subdomain j holds nodes off[j]..off[j+1] inclusive."""
    E = nx - 1
    base, extra = divmod(E, nsub)
    off = [0]
    for j in range(nsub):
        off.append(off[-1] + base + (1 if j < extra else 0))
    return np.array(off, dtype=np.int64)


# --------------------------------------------------------------------------
# Problem description
# --------------------------------------------------------------------------
TC_ROBIN, TC_S02, TC_S03, TC_S04, TC_S12, TC_S14 = 0, 1, 2, 3, 4, 5
TC_NAMES = {TC_ROBIN: "Robin", TC_S02: "S_0^2", TC_S03: "S_0^3", TC_S04: "S_0^4",
            TC_S12: "S_1^2", TC_S14: "S_1^4"}
V_STATIC, V_TIME, V_NONLINEAR = 0, 1, 2


@dataclass
class Problem:
    """One SWR problem: i u_t + u_xx + V u = 0 on (a0, b0), Neumann ends (Eq. Schequ)."""
    a0: float
    b0: float
    nx: int
    dt: float
    nt: int
    off: np.ndarray              # nsub+1 node offsets
    u0: np.ndarray               # complex, nx
    V: np.ndarray                # static: (nx,); time: (nt+1, nx); nonlinear: V0 (nx,)
    vkind: int = V_STATIC
    tc: int = TC_ROBIN
    sigma: complex = 0.0         # Robin: S-bar v = sigma v
    nl_coef: float = 1.0         # nonlinear: f(v) = nl_coef |v|^2
    nl_maxit: int = 50
    nl_tol: float = 1e-13

    @property
    def h(self):
        return (self.b0 - self.a0) / (self.nx - 1)

    @property
    def nsub(self):
        return len(self.off) - 1

    @property
    def nblk(self):
        return 2 * self.nsub - 2

    def beta(self):
        return beta_coefficients(self.nt)

    def c2(self):
        return s02_c2(self.dt)

    def sigma0(self):
        return self.sigma if self.tc == TC_ROBIN else self.c2() * 1.0

    def local_V(self, j, V=None):
        V = self.V if V is None else V
        a, b = int(self.off[j]), int(self.off[j + 1])
        if V.ndim == 1:
            return np.ascontiguousarray(V[a:b + 1])
        return np.ascontiguousarray(V[:, a:b + 1])


def blk_r(j):
    """Block of g holding r_j (flux at the right end of subdomain j, 0-based)."""
    return 2 * j


def blk_l(j):
    """Block of g holding l_j (flux at the left end of subdomain j, 0-based)."""
    return 2 * j - 1


# --------------------------------------------------------------------------
# Marches
# --------------------------------------------------------------------------
@dataclass
class MarchResult:
    va: np.ndarray       # v_t at the left end, t = 0..nt
    vb: np.ndarray       # v_t at the right end
    uT: np.ndarray
    nl_iters: np.ndarray
    vsel: Optional[np.ndarray] = None


def march(n, h, dt, nt, V, u0, *, vkind=V_STATIC, tc=TC_ROBIN, sigma=0.0, tc_left=False,
          tc_right=False, l=None, r=None, nl_coef=1.0, nl_maxit=50, nl_tol=1e-13,
          sel=None, wl=None, wr=None) -> MarchResult:
    """One Crank-Nicolson march on n nodes (Eq. AvML / AvMNL); see or_march in
    swr_oracle.c for the exact statement.  tc >= TC_S03: the ends' S-bar are given
    by their weight matrices wl, wr ((nt+1) x (nt+1), S-bar v_n = sum_s w[n, s] v_s)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    vstride = V.shape[1] if V.ndim == 2 else 0
    u0 = np.ascontiguousarray(u0, dtype=np.complex128)
    assert u0.shape == (n,)
    lc = None if l is None else np.ascontiguousarray(l, dtype=np.complex128)
    rc = None if r is None else np.ascontiguousarray(r, dtype=np.complex128)
    beta = beta_coefficients(nt)
    c2 = s02_c2(dt)
    va = np.zeros(nt + 1, np.complex128)
    vb = np.zeros(nt + 1, np.complex128)
    uT = np.zeros(n, np.complex128)
    its = np.zeros(nt, np.int32)
    if sel is not None:
        sel = np.ascontiguousarray(sel, dtype=np.int32)
        vsel = np.zeros((nt + 1, len(sel)), np.complex128)
    else:
        vsel = None
    sig = complex(sigma)
    ctc = tc if tc <= TC_S02 else 2          # the C march: 0 Robin, 1 S_0^2, 2 weights
    wlc = None if (wl is None or not tc_left) else np.ascontiguousarray(wl, np.complex128)
    wrc = None if (wr is None or not tc_right) else np.ascontiguousarray(wr, np.complex128)
    if ctc == 2 and ((tc_left and wlc is None) or (tc_right and wrc is None)):
        raise ValueError("weights needed at every end with a transmission condition")
    st = lib().or_march(n, h, dt, nt, vkind, _p(V), vstride, nl_coef, nl_maxit, nl_tol, ctc,
                        sig.real, sig.imag, c2.real, c2.imag, _p(beta), int(tc_left),
                        int(tc_right), _p(u0), _p(lc), _p(rc), _p(va), _p(vb), _p(uT),
                        _ip(its), 0 if sel is None else len(sel), _ip(sel), _p(vsel),
                        _p(wlc), _p(wrc))
    if st == -1000000:
        raise RuntimeError("nonlinear fixed point did not converge")
    if st != 0:
        raise ZeroDivisionError(f"zero pivot at row {-st - 1}")
    return MarchResult(va, vb, uT, its, vsel)


def march_ext(n, h, dt, nt, V, u0, *, tc=TC_ROBIN, sigma=0.0, tc_left=False,
              tc_right=False, l=None, r=None, wl=None, wr=None) -> MarchResult:
    """The static-V march of ``march`` carried in extended precision (C long double:
    64-bit significand on x86-64, binary128 on AArch64); see or_march_ext.  The
    inputs are the binary64 values that define the problem; the end traces va, vb
    and u(T) come back as np.clongdouble.  Used to tell rounding from error where a
    binary64 result cancels."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    assert V.ndim == 1
    u0 = np.ascontiguousarray(u0, dtype=np.complex128)
    lc = None if l is None else np.ascontiguousarray(l, dtype=np.complex128)
    rc = None if r is None else np.ascontiguousarray(r, dtype=np.complex128)
    beta = beta_coefficients(nt)
    c2 = s02_c2(dt)
    va = np.zeros(nt + 1, np.clongdouble)
    vb = np.zeros(nt + 1, np.clongdouble)
    uT = np.zeros(n, np.clongdouble)
    sig = complex(sigma)
    ctc = tc if tc <= TC_S02 else 2
    wlc = None if (wl is None or not tc_left) else np.ascontiguousarray(wl, np.complex128)
    wrc = None if (wr is None or not tc_right) else np.ascontiguousarray(wr, np.complex128)
    if ctc == 2 and ((tc_left and wlc is None) or (tc_right and wrc is None)):
        raise ValueError("weights needed at every end with a transmission condition")
    st = lib().or_march_ext(n, h, dt, nt, _p(V), ctc, sig.real, sig.imag, c2.real, c2.imag,
                            _p(beta), int(tc_left), int(tc_right), _p(u0), _p(lc), _p(rc),
                            va.ctypes.data, vb.ctypes.data, uT.ctypes.data, _p(wlc), _p(wrc))
    if st != 0:
        raise ZeroDivisionError(f"zero pivot at row {-st - 1}")
    return MarchResult(va, vb, uT, np.zeros(nt, np.int32))


def tc_weights(P: Problem, j, side, V=None):
    """Weights w[n, s], 0 <= s <= n <= nt, of the discrete transmission operator at one
    end of subdomain j (side 0: a_j, side 1: b_j), S-bar v_n = sum_s w[n, s] v_s, written
    out from the discrete operators of Section 2.2 for V = V(x):
      S_0^2: c2 beta_{n-s},  c2 = e^{-i pi/4} sqrt(2/dt);
      S_0^3: S_0^2 - e^{i pi/4} sqrt(dt/2) (W_n / 2) alpha_{n-s};
      S_0^4: S_0^3 - i (d_n W_n / 4) (dt/2) gamma_{n-s};
      S_1^2: c2 e^{i Wc_n} beta_{n-s} e^{-i Wc_s};
      S_1^4: S_1^2 - i sgn(d_n W_n) (sqrt|d_n W_n| / 2) e^{i Wc_n} (dt/2) gamma_{n-s}
                     (sqrt|d_n W_s| / 2) e^{-i Wc_s}.
    Readings: W_n is the potential at the end node (W_n = (V_n + V_{n-1})/2 = V there);
    d_n W its outward normal derivative at the end, the central difference on the whole
    grid (the end is an interior node of the whole grid), sign + at b_j and - at a_j;
    Wc_n = (Vc_n + Vc_{n-1})/2 with Vc_n = int_0^{t_n} V ds = t_n V, and Wc_0 = 0 (Vc_{-1}
    is not defined); sgn(0) = 0."""
    if P.vkind != V_STATIC:
        raise NotImplementedError("S_0^3, S_0^4, S_1^2, S_1^4: V = V(x) only")
    V = P.V if V is None else V
    nt, dt, h = P.nt, P.dt, P.h
    g = int(P.off[j + side])
    Wb = float(V[g])
    dn = (float(V[g + 1]) - float(V[g - 1])) / (2.0 * h) * (1.0 if side == 1 else -1.0)
    al, be, ga = alpha_coefficients(nt), beta_coefficients(nt), gamma_coefficients(nt)
    c2 = s02_c2(dt)
    c3 = np.exp(1j * math.pi / 4) * math.sqrt(dt / 2.0)
    Wc = np.array([0.0] + [(n - 0.5) * dt * Wb for n in range(1, nt + 1)])
    w = np.zeros((nt + 1, nt + 1), np.complex128)
    for n in range(nt + 1):
        for s_ in range(n + 1):
            m = n - s_
            if P.tc in (TC_S03, TC_S04):
                x = c2 * be[m] - c3 * (Wb / 2.0) * al[m]
                if P.tc == TC_S04:
                    x += -1j * (dn / 4.0) * (dt / 2.0) * ga[m]
            elif P.tc in (TC_S12, TC_S14):
                ph = np.exp(1j * Wc[n]) * np.exp(-1j * Wc[s_])
                x = c2 * ph * be[m]
                if P.tc == TC_S14:
                    r = math.sqrt(abs(dn)) / 2.0
                    x += -1j * np.sign(dn) * r * ph * (dt / 2.0) * ga[m] * r
            else:
                raise ValueError("tc_weights: S_0^3, S_0^4, S_1^2 or S_1^4")
            w[n, s_] = x
    return w


def sub_march(P: Problem, j, u0_local, l=None, r=None, V=None) -> MarchResult:
    """March of subdomain j (0-based) with fluxes l, r (Eq. AvML with
    Eq. TransmissionCondlocal); outer ends keep the Neumann condition."""
    a, b = int(P.off[j]), int(P.off[j + 1])
    wl = wr = None
    if P.tc >= TC_S03:
        wl = tc_weights(P, j, 0, V) if j > 0 else None
        wr = tc_weights(P, j, 1, V) if j < P.nsub - 1 else None
    return march(b - a + 1, P.h, P.dt, P.nt, P.local_V(j, V), u0_local, vkind=P.vkind,
                 tc=P.tc, sigma=P.sigma, tc_left=(j > 0), tc_right=(j < P.nsub - 1),
                 l=l, r=r, nl_coef=P.nl_coef, nl_maxit=P.nl_maxit, nl_tol=P.nl_tol,
                 wl=wl, wr=wr)


def s_tilde(P: Problem, vtrace, j=None, side=None, V=None):
    """Fully discrete S-tilde applied to a boundary trace v_0..v_nt; returns
    entries for n = 1..nt (Eq. TransmissionCond_disc).  Robin: sigma v_n.
    S_0^2: c_2 sum_{s=0}^{n} beta_{n-s} v_s.  S_0^3, S_0^4, S_1^2, S_1^4: the weights
    of tc_weights at end `side` of subdomain j."""
    if P.tc == TC_ROBIN:
        return P.sigma * vtrace[1:]
    if P.tc >= TC_S03:
        return (tc_weights(P, j, side, V) @ np.asarray(vtrace, np.complex128))[1:]
    beta = P.beta()
    nt = P.nt
    out = np.zeros(nt, np.complex128)
    for n in range(1, nt + 1):
        out[n - 1] = P.c2() * np.dot(beta[n::-1][: n + 1], vtrace[: n + 1])
    return out


def s_flux(P: Problem, vtrace, j, side, V=None):
    """The operator the flux update of Eq. TransmisionCond applies to the trace of
    subdomain j at its end `side`: l_{j+1} = -r_j + (S_j + S_{j+1}) v_j(b_j) and
    r_{j-1} = -l_j + (S_j + S_{j-1}) v_j(a_j), the sum of the two subdomains'
    operators at the interface.  Reading: the paper prints 2 S-bar, which is this sum
    whenever the two sides' operators agree (Robin, S_0^2, S_0^3, S_1^2); for S_0^4 and
    S_1^4 the d_n W terms of the two sides have opposite signs and cancel in the sum,
    which is what makes converged SWR reproduce the monodomain solution."""
    nb, nside = (j + 1, 0) if side == 1 else (j - 1, 1)
    if P.tc >= TC_S03:
        return s_tilde(P, vtrace, j, side, V) + s_tilde(P, vtrace, nb, nside, V)
    return 2.0 * s_tilde(P, vtrace)


def apply_R(P: Problem, g, *, zero_u0=False, V=None):
    """One application of the interface operator R (Eq. interfacepbR): march
    every subdomain with the fluxes held in g, then form the new fluxes by
    Eq. TransmisionCond:
        r_{j-1} <- -l_j + 2 S-tilde v_j(a_j),   l_{j+1} <- -r_j + 2 S-tilde v_j(b_j)."""
    N, nt = P.nsub, P.nt
    g = np.asarray(g, dtype=np.complex128).reshape(P.nblk, nt)
    out = np.zeros_like(g)
    for j in range(N):
        a, b = int(P.off[j]), int(P.off[j + 1])
        u0 = np.zeros(b - a + 1, np.complex128) if zero_u0 else P.u0[a:b + 1]
        lj = g[blk_l(j)] if j > 0 else None
        rj = g[blk_r(j)] if j < N - 1 else None
        m = sub_march(P, j, u0, lj, rj, V=V)
        if j > 0:
            out[blk_r(j - 1)] = -lj + s_flux(P, m.va, j, 0, V)
        if j < N - 1:
            out[blk_l(j + 1)] = -rj + s_flux(P, m.vb, j, 1, V)
    return out


def build_d(P: Problem):
    """d = R 0 (Section 4.1): one march per subdomain with l = r = 0."""
    return apply_R(P, np.zeros((P.nblk, P.nt), np.complex128))


def build_columns(P: Problem, mode="zero_u0", d=None, V=None):
    """First columns of X^{j,1..4} (Section 4.1).  cols[j, p-1] is the first
    column of X^{j,p} (zero where the block does not exist).
    mode 'minus_d': the paper's construction, march with the true u_0 and a
    unit flux l_{j,1} = 1 (or r_{j,1} = 1), then subtract d.
    mode 'zero_u0': the same march with u_0 = 0, which by linearity
    (Props. 1-2) gives the column directly."""
    N, nt = P.nsub, P.nt
    cols = np.zeros((N, 4, nt), np.complex128)
    if mode == "minus_d" and d is None:
        d = build_d(P)
    e1 = np.zeros(nt, np.complex128)
    e1[0] = 1.0
    for j in range(N):
        a, b = int(P.off[j]), int(P.off[j + 1])
        u0 = P.u0[a:b + 1] if mode == "minus_d" else np.zeros(b - a + 1, np.complex128)
        zero = np.zeros(nt, np.complex128)
        for which in ("l", "r"):
            if which == "l" and j == 0:
                continue
            if which == "r" and j == N - 1:
                continue
            lj = (e1 if which == "l" else zero) if j > 0 else None
            rj = (e1 if which == "r" else zero) if j < N - 1 else None
            m = sub_march(P, j, u0, lj, rj, V=V)
            pa = 0 if which == "l" else 1     # X^{j,1} / X^{j,2}: output r_{j-1}
            pb = 2 if which == "l" else 3     # X^{j,3} / X^{j,4}: output l_{j+1}
            if j > 0:
                col = -lj + s_flux(P, m.va, j, 0, V)
                if mode == "minus_d":
                    col = col - d[blk_r(j - 1)]
                cols[j, pa] = col
            if j < N - 1:
                col = -rj + s_flux(P, m.vb, j, 1, V)
                if mode == "minus_d":
                    col = col - d[blk_l(j + 1)]
                cols[j, pb] = col
    return cols


def _s_flux_ext(P: Problem, vtrace, j, side):
    """s_flux in extended precision: the operator's binary64 coefficients (sigma, c2,
    beta, the weights of tc_weights) applied to an np.clongdouble trace in
    np.clongdouble arithmetic; entries n = 1..nt.  Also returns the magnitude of the
    summands of every entry, sum_s |K[n, s]| |v_s| (K the operator's weights)."""
    v = np.asarray(vtrace, np.clongdouble)
    av = np.abs(v)
    nt = P.nt
    out = np.zeros(nt, np.clongdouble)
    mag = np.zeros(nt, np.longdouble)
    if P.tc == TC_ROBIN:
        k = 2 * np.clongdouble(P.sigma)
        return k * v[1:], np.abs(k) * av[1:]
    if P.tc == TC_S02:
        beta = P.beta().astype(np.longdouble)
        c2 = 2 * np.clongdouble(P.c2())
        for n in range(1, nt + 1):
            acc = np.clongdouble(0)
            for s_ in range(n + 1):
                acc += beta[n - s_] * v[s_]
                mag[n - 1] += abs(beta[n - s_]) * av[s_]
            out[n - 1] = c2 * acc
        return out, np.abs(c2) * mag
    nb, nside = (j + 1, 0) if side == 1 else (j - 1, 1)
    w = (tc_weights(P, j, side).astype(np.clongdouble)
         + tc_weights(P, nb, nside).astype(np.clongdouble))
    for n in range(1, nt + 1):
        acc = np.clongdouble(0)
        for s_ in range(n + 1):
            acc += w[n, s_] * v[s_]
            mag[n - 1] += abs(w[n, s_]) * av[s_]
        out[n - 1] = acc
    return out, mag


def build_ext(P: Problem):
    """d = R 0 and the first columns (zero-u0 form) of ``build_d`` / ``build_columns``
    for a static potential, every march and flux in extended precision (march_ext).
    Returns (d, cols, d_mag, cols_mag): d and cols as np.clongdouble arrays shaped like
    theirs, and for every entry the magnitude of the summands that form it,
    |input flux| + sum_s |K[n, s]| |v_s|, which bounds what rounding of the trace v can
    do to an entry whose summands cancel (an almost transparent condition)."""
    if P.vkind != V_STATIC:
        raise NotImplementedError("build_ext: static V only")
    N, nt = P.nsub, P.nt
    d = np.zeros((P.nblk, nt), np.clongdouble)
    cols = np.zeros((N, 4, nt), np.clongdouble)
    dmag = np.zeros((P.nblk, nt), np.longdouble)
    cmag = np.zeros((N, 4, nt), np.longdouble)
    e1 = np.zeros(nt, np.complex128)
    e1[0] = 1.0
    zero = np.zeros(nt, np.complex128)
    for j in range(N):
        a, b = int(P.off[j]), int(P.off[j + 1])
        wl = tc_weights(P, j, 0) if (P.tc >= TC_S03 and j > 0) else None
        wr = tc_weights(P, j, 1) if (P.tc >= TC_S03 and j < N - 1) else None

        def run(u0, lj, rj):
            return march_ext(b - a + 1, P.h, P.dt, nt, P.local_V(j), u0, tc=P.tc,
                             sigma=P.sigma, tc_left=(j > 0), tc_right=(j < N - 1),
                             l=lj, r=rj, wl=wl, wr=wr)
        m = run(P.u0[a:b + 1], zero if j > 0 else None, zero if j < N - 1 else None)
        if j > 0:
            d[blk_r(j - 1)], dmag[blk_r(j - 1)] = _s_flux_ext(P, m.va, j, 0)
        if j < N - 1:
            d[blk_l(j + 1)], dmag[blk_l(j + 1)] = _s_flux_ext(P, m.vb, j, 1)
        z0 = np.zeros(b - a + 1, np.complex128)
        for which in ("l", "r"):
            if (which == "l" and j == 0) or (which == "r" and j == N - 1):
                continue
            lj = (e1 if which == "l" else zero) if j > 0 else None
            rj = (e1 if which == "r" else zero) if j < N - 1 else None
            m = run(z0, lj, rj)
            pa = 0 if which == "l" else 1
            pb = 2 if which == "l" else 3
            if j > 0:
                f, mg = _s_flux_ext(P, m.va, j, 0)
                cols[j, pa] = f - np.asarray(lj, np.clongdouble)
                cmag[j, pa] = mg + np.abs(np.asarray(lj, np.clongdouble))
            if j < N - 1:
                f, mg = _s_flux_ext(P, m.vb, j, 1)
                cols[j, pb] = f - np.asarray(rj, np.clongdouble)
                cmag[j, pb] = mg + np.abs(np.asarray(rj, np.clongdouble))
    return d, cols, dmag, cmag


def causal_conv(c, x):
    """y[n] = sum_{s<=n} c[n-s] x[s]: a lower-triangular Toeplitz block times x."""
    c = np.ascontiguousarray(c, dtype=np.complex128)
    x = np.ascontiguousarray(x, dtype=np.complex128)
    y = np.zeros(len(x), np.complex128)
    lib().or_causal_conv(len(x), _p(c), _p(x), _p(y))
    return y


def apply_L(P: Problem, cols, x):
    """L x from the first columns (Eq. chp1_Rlgb_lr with the Toeplitz blocks of
    Props. 3-4):  r_{j-1} = X^{j,1} l_j + X^{j,2} r_j,  l_{j+1} = X^{j,3} l_j + X^{j,4} r_j."""
    N, nt = P.nsub, P.nt
    x = np.asarray(x, dtype=np.complex128).reshape(P.nblk, nt)
    y = np.zeros_like(x)
    for j in range(N):
        xl = x[blk_l(j)] if j > 0 else None
        xr = x[blk_r(j)] if j < N - 1 else None
        if j > 0:
            acc = causal_conv(cols[j, 0], xl)
            if xr is not None:
                acc = acc + causal_conv(cols[j, 1], xr)
            y[blk_r(j - 1)] = acc
        if j < N - 1:
            acc = causal_conv(cols[j, 3], xr)
            if xl is not None:
                acc = acc + causal_conv(cols[j, 2], xl)
            y[blk_l(j + 1)] = acc
    return y


def apply_I_minus_L(P: Problem, cols, x):
    """(I - L) x (Eq. chp1_ILgd)."""
    x = np.asarray(x, dtype=np.complex128).reshape(P.nblk, P.nt)
    return x - apply_L(P, cols, x)


def dense_L(P: Problem, V=None):
    """Brute force: column (b, s) of L is R(e_{b,s}) - R(0), one march set per
    unit vector.  Tiny grids only."""
    nb, nt = P.nblk, P.nt
    d = apply_R(P, np.zeros((nb, nt)), V=V)
    Ld = np.zeros((nb * nt, nb * nt), np.complex128)
    for b in range(nb):
        for s in range(nt):
            e = np.zeros((nb, nt), np.complex128)
            e[b, s] = 1.0
            Ld[:, b * nt + s] = (apply_R(P, e, V=V) - d).ravel()
    return Ld, d


# --------------------------------------------------------------------------
# Krylov and fixed-point solvers
# --------------------------------------------------------------------------
@dataclass
class SolveResult:
    x: np.ndarray
    iterations: int
    residual: float
    history: list = field(default_factory=list)
    converged: bool = True


def gmres(apply_A, b, x0=None, m=30, tol=1e-10, maxit=2000, apply_Minv=None,
          rtol=0.0) -> SolveResult:
    """Restarted GMRES(m), Saad Alg. 6.9 (Arnoldi by modified Gram-Schmidt,
    Alg. 6.2, least squares by Givens rotations, Section 6.5.3).

    Optional left preconditioner apply_Minv: the Krylov space is that of
    M^{-1} A and the minimised residual is M^{-1}(b - A x) (the form of
    Eq. chp2_algopd_Lpf).  Convergence is declared on the TRUE residual
    ||b - A x||_2 <= max(tol, rtol ||b||) (absolute Euclidean norm), which is
    evaluated explicitly after every inner step."""
    b = np.asarray(b, dtype=np.complex128).ravel()
    n = b.size
    x = np.zeros(n, np.complex128) if x0 is None else np.array(x0, np.complex128).ravel()
    Minv = (lambda v: v) if apply_Minv is None else apply_Minv
    A = lambda v: np.asarray(apply_A(v), np.complex128).ravel()
    thresh = max(tol, rtol * np.linalg.norm(b))
    hist = []
    true_res = np.linalg.norm(b - A(x))
    hist.append(true_res)
    if true_res <= thresh:
        return SolveResult(x, 0, true_res, hist)
    it = 0
    while it < maxit:
        r = np.asarray(Minv(b - A(x)), np.complex128).ravel()
        beta = np.linalg.norm(r)
        if beta == 0.0:
            break
        Vb = np.zeros((m + 1, n), np.complex128)
        H = np.zeros((m + 1, m), np.complex128)
        cs = np.zeros(m, np.complex128)
        sn = np.zeros(m, np.complex128)
        s = np.zeros(m + 1, np.complex128)
        s[0] = beta
        Vb[0] = r / beta
        jdone = 0
        for jj in range(m):
            w = np.asarray(Minv(A(Vb[jj])), np.complex128).ravel()
            for i in range(jj + 1):                      # modified Gram-Schmidt
                H[i, jj] = np.vdot(Vb[i], w)
                w = w - H[i, jj] * Vb[i]
            H[jj + 1, jj] = np.linalg.norm(w)
            if H[jj + 1, jj] != 0.0:
                Vb[jj + 1] = w / H[jj + 1, jj]
            for i in range(jj):                          # previous rotations
                t = cs[i] * H[i, jj] + sn[i] * H[i + 1, jj]
                H[i + 1, jj] = -np.conj(sn[i]) * H[i, jj] + np.conj(cs[i]) * H[i + 1, jj]
                H[i, jj] = t
            # new rotation G = [[c, s], [-conj(s), c]], c real, zeroing H[jj+1, jj]
            a_, b_ = H[jj, jj], H[jj + 1, jj]
            breakdown = (b_ == 0.0)
            den = math.hypot(abs(a_), abs(b_))
            if den == 0.0:
                cs[jj], sn[jj] = 1.0, 0.0
            else:
                ph = a_ / abs(a_) if abs(a_) > 0 else 1.0
                cs[jj] = abs(a_) / den
                sn[jj] = ph * np.conj(b_) / den
            H[jj, jj] = cs[jj] * a_ + sn[jj] * b_
            H[jj + 1, jj] = 0.0
            s[jj + 1] = -np.conj(sn[jj]) * s[jj]
            s[jj] = cs[jj] * s[jj]
            it += 1
            jdone = jj + 1
            # current iterate and its true residual
            y = np.linalg.solve(np.triu(H[:jdone, :jdone]), s[:jdone])
            xk = x + Vb[:jdone].T @ y
            true_res = np.linalg.norm(b - A(xk))
            hist.append(true_res)
            if true_res <= thresh or it >= maxit:
                return SolveResult(xk, it, true_res, hist, true_res <= thresh)
            if breakdown:
                break
        y = np.linalg.solve(np.triu(H[:jdone, :jdone]), s[:jdone])
        x = x + Vb[:jdone].T @ y
    true_res = np.linalg.norm(b - A(x))
    return SolveResult(x, it, true_res, hist, true_res <= thresh)


def fixed_point(step, g0, tol=1e-10, maxit=2000) -> SolveResult:
    """Iterate g <- step(g) until ||g^{k+1} - g^k||_2 < tol (Algorithm 1)."""
    g = np.array(g0, np.complex128)
    hist = []
    for k in range(1, maxit + 1):
        gn = step(g)
        diff = np.linalg.norm((gn - g).ravel())
        hist.append(diff)
        g = gn
        if diff < tol:
            return SolveResult(g, k, diff, hist, True)
    return SolveResult(g, maxit, hist[-1] if hist else np.inf, hist, False)


def zero_potential_problem(P: Problem) -> Problem:
    """The same problem with V = 0 (preconditioner of Section 5, P = I - L_0)."""
    return Problem(P.a0, P.b0, P.nx, P.dt, P.nt, P.off, P.u0, np.zeros(P.nx), V_STATIC, P.tc,
                   P.sigma, P.nl_coef, P.nl_maxit, P.nl_tol)


def make_precond_inner(P: Problem, cols0, inner_rtol=1e-13):
    """x = P^{-1} y with P = I - L_0, by GMRES from the zero vector (Eq. Pxg)."""
    def apply(y):
        res = gmres(lambda v: apply_I_minus_L(P, cols0, v), y, None, m=30, tol=0.0,
                    rtol=inner_rtol, maxit=5000)
        return res.x
    return apply


def make_precond_dense(P: Problem, cols0):
    """x = P^{-1} y by a dense LU of P = I - L_0 (tiny grids; for cross-checks)."""
    n = P.nblk * P.nt
    Pm = np.zeros((n, n), np.complex128)
    for k in range(n):
        e = np.zeros(n, np.complex128)
        e[k] = 1.0
        Pm[:, k] = apply_I_minus_L(P, cols0, e).ravel()
    import scipy.linalg
    lu = scipy.linalg.lu_factor(Pm)
    return lambda y: scipy.linalg.lu_solve(lu, np.asarray(y, np.complex128).ravel())


# --------------------------------------------------------------------------
# Whole algorithms
# --------------------------------------------------------------------------
@dataclass
class SWRResult:
    g: np.ndarray
    uT: np.ndarray
    iterations: int
    residual: float
    d: Optional[np.ndarray] = None
    cols: Optional[np.ndarray] = None
    history: list = field(default_factory=list)
    jump: float = 0.0


def final_march(P: Problem, g):
    """Last step of Algorithms 2-3: march every subdomain with the converged
    fluxes; the interface node takes the left subdomain's value.  Also returns
    the largest mismatch |v_j(b_j) - v_{j+1}(a_{j+1})| (diagnostic)."""
    N = P.nsub
    g = np.asarray(g, np.complex128).reshape(P.nblk, P.nt)
    uT = np.zeros(P.nx, np.complex128)
    traces = []
    for j in range(N):
        a, b = int(P.off[j]), int(P.off[j + 1])
        lj = g[blk_l(j)] if j > 0 else None
        rj = g[blk_r(j)] if j < N - 1 else None
        m = sub_march(P, j, P.u0[a:b + 1], lj, rj)
        lo = a + (1 if j > 0 else 0)
        uT[lo:b + 1] = m.uT[lo - a:]
        traces.append(m)
    jump = 0.0
    for j in range(N - 1):
        jump = max(jump, float(np.max(np.abs(traces[j].vb - traces[j + 1].va))))
    return uT, jump


def residual(P: Problem, cols, d, g):
    return float(np.linalg.norm((d - apply_I_minus_L(P, cols, g)).ravel()))


def solve_new(P: Problem, solver="gmres", tol=1e-10, restart=30, maxit=2000, g0=None,
              cols_mode="zero_u0", rtol=0.0) -> SWRResult:
    """Algorithm 3 (new algorithm, V = V(x)): build d and L explicitly, solve
    (I - L) g = d by GMRES or the fixed point g <- L g + d, final march."""
    d = build_d(P)
    cols = build_columns(P, cols_mode, d=d)
    g0 = np.zeros_like(d) if g0 is None else np.asarray(g0, np.complex128).reshape(d.shape)
    if solver == "gmres":
        res = gmres(lambda v: apply_I_minus_L(P, cols, v), d, g0, m=restart, tol=tol,
                    maxit=maxit, rtol=rtol)
        g = res.x.reshape(d.shape)
        it, hist = res.iterations, res.history
    else:
        res = fixed_point(lambda v: apply_L(P, cols, v) + d, g0, tol=tol, maxit=maxit)
        g, it, hist = res.x, res.iterations, res.history
    uT, jump = final_march(P, g)
    return SWRResult(g, uT, it, residual(P, cols, d, g), d, cols, hist, jump)


def solve_classical(P: Problem, tol=1e-10, maxit=2000, g0=None) -> SWRResult:
    """Algorithm 1: g^{k+1} = R g^k with full marches until ||g^{k+1}-g^k|| < tol."""
    g0 = np.zeros((P.nblk, P.nt), np.complex128) if g0 is None else g0
    res = fixed_point(lambda v: apply_R(P, v), g0, tol=tol, maxit=maxit)
    uT, jump = final_march(P, res.x)
    return SWRResult(res.x, uT, res.iterations, res.history[-1], None, None, res.history,
                     jump)


def solve_matrix_free(P: Problem, precond="zero_potential", tol=1e-10, restart=30,
                      maxit=2000, g0=None, inner="gmres", rtol=0.0) -> SWRResult:
    """Algorithm 2 / Section 5 for V = V(t,x): d = R 0, (I - L) g = g - R g + d
    applied matrix-free, GMRES left-preconditioned by P = I - L_0
    (Eq. chp2_algopd_Lpf) with P^{-1} by inner GMRES (Eq. Pxg) or, on tiny grids,
    a dense LU ('dense')."""
    d = build_d(P)
    A = lambda v: (np.asarray(v, np.complex128).reshape(d.shape)
                   - apply_R(P, np.asarray(v).reshape(d.shape)) + d)
    Minv = None
    if precond == "zero_potential":
        P0 = zero_potential_problem(P)
        cols0 = build_columns(P0, "zero_u0")
        Minv = make_precond_dense(P0, cols0) if inner == "dense" else \
            make_precond_inner(P0, cols0)
    g0 = np.zeros_like(d) if g0 is None else g0
    res = gmres(A, d, g0, m=restart, tol=tol, maxit=maxit, apply_Minv=Minv, rtol=rtol)
    g = res.x.reshape(d.shape)
    uT, jump = final_march(P, g)
    return SWRResult(g, uT, res.iterations, res.residual, d, None, res.history, jump)


def solve_nonlinear(P: Problem, precond=True, tol=1e-10, maxit=2000, g0=None,
                    inner="gmres") -> SWRResult:
    """Section 5 for V = f(u): g^{k+1} = g^k - P^{-1}(g^k - R_nl g^k)
    (reading of Eq. chp2_algopd_NL), P = I - L_0; without the preconditioner
    this is Algorithm 1.  Stops when ||g^{k+1} - g^k||_2 < tol."""
    g0 = np.zeros((P.nblk, P.nt), np.complex128) if g0 is None else g0
    if precond:
        P0 = zero_potential_problem(P)
        cols0 = build_columns(P0, "zero_u0")
        Minv = make_precond_dense(P0, cols0) if inner == "dense" else \
            make_precond_inner(P0, cols0)
        step = lambda g: g - np.asarray(Minv((g - apply_R(P, g)).ravel())).reshape(g.shape)
    else:
        step = lambda g: apply_R(P, g)
    res = fixed_point(step, g0, tol=tol, maxit=maxit)
    uT, jump = final_march(P, res.x)
    return SWRResult(res.x, uT, res.iterations, res.history[-1], None, None, res.history,
                     jump)


# --------------------------------------------------------------------------
# Monodomain reference and the interface vector it implies
# --------------------------------------------------------------------------
def mono_march(P: Problem, sel=None) -> MarchResult:
    """Crank-Nicolson + P1 on the whole of (a0, b0) with Neumann ends
    (Eq. Schequ, Eq. CNS_L / CNS_NL), the solution converged SWR reproduces."""
    return march(P.nx, P.h, P.dt, P.nt, P.V, P.u0, vkind=P.vkind, tc=P.tc, sigma=P.sigma,
                 tc_left=False, tc_right=False, nl_coef=P.nl_coef, nl_maxit=P.nl_maxit,
                 nl_tol=P.nl_tol, sel=sel)


def mono_interface(P: Problem):
    """The interface vector g* that converged SWR must reach, computed from the
    monodomain solution.  At interface node k between subdomains j and j+1 the
    FEM rows of the two halves give the normal derivatives
      d_n v_left(b_j)  = [(2i/dt) M_L u_{n-1} - A_L v_n]_last,
      d_n v_right(a_{j+1}) = [(2i/dt) M_R u_{n-1} - A_R v_n]_first,
    (A = (2i/dt)M - S + M_W on the half-subdomain, Eq. AvML; nonlinear case
    with b_f of Eq. AvMNL) and the fluxes of Section 2.2 are
      r_j = d_n v_left(b_j) + S-bar v(x_k),  l_{j+1} = d_n v_right(a_{j+1}) + S-bar v(x_k).
    Returns (g*, u(T) of the monodomain)."""
    N, nt, h, dt = P.nsub, P.nt, P.h, P.dt
    ks = [int(P.off[j]) for j in range(1, N)]
    sel = []
    for k in ks:
        sel += [k - 1, k, k + 1]
    m = mono_march(P, sel=np.array(sel))
    vs = m.vsel                                   # (nt+1, 3(N-1)), row 0 = u0
    us = np.zeros_like(vs)                        # u_t at the selected nodes
    us[0] = P.u0[np.array(sel)]
    for t in range(1, nt + 1):
        us[t] = 2.0 * vs[t] - us[t - 1]
    I2 = 2j / dt
    g = np.zeros((P.nblk, nt), np.complex128)
    for q, k in enumerate(ks):
        j = q                                      # interface between j and j+1
        vm, v0, vp = vs[1:, 3 * q], vs[1:, 3 * q + 1], vs[1:, 3 * q + 2]
        um, u0_, up = us[:-1, 3 * q], us[:-1, 3 * q + 1], us[:-1, 3 * q + 2]
        if P.vkind == V_TIME:
            Vt = P.V[:, k - 1:k + 2]
            W = 0.5 * (Vt[1:] + Vt[:-1])          # (nt, 3)
            Wm, W0, Wp = W[:, 0], W[:, 1], W[:, 2]
        elif P.vkind == V_STATIC:
            Wm, W0, Wp = (np.full(nt, P.V[k - 1]), np.full(nt, P.V[k]), np.full(nt, P.V[k + 1]))
        else:
            Wm = np.full(nt, P.V[k - 1]) + P.nl_coef * np.abs(vm) ** 2
            W0 = np.full(nt, P.V[k]) + P.nl_coef * np.abs(v0) ** 2
            Wp = np.full(nt, P.V[k + 1]) + P.nl_coef * np.abs(vp) ** 2
        # last row of the left half: element [k-1, k]
        dnl = (I2 * (h / 6 * (um - vm) + h / 3 * (u0_ - v0)) + (v0 - vm) / h
               - (h / 12 * (Wm + W0) * vm + h / 12 * (Wm + 3 * W0) * v0))
        # first row of the right half: element [k, k+1]
        dnr = (I2 * (h / 3 * (u0_ - v0) + h / 6 * (up - vp)) + (v0 - vp) / h
               - (h / 12 * (3 * W0 + Wp) * v0 + h / 12 * (W0 + Wp) * vp))
        vtrace = vs[:, 3 * q + 1]
        g[blk_r(j)] = dnl + s_tilde(P, vtrace, j, 1)
        g[blk_l(j + 1)] = dnr + s_tilde(P, vtrace, j + 1, 0)
    return g, m.uT


# --------------------------------------------------------------------------
# Gradient of a final-time misfit (discrete adjoint of the monodomain scheme)
# --------------------------------------------------------------------------
def _mass_apply(md, mo, x):
    """M x for the P1 mass matrix given as (diag, offdiag)."""
    y = md * x
    y[:-1] += mo * x[1:]
    y[1:] += mo * x[:-1]
    return y


def misfit(P: Problem, uT, u_target):
    """J = (u(T) - u_target)^H M (u(T) - u_target), the M-weighted misfit."""
    md, mo, _, _, _, _ = p1_matrices(P.nx, P.h, None)
    e = np.asarray(uT, np.complex128) - np.asarray(u_target, np.complex128)
    return float(np.real(np.vdot(e, _mass_apply(md, mo, e))))


def potential_form(x, y, h):
    """Re( x^H (dM_W / dW_k) y ) for every node k: the derivative of the P1
    generalised mass matrix (exact quadrature of the P1 interpolant of W,
    Eq. AvML) with respect to the nodal value W_k.  Element [a, b] contributes
    h/12 (3 x_a* y_a + x_a* y_b + x_b* y_a + x_b* y_b) to k = a and
    h/12 (x_a* y_a + x_a* y_b + x_b* y_a + 3 x_b* y_b) to k = b."""
    s = np.conj(x) * y
    c = np.conj(x[:-1]) * y[1:] + np.conj(x[1:]) * y[:-1]
    g = np.zeros(len(x), np.complex128)
    g[:-1] += h / 12.0 * (3.0 * s[:-1] + c + s[1:])
    g[1:] += h / 12.0 * (s[:-1] + c + 3.0 * s[1:])
    return np.real(g)


def adjoint_gradient(P: Problem, u_target):
    """dJ/dV for J = (u_N - u_target)^H M (u_N - u_target), u_N the monodomain
    Crank-Nicolson solution at T (Eq. CNS_L with the P1 matrices of Eq. AvML,
    Neumann ends; converged SWR reproduces it), V static and real.

    Discrete adjoint of the scheme A v_n = B u_{n-1}, u_n = 2 v_n - u_{n-1}
    with A = (2i/dt) M - S + M_V and B = (2i/dt) M: with dJ = Re(lam_n^H du_n),
    lam_N = 2 M (u_N - u_target) and, for n = N..1,
        A^H mu_n = lam_n,                      (A^H = conj(A): A is symmetric)
        dJ/dV   += -2 Re(mu_n^H (dM_V/dV) v_n),
        lam_{n-1} = 2 B^H mu_n - lam_n.
    Every v_n comes from the forward march.  Returns (J, dJ/dV)."""
    if P.vkind != V_STATIC:
        raise NotImplementedError("adjoint gradient: static V only")
    n, h, dt, nt = P.nx, P.h, P.dt, P.nt
    m = mono_march(P, sel=np.arange(n))
    vs = m.vsel                                   # row t = v_t (row 0 = u0)
    md, mo, sd, so, wd, wo = p1_matrices(n, h, P.V)
    I2 = 2j / dt
    dg = I2 * md - sd + wd
    lo = I2 * mo - so + wo
    e = m.uT - np.asarray(u_target, np.complex128)
    Me = _mass_apply(md, mo, e)
    J = float(np.real(np.vdot(e, Me)))
    lam = 2.0 * Me
    grad = np.zeros(n)
    for t in range(nt, 0, -1):
        mu = thomas(np.conj(lo), np.conj(dg), np.conj(lo), lam)
        grad += -2.0 * potential_form(mu, vs[t], h)
        lam = 2.0 * np.conj(I2) * _mass_apply(md, mo, mu) - lam
    return J, grad


def adjoint_gradient_tdep(P: Problem, u_target):
    """dJ/dV(t_m, x_k) for a tabulated time-dependent potential (rows m = 0..nt),
    J = (u_N - u_target)^H M (u_N - u_target), u_N the monodomain Crank-Nicolson
    solution (Eq. CNS_L with W_n = (V_n + V_{n-1})/2, Neumann ends).

    Discrete adjoint of A_n v_n = B u_{n-1}, u_n = 2 v_n - u_{n-1}, with
    A_n = (2i/dt) M - S + M_{W_n} (complex symmetric, so A_n^H = conj(A_n)) and
    B = (2i/dt) M: with lam_N = 2 M (u_N - u_target) and, for n = N..1,
        conj(A_n) mu_n = lam_n,
        G_n(k) = -2 Re(mu_n^H (dM_W/dW_k) v_n)       (= dJ/dW_n(k)),
        lam_{n-1} = 2 B^H mu_n - lam_n;
    since W_n = (V_n + V_{n-1})/2, dJ/dV_m = (G_m + G_{m+1}) / 2 (G_0 = G_{N+1} = 0).
    Every v_n comes from the forward march.  Returns (J, dJ/dV) with dJ/dV of
    shape (nt + 1, nx)."""
    if P.vkind != V_TIME:
        raise NotImplementedError("adjoint_gradient_tdep: time-dependent V only")
    n, h, dt, nt = P.nx, P.h, P.dt, P.nt
    m = mono_march(P, sel=np.arange(n))
    vs = m.vsel                                   # row t = v_t (row 0 = u0)
    md, mo, sd, so, _, _ = p1_matrices(n, h, None)
    I2 = 2j / dt
    e = m.uT - np.asarray(u_target, np.complex128)
    Me = _mass_apply(md, mo, e)
    J = float(np.real(np.vdot(e, Me)))
    lam = 2.0 * Me
    G = np.zeros((nt + 2, n))
    for t in range(nt, 0, -1):
        W = 0.5 * (P.V[t] + P.V[t - 1])
        _, _, _, _, wd, wo = p1_matrices(n, h, W)
        dg = I2 * md - sd + wd
        lo = I2 * mo - so + wo
        mu = thomas(np.conj(lo), np.conj(dg), np.conj(lo), lam)
        G[t] = -2.0 * potential_form(mu, vs[t], h)
        lam = 2.0 * np.conj(I2) * _mass_apply(md, mo, mu) - lam
    grad = 0.5 * (G[0:nt + 1] + G[1:nt + 2])
    return J, grad


def _potential_form_matrix(v, h):
    """The real-linear map w -> r(w), r_k = Re( sum_ab v_a (dM_W/dW_k)_ab w_b )
    (the P1 rule of Eq. AvML, no conjugation), as a sparse real matrix acting
    on [Re w; Im w].  Element [a, b]: dM/dW_a = h/12 (3,1;1,1), dM/dW_b =
    h/12 (1,1;1,3)."""
    import scipy.sparse as sp
    n = len(v)
    rows, cols, vals = [], [], []

    def add(k, a, b, wgt):          # r_k += wgt Re(v_a w_b)
        # Re(v_a w_b) = v_a.re w_b.re - v_a.im w_b.im
        rows.extend([k, k]); cols.extend([b, n + b])
        vals.extend([wgt * v[a].real, -wgt * v[a].imag])

    c = h / 12.0
    for e in range(n - 1):
        a, b = e, e + 1
        for (ia, ib, wa, wb) in ((a, a, 3.0, 1.0), (a, b, 1.0, 1.0), (b, a, 1.0, 1.0),
                                 (b, b, 1.0, 3.0)):
            add(a, ia, ib, c * wa)
            add(b, ia, ib, c * wb)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, 2 * n))


def adjoint_gradient_nl(P: Problem, u_target):
    """dJ/dV0 for J = (u_N - u_target)^H M (u_N - u_target), u_N the monodomain
    solution of the nonlinear scheme (Eq. CNS_NL / AvMNL with f(v) = c|v|^2 and
    the static V0, Neumann ends), each step solved to convergence:
        F(v_n) = A0 v_n + M_{c|v_n|^2} v_n - B u_{n-1} = 0,  u_n = 2 v_n - u_{n-1},
    A0 = (2i/dt) M - S + M_V0, B = (2i/dt) M.  The linearisation in v is real-
    linear, T(x) = At x + K(x) with At = A0 + M_{c|v|^2} and
    K(x) = M_{2c Re(conj(v) x)} v, whose adjoint for Re(y^H x) is
    T*(y) = conj(At) y + 2c v . Re(v^H (dM/dW_k) y).  With lam_N = 2 M (u_N - u_t):
        T_n* mu_n = 2 lam_n  (solved exactly as a real 2n x 2n sparse system),
        dJ/dV0 += -Re(mu_n^H (dM/dV0) v_n),
        lam_{n-1} = B^H mu_n - lam_n.
    Returns (J, dJ/dV0)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    if P.vkind != V_NONLINEAR:
        raise NotImplementedError("adjoint_gradient_nl: nonlinear problems only")
    n, h, dt, nt, coef = P.nx, P.h, P.dt, P.nt, P.nl_coef
    m = mono_march(P, sel=np.arange(n))
    vs = m.vsel
    md, mo, sd, so, wd, wo = p1_matrices(n, h, P.V)
    I2 = 2j / dt
    dg0 = I2 * md - sd + wd
    lo0 = I2 * mo - so + wo
    e = m.uT - np.asarray(u_target, np.complex128)
    Me = _mass_apply(md, mo, e)
    J = float(np.real(np.vdot(e, Me)))
    lam = 2.0 * Me
    grad = np.zeros(n)
    for t in range(nt, 0, -1):
        v = vs[t]
        _, _, _, _, wdv, wov = p1_matrices(n, h, coef * np.abs(v) ** 2)
        Ct = sp.diags([np.conj(lo0 + wov), np.conj(dg0 + wdv), np.conj(lo0 + wov)], [-1, 0, 1],
                      format="csr")                                  # conj(At)
        Creal = sp.bmat([[Ct.real, -Ct.imag], [Ct.imag, Ct.real]], format="csr")
        # 2c v . Re(v^H dM_k y) = 2c v . R(conj(v)) y
        R = _potential_form_matrix(np.conj(v), h)
        Kreal = sp.vstack([sp.diags(2 * coef * v.real) @ R, sp.diags(2 * coef * v.imag) @ R])
        rhs = 2.0 * lam
        x = spla.spsolve((Creal + Kreal).tocsc(), np.concatenate([rhs.real, rhs.imag]))
        mu = x[:n] + 1j * x[n:]
        grad += -potential_form(mu, v, h)
        lam = np.conj(I2) * _mass_apply(md, mo, mu) - lam
    return J, grad
