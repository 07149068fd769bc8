"""Writes nl_gradient_config5.npz: the oracle's discrete-adjoint gradient dJ/dV0
(and J) of the final-time misfit for the full-size nonlinear workload (20001
nodes, 1000 steps of dt = 5e-4, Eq. CNS_NL with f = |v|^2, inner fixed points to
1e-13).  The target u_target is the oracle's monodomain u(T) of the same problem
with the seeded perturbed potential (every well depth scaled by 1 + 0.05 xi), and
is stored with the gradient.  Calls only the oracle and the input generators;
about five minutes on one core.

    python tests/golden/make_nl_gradient.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_1503_02564_gb300 import workloads as W  # noqa: E402


def main():
    wl = W.config5()
    P = O.Problem(wl.a0, wl.b0, wl.nx, wl.dt, wl.nt, wl.off.astype(np.int64), wl.u0, wl.V,
                  vkind=wl.vkind, tc=wl.tc, sigma=wl.sigma, nl_coef=wl.nl_coef, nl_tol=1e-13,
                  nl_maxit=50)
    Pt = O.Problem(wl.a0, wl.b0, wl.nx, wl.dt, wl.nt, wl.off.astype(np.int64), wl.u0,
                   W.config5_target_potential(wl), vkind=wl.vkind, tc=wl.tc, sigma=wl.sigma,
                   nl_coef=wl.nl_coef, nl_tol=1e-13, nl_maxit=50)
    u_target = O.mono_march(Pt).uT
    J, g = O.adjoint_gradient_nl(P, u_target)
    np.savez_compressed(os.path.join(HERE, "nl_gradient_config5.npz"), J=np.float64(J), grad=g,
                        u_target=u_target)
    print("J =", J, " |dJ/dV0| =", np.linalg.norm(g))


if __name__ == "__main__":
    main()
