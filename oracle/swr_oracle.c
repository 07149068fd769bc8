/*
 * Plain FP64 CPU oracle for the Schwarz waveform relaxation (SWR) hot path of
 * Besse & Xing, "Schwarz waveform relaxation method for one dimensional
 * Schroedinger equation with general potential" (arXiv 1503.02564).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path and is deliberately slow and literal: one textbook Thomas solve
 * per time step, no blocking, no fusion, no reordering.
 *
 * Compiled with -O2 -ffp-contract=off (no fused multiply-add, IEEE binary64,
 * round to nearest).  Complex numbers are C99 `double complex`; at the ABI the
 * arrays are interleaved (re, im) doubles, which C99 guarantees is the same
 * layout.
 *
 * Notation follows the paper: Crank-Nicolson in the variable
 * v_n = (u_n + u_{n-1})/2 (Eq. CNS_L), P1 finite elements in space with mass
 * matrix M, stiffness matrix S and generalised mass matrix M_W (Eq. AvML),
 * transmission operator B = d_n + S-bar (Eq. S1S2 / condlimit), with the
 * boundary matrix B and boundary vector b of Eq. AvML.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------------ */
/* P1 finite element matrices on a uniform mesh (Section 2.2, Eq. AvML).     */
/* ------------------------------------------------------------------------ */
/*
 * n nodes, spacing h.  Element [x_e, x_{e+1}] contributes
 *   mass:      h/6 * [[2,1],[1,2]]
 *   stiffness: 1/h * [[1,-1],[-1,1]]
 *   generalised mass for int W v phi with W interpolated as a P1 function and
 *   integrated exactly (int phi_e^3 = h/4, int phi_e^2 phi_{e+1} = h/12):
 *              h/12 * [[3W_e+W_{e+1}, W_e+W_{e+1}], [W_e+W_{e+1}, W_e+3W_{e+1}]]
 * Outputs: diagonals (length n) and the (symmetric) off-diagonals (length n-1).
 * W may be NULL (then wd, wo are zero).
 */
void or_p1_matrices(int n, double h, const double *W, double *md, double *mo,
                    double *sd, double *so, double *wd, double *wo)
{
    int i, e;
    for (i = 0; i < n; ++i) { md[i] = 0.0; sd[i] = 0.0; wd[i] = 0.0; }
    for (i = 0; i < n - 1; ++i) { mo[i] = 0.0; so[i] = 0.0; wo[i] = 0.0; }
    for (e = 0; e < n - 1; ++e) {
        md[e] += h / 3.0;
        md[e + 1] += h / 3.0;
        mo[e] += h / 6.0;
        sd[e] += 1.0 / h;
        sd[e + 1] += 1.0 / h;
        so[e] += -1.0 / h;
        if (W) {
            wd[e] += h / 12.0 * (3.0 * W[e] + W[e + 1]);
            wd[e + 1] += h / 12.0 * (W[e] + 3.0 * W[e + 1]);
            wo[e] += h / 12.0 * (W[e] + W[e + 1]);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Textbook Thomas algorithm (no pivoting) for a tridiagonal system.         */
/* ------------------------------------------------------------------------ */
/*
 * lo[i] couples row i+1 to column i, up[i] couples row i to column i+1
 * (both length n-1), dg the diagonal.  x holds the right-hand side on entry
 * and the solution on exit.  work must hold n complex values.
 * Returns 0, or -(i+1) when pivot i is exactly zero.
 */
int or_thomas(int n, const cplx *lo, const cplx *dg, const cplx *up, cplx *x,
              cplx *work)
{
    int i;
    cplx piv = dg[0];
    if (piv == 0.0) return -1;
    work[0] = (n > 1) ? up[0] / piv : 0.0;
    x[0] = x[0] / piv;
    for (i = 1; i < n; ++i) {
        piv = dg[i] - lo[i - 1] * work[i - 1];
        if (piv == 0.0) return -(i + 1);
        work[i] = (i < n - 1) ? up[i] / piv : 0.0;
        x[i] = (x[i] - lo[i - 1] * x[i - 1]) / piv;
    }
    for (i = n - 2; i >= 0; --i) x[i] = x[i] - work[i] * x[i + 1];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One Crank-Nicolson march on a segment of n nodes.                          */
/* ------------------------------------------------------------------------ */
/*
 * Solves, for n_step = 1..nt, the subdomain system of Eq. AvML
 *   (A_n - B_n) v_n = (2i/dt) M u_{n-1} + b_n - Q^T (l_n, r_n)^T,
 *   A_n = (2i/dt) M - S + M_{W_n},          u_n = 2 v_n - u_{n-1},
 * with W_n = (V_n + V_{n-1})/2 (Eq. CNS_L).  An end that carries a
 * transmission condition gets the boundary matrix entry sigma0 (B = sigma0 Q^T Q)
 * and the boundary vector b_n; a Neumann end gets neither (natural condition,
 * Eq. Schequ).  With both ends Neumann and no fluxes this is the monodomain
 * scheme.
 *
 * Transmission operator S-bar (Section 2.2):
 *   tc == 0, Robin:   S-bar v_n = sigma * v_n            -> sigma0 = sigma, b_n = 0
 *   tc == 1, S_0^2:   S-bar v_n = c2 sum_{s=0}^{n} beta_{n-s} v_s
 *                     -> sigma0 = c2 beta_0, b_n = c2 sum_{s=0}^{n-1} beta_{n-s} v_s
 *                        at that end (sign from the proof of Prop. 1), v_0 = u_0.
 *   tc == 2, any S-bar linear in the trace: S-bar v_n = sum_{s=0}^{n} w[n][s] v_s
 *                     with w given per end (wl, wr: (nt+1) x (nt+1), row n holds
 *                     s = 0..n) -> the end's matrix entry at step n is w[n][n] and
 *                     b_n = sum_{s<n} w[n][s] v_s (S_0^3, S_0^4, S_1^2, S_1^4).
 *
 * Potential (vkind):
 *   0  static V(x): V has n entries;
 *   1  time dependent: row t (0..nt) of V, V + t*vstride, holds V(t_t, x);
 *   2  nonlinear f(v) v with f(v) = nl_coef |v|^2 (Eq. CNS_NL) plus a static
 *      V0(x) (V, n entries) kept in the matrix.  Each step runs the fixed point
 *      of Eq. AvMNL: zeta^0 = v_{n-1}, and
 *        (2i/dt M - S + M_{V0} - B) zeta^{s+1}
 *            = (2i/dt) M u_{n-1} - b_{f(zeta^s)} + b_n - Q^T (l_n, r_n)^T,
 *      with b_f = M_{nl_coef |zeta|^2} zeta (the P1 rule above applied to
 *      W = nl_coef |zeta|^2), stopping when
 *        max|zeta^{s+1} - zeta^s| <= nl_tol * max(1, max|zeta^s|)
 *      or after nl_maxit iterations.
 *
 * Inputs (interleaved complex): u0 (n), l and r (nt each; entry n_step-1 is the
 * flux of step n_step; NULL means zero), beta (nt+1, used when tc == 1), wl and
 * wr (used when tc == 2, NULL at an end without a transmission condition).
 * Outputs: va, vb (nt+1 each; entry t is v_t at the left / right end, entry 0
 * is u_0 there), uT (n, u at the final time), nl_iters (nt, inner counts;
 * optional), vsel (optional: (nt+1) x nsel values of v_t at the nodes sel[]).
 * Returns 0, or a negative code if a zero pivot appears (SINGULAR), or -1000000
 * when the nonlinear fixed point did not converge within nl_maxit.
 */
int or_march(int n, double h, double dt, int nt, int vkind, const double *V,
             long vstride, double nl_coef, int nl_maxit, double nl_tol, int tc,
             double sig_re, double sig_im, double c2_re, double c2_im,
             const double *beta, int tc_left, int tc_right, const double *u0_,
             const double *l_, const double *r_, double *va_, double *vb_,
             double *uT_, int *nl_iters, int nsel, const int *sel, double *vsel_,
             const double *wl_, const double *wr_)
{
    const cplx *wl = (const cplx *)wl_, *wr = (const cplx *)wr_;
    const long nw = nt + 1;
    const cplx I2dt = 2.0 * I / dt;
    const cplx sigma = sig_re + I * sig_im;
    const cplx c2 = c2_re + I * c2_im;
    const cplx *u0 = (const cplx *)u0_;
    const cplx *l = (const cplx *)l_;
    const cplx *r = (const cplx *)r_;
    cplx *va = (cplx *)va_, *vb = (cplx *)vb_, *uT = (cplx *)uT_;
    cplx *vsel = (cplx *)vsel_;
    double *md = malloc(sizeof(double) * n), *mo = malloc(sizeof(double) * n);
    double *sd = malloc(sizeof(double) * n), *so = malloc(sizeof(double) * n);
    double *wd = malloc(sizeof(double) * n), *wo = malloc(sizeof(double) * n);
    double *W = malloc(sizeof(double) * n);
    double *fd = malloc(sizeof(double) * n), *fo = malloc(sizeof(double) * n);
    double *tmp1 = malloc(sizeof(double) * n), *tmp2 = malloc(sizeof(double) * n);
    double *tmp3 = malloc(sizeof(double) * n), *tmp4 = malloc(sizeof(double) * n);
    cplx *u = malloc(sizeof(cplx) * n), *v = malloc(sizeof(cplx) * n);
    cplx *rhs = malloc(sizeof(cplx) * n), *rhs0 = malloc(sizeof(cplx) * n);
    cplx *zeta = malloc(sizeof(cplx) * n), *vprev = malloc(sizeof(cplx) * n);
    cplx *dg = malloc(sizeof(cplx) * n), *lo = malloc(sizeof(cplx) * n);
    cplx *work = malloc(sizeof(cplx) * n);
    cplx sigma0 = (tc == 0) ? sigma : c2 * beta[0];
    int status = 0, i, t, q;

    for (i = 0; i < n; ++i) { u[i] = u0[i]; vprev[i] = u0[i]; }
    va[0] = u0[0];
    vb[0] = u0[n - 1];
    if (vsel) for (q = 0; q < nsel; ++q) vsel[q] = u0[sel[q]];

    /* Static potential (vkind 0) or static V0 (vkind 2): matrices once. */
    or_p1_matrices(n, h, (vkind == 1) ? NULL : V, md, mo, sd, so, wd, wo);

    for (t = 1; t <= nt && status == 0; ++t) {
        if (vkind == 1) {
            /* W_n = (V_n + V_{n-1}) / 2, Eq. CNS_L */
            for (i = 0; i < n; ++i)
                W[i] = 0.5 * (V[(long)t * vstride + i] + V[(long)(t - 1) * vstride + i]);
            or_p1_matrices(n, h, W, md, mo, sd, so, wd, wo);
        }
        /* Matrix A_n - B_n (complex symmetric tridiagonal). */
        for (i = 0; i < n; ++i) dg[i] = I2dt * md[i] - sd[i] + wd[i];
        for (i = 0; i < n - 1; ++i) lo[i] = I2dt * mo[i] - so[i] + wo[i];
        if (tc_left) dg[0] -= (tc == 2) ? wl[(long)t * nw + t] : sigma0;
        if (tc_right) dg[n - 1] -= (tc == 2) ? wr[(long)t * nw + t] : sigma0;

        /* (2i/dt) M u_{n-1} */
        for (i = 0; i < n; ++i) {
            cplx s = md[i] * u[i];
            if (i > 0) s += mo[i - 1] * u[i - 1];
            if (i < n - 1) s += mo[i] * u[i + 1];
            rhs0[i] = I2dt * s;
        }
        /* + b_n (S_0^2 history), - Q^T (l_n, r_n)^T */
        if (tc == 1) {
            int s;
            if (tc_left) {
                cplx acc = 0.0;
                for (s = 0; s < t; ++s) acc += beta[t - s] * va[s];
                rhs0[0] += c2 * acc;
            }
            if (tc_right) {
                cplx acc = 0.0;
                for (s = 0; s < t; ++s) acc += beta[t - s] * vb[s];
                rhs0[n - 1] += c2 * acc;
            }
        }
        if (tc == 2) {
            int s;
            if (tc_left) {
                cplx acc = 0.0;
                for (s = 0; s < t; ++s) acc += wl[(long)t * nw + s] * va[s];
                rhs0[0] += acc;
            }
            if (tc_right) {
                cplx acc = 0.0;
                for (s = 0; s < t; ++s) acc += wr[(long)t * nw + s] * vb[s];
                rhs0[n - 1] += acc;
            }
        }
        if (tc_left && l) rhs0[0] -= l[t - 1];
        if (tc_right && r) rhs0[n - 1] -= r[t - 1];

        if (vkind != 2) {
            for (i = 0; i < n; ++i) v[i] = rhs0[i];
            status = or_thomas(n, lo, dg, lo, v, work);
            if (nl_iters) nl_iters[t - 1] = 0;
        } else {
            /* Fixed point of Eq. AvMNL, zeta^0 = v_{n-1}. */
            int it, conv = 0;
            for (i = 0; i < n; ++i) zeta[i] = vprev[i];
            for (it = 1; it <= nl_maxit; ++it) {
                double dmax = 0.0, zmax = 0.0;
                for (i = 0; i < n; ++i) W[i] = nl_coef * creal(zeta[i] * conj(zeta[i]));
                or_p1_matrices(n, h, W, tmp1, tmp2, tmp3, tmp4, fd, fo);
                for (i = 0; i < n; ++i) {
                    cplx bf = fd[i] * zeta[i];
                    if (i > 0) bf += fo[i - 1] * zeta[i - 1];
                    if (i < n - 1) bf += fo[i] * zeta[i + 1];
                    rhs[i] = rhs0[i] - bf;
                }
                status = or_thomas(n, lo, dg, lo, rhs, work);
                if (status) break;
                for (i = 0; i < n; ++i) {
                    double d = cabs(rhs[i] - zeta[i]), z = cabs(zeta[i]);
                    if (d > dmax) dmax = d;
                    if (z > zmax) zmax = z;
                }
                for (i = 0; i < n; ++i) zeta[i] = rhs[i];
                if (dmax <= nl_tol * (zmax > 1.0 ? zmax : 1.0)) { conv = 1; break; }
            }
            if (nl_iters) nl_iters[t - 1] = it;
            if (!conv && status == 0) status = -1000000;
            for (i = 0; i < n; ++i) v[i] = zeta[i];
        }
        for (i = 0; i < n; ++i) {
            u[i] = 2.0 * v[i] - u[i];
            vprev[i] = v[i];
        }
        va[t] = v[0];
        vb[t] = v[n - 1];
        if (vsel) for (q = 0; q < nsel; ++q) vsel[(long)t * nsel + q] = v[sel[q]];
    }
    for (i = 0; i < n; ++i) uT[i] = u[i];

    free(md); free(mo); free(sd); free(so); free(wd); free(wo); free(W);
    free(fd); free(fo); free(tmp1); free(tmp2); free(tmp3); free(tmp4);
    free(u); free(v); free(rhs); free(rhs0); free(zeta); free(vprev);
    free(dg); free(lo); free(work);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Causal (lower-triangular Toeplitz) product, the block structure of        */
/* Props. 3-4: y[t] = sum_{s=0}^{t} c[t-s] x[s], t = 0..nt-1.                  */
/* ------------------------------------------------------------------------ */
void or_causal_conv(int nt, const double *c_, const double *x_, double *y_)
{
    const cplx *c = (const cplx *)c_, *x = (const cplx *)x_;
    cplx *y = (cplx *)y_;
    int t, s;
    for (t = 0; t < nt; ++t) {
        cplx acc = 0.0;
        for (s = 0; s <= t; ++s) acc += c[t - s] * x[s];
        y[t] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* The same march in extended precision (static V, linear ends).            */
/* ------------------------------------------------------------------------ */
/*
 * or_march_ext repeats or_march for a static potential (vkind 0) with every
 * intermediate quantity in C `long double` (x86-64: the 64-bit-significand
 * extended format, unit roundoff 5.4e-20; AArch64: IEEE binary128, 9.6e-35).
 * The inputs are the same binary64 values as for or_march (they define the
 * problem); the matrices of Eq. AvML, the Thomas solves, the S_0^2 history
 * b_n and the CN update are carried in long double, and the end traces and
 * u(T) are returned in long double.  It exists to decide, where a result
 * cancels (the flux 2 S-tilde v - l of an almost transparent condition), how
 * much of a difference between two binary64 computations is rounding of
 * either, and it is kept as literal as or_march: one Thomas solve per step.
 *
 * Arguments as for or_march (tc 0 Robin, 1 S_0^2, 2 weights wl / wr), except:
 * no potential kind, no nonlinear arguments, no selected nodes; va, vb (nt+1)
 * and uT (n) are arrays of `long double complex`.
 * Returns 0, or -(i+1) when pivot i of a step is exactly zero.
 */
typedef long double complex cplxl;

static int or_thomas_ext(int n, const cplxl *lo, const cplxl *dg, cplxl *x, cplxl *work)
{
    int i;
    cplxl piv = dg[0];
    if (piv == 0.0L) return -1;
    work[0] = (n > 1) ? lo[0] / piv : 0.0L;
    x[0] = x[0] / piv;
    for (i = 1; i < n; ++i) {
        piv = dg[i] - lo[i - 1] * work[i - 1];
        if (piv == 0.0L) return -(i + 1);
        work[i] = (i < n - 1) ? lo[i] / piv : 0.0L;
        x[i] = (x[i] - lo[i - 1] * x[i - 1]) / piv;
    }
    for (i = n - 2; i >= 0; --i) x[i] = x[i] - work[i] * x[i + 1];
    return 0;
}

int or_march_ext(int n, double h_, double dt_, int nt, const double *V, int tc,
                 double sig_re, double sig_im, double c2_re, double c2_im,
                 const double *beta, int tc_left, int tc_right, const double *u0_,
                 const double *l_, const double *r_, long double *va_, long double *vb_,
                 long double *uT_, const double *wl_, const double *wr_)
{
    const cplx *u0 = (const cplx *)u0_, *l = (const cplx *)l_, *r = (const cplx *)r_;
    const cplx *wl = (const cplx *)wl_, *wr = (const cplx *)wr_;
    cplxl *va = (cplxl *)va_, *vb = (cplxl *)vb_, *uT = (cplxl *)uT_;
    const long nw = nt + 1;
    const long double h = h_, dt = dt_;
    const cplxl I2dt = 2.0L * I / dt;
    const cplxl sigma = (long double)sig_re + I * (long double)sig_im;
    const cplxl c2 = (long double)c2_re + I * (long double)c2_im;
    const cplxl sigma0 = (tc == 0) ? sigma : c2 * (long double)beta[0];
    long double *md = calloc(n, sizeof(long double)), *mo = calloc(n, sizeof(long double));
    long double *sd = calloc(n, sizeof(long double)), *so = calloc(n, sizeof(long double));
    long double *wd = calloc(n, sizeof(long double)), *wo = calloc(n, sizeof(long double));
    cplxl *u = malloc(sizeof(cplxl) * n), *v = malloc(sizeof(cplxl) * n);
    cplxl *dg = malloc(sizeof(cplxl) * n), *lo = malloc(sizeof(cplxl) * n);
    cplxl *work = malloc(sizeof(cplxl) * n);
    int status = 0, i, t, e, s;

    /* P1 matrices of Eq. AvML, element by element (as or_p1_matrices). */
    for (e = 0; e < n - 1; ++e) {
        const long double We = V[e], Wf = V[e + 1];
        md[e] += h / 3.0L;
        md[e + 1] += h / 3.0L;
        mo[e] += h / 6.0L;
        sd[e] += 1.0L / h;
        sd[e + 1] += 1.0L / h;
        so[e] += -1.0L / h;
        wd[e] += h / 12.0L * (3.0L * We + Wf);
        wd[e + 1] += h / 12.0L * (We + 3.0L * Wf);
        wo[e] += h / 12.0L * (We + Wf);
    }
    for (i = 0; i < n; ++i) u[i] = (long double)creal(u0[i]) + I * (long double)cimag(u0[i]);
    va[0] = u[0];
    vb[0] = u[n - 1];

    for (t = 1; t <= nt && status == 0; ++t) {
        for (i = 0; i < n; ++i) dg[i] = I2dt * md[i] - sd[i] + wd[i];
        for (i = 0; i < n - 1; ++i) lo[i] = I2dt * mo[i] - so[i] + wo[i];
        if (tc_left)
            dg[0] -= (tc == 2) ? (long double)creal(wl[(long)t * nw + t])
                                     + I * (long double)cimag(wl[(long)t * nw + t])
                               : sigma0;
        if (tc_right)
            dg[n - 1] -= (tc == 2) ? (long double)creal(wr[(long)t * nw + t])
                                         + I * (long double)cimag(wr[(long)t * nw + t])
                                   : sigma0;
        /* (2i/dt) M u_{n-1} */
        for (i = 0; i < n; ++i) {
            cplxl acc = md[i] * u[i];
            if (i > 0) acc += mo[i - 1] * u[i - 1];
            if (i < n - 1) acc += mo[i] * u[i + 1];
            v[i] = I2dt * acc;
        }
        /* + b_n (history of the end trace), - Q^T (l_n, r_n)^T */
        if (tc == 1 && tc_left) {
            cplxl acc = 0.0L;
            for (s = 0; s < t; ++s) acc += (long double)beta[t - s] * va[s];
            v[0] += c2 * acc;
        }
        if (tc == 1 && tc_right) {
            cplxl acc = 0.0L;
            for (s = 0; s < t; ++s) acc += (long double)beta[t - s] * vb[s];
            v[n - 1] += c2 * acc;
        }
        if (tc == 2 && tc_left) {
            cplxl acc = 0.0L;
            for (s = 0; s < t; ++s)
                acc += ((long double)creal(wl[(long)t * nw + s])
                        + I * (long double)cimag(wl[(long)t * nw + s])) * va[s];
            v[0] += acc;
        }
        if (tc == 2 && tc_right) {
            cplxl acc = 0.0L;
            for (s = 0; s < t; ++s)
                acc += ((long double)creal(wr[(long)t * nw + s])
                        + I * (long double)cimag(wr[(long)t * nw + s])) * vb[s];
            v[n - 1] += acc;
        }
        if (tc_left && l)
            v[0] -= (long double)creal(l[t - 1]) + I * (long double)cimag(l[t - 1]);
        if (tc_right && r)
            v[n - 1] -= (long double)creal(r[t - 1]) + I * (long double)cimag(r[t - 1]);

        status = or_thomas_ext(n, lo, dg, v, work);
        for (i = 0; i < n; ++i) u[i] = 2.0L * v[i] - u[i];
        va[t] = v[0];
        vb[t] = v[n - 1];
    }
    for (i = 0; i < n; ++i) uT[i] = u[i];
    free(md); free(mo); free(sd); free(so); free(wd); free(wo);
    free(u); free(v); free(dg); free(lo); free(work);
    return status;
}
