/*
 * swr.h - C ABI of the GB300 Schwarz waveform relaxation (SWR) library.
 *
 * Method: Besse & Xing, "Schwarz waveform relaxation method for one dimensional
 * Schroedinger equation with general potential" (arXiv 1503.02564).  The library
 * solves  i u_t + u_xx + V u = 0  on (a0, b0) x (0, T) with homogeneous Neumann
 * ends (Eq. Schequ) by non-overlapping SWR: N subdomains, each advanced by a
 * Crank-Nicolson march with P1 finite elements (Eq. CNS_L / AvML, nonlinear
 * Eq. CNS_NL / AvMNL), coupled through transmission conditions written as
 * fluxes (Eq. TransmissionCondlocal, TransmisionCond).  The unknown of the outer
 * iteration is the interface vector g of Section 3.
 *
 * Conventions for every entry point
 *   - Complex arrays are interleaved (re, im) doubles: "cplx[n]" means 2n doubles.
 *   - Unless stated otherwise an array argument is a DEVICE pointer, borrowed for
 *     the duration of the call; the caller owns it.  The plan owns everything it
 *     allocates (factors, interface operator, Krylov workspace).
 *   - Work is enqueued on the plan's stream (the cudaStream_t given to swr_plan,
 *     passed as void*; NULL = legacy default stream).  Calls that report a scalar
 *     result to the host (swr_solve) synchronise that stream.
 *   - Every call returns an swr_status and never aborts the process.  Device-side
 *     faults of the numerics (zero pivot, non-finite values) are recorded in a
 *     device status word and reported by the next call that reads it.
 *
 * Interface vector layout (Section 3): g = (r_1; l_2, r_2; ...; l_N), 2N-2 blocks
 * of nt values; with 0-based subdomain j the flux r_j is block 2j (j <= N-2) and
 * l_j is block 2j-1 (j >= 1).  Entry n-1 of a block is the flux at t_n = n dt.
 */
#ifndef SWR_H
#define SWR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum swr_status {
    SWR_OK = 0,
    SWR_ERR_ARG = 1,            /* invalid argument or plan field                       */
    SWR_ERR_SINGULAR = 2,       /* zero or non-finite pivot in A - B (Props. 1-2 assume  */
                                /* A - B nonsingular)                                    */
    SWR_ERR_NOT_CONVERGED = 3,  /* iteration cap reached; outputs hold the last iterate  */
    SWR_ERR_NONFINITE = 4,      /* NaN/Inf in a residual or a march output               */
    SWR_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up                    */
    SWR_ERR_NOMEM = 6,          /* device allocation failed                              */
    SWR_ERR_CUDA = 7,           /* other CUDA runtime error                              */
    SWR_ERR_STATE = 8,          /* call order violated (e.g. solve before build)         */
    SWR_ERR_UNSUPPORTED = 9     /* combination not supported by the library              */
} swr_status;

/* Potential kinds (Eq. Schequ: V(t,x) or f(u)). */
enum { SWR_V_STATIC = 0, SWR_V_TIME = 1, SWR_V_NONLINEAR = 2 };
/* Transmission operators S-bar (Section 2.2): Robin S-bar v = p v (the paper's
 * S = -ip corresponds to p = -i p_paper); potential strategy of order 2, S_0^2:
 * S-bar v_n = c2 sum_{s=0}^{n} beta_{n-s} v_s, c2 = e^{-i pi/4} sqrt(2/dt),
 * beta_s = (-1)^s alpha_s the coefficients of sqrt((1-z)/(1+z)), v_0 = u_0 at
 * the end.  The s = n term enters the subdomain matrix (sigma0 = c2), the
 * history sum the end rows and the emitted fluxes.  S_0^2 with V(t,x) needs the
 * streamed per-step factors (swr_build_interface returns SWR_ERR_UNSUPPORTED
 * when they do not fit in half of the free device memory). */
enum { SWR_TC_ROBIN = 0, SWR_TC_S02 = 1, SWR_TC_S03 = 2, SWR_TC_S04 = 3, SWR_TC_S12 = 4,
       SWR_TC_S14 = 5 };
/* SWR_TC_S03, S04 (potential strategy, orders 3 and 4) and S12, S14 (gauge change
 * strategy, orders 2 and 4), Section 2.2, for SWR_V_STATIC only, with the NONE or
 * CAUSAL preconditioner.  At an end with node potential W and outward derivative
 * d_nW (central difference on the whole grid), with c2 = e^{-i pi/4} sqrt(2/dt):
 *   S03: S-bar v_n = sum_s [c2 beta_{n-s} - e^{i pi/4} sqrt(dt/2) (W/2) alpha_{n-s}] v_s
 *   S04: S03 - i (d_nW / 4) (dt/2) sum_s gamma_{n-s} v_s,  gamma = (1, 2, 2, ...)
 *   S12: c2 e^{i Wc_n} sum_s beta_{n-s} e^{-i Wc_s} v_s,  Wc_n = (n - 1/2) dt W, Wc_0 = 0
 *   S14: S12 - i (d_nW / 4) (dt/2) e^{i Wc_n} sum_s gamma_{n-s} e^{-i Wc_s} v_s.
 * The flux update applies the sum of the two subdomains' operators at an interface
 * (2 S-bar when they agree; for S04/S14 the d_nW terms cancel in the sum). */
/* Interface solvers: GMRES (Algorithms 2-3), fixed point on (I - L) g = d
 * (Algorithm 3 with the fixed point), classical iteration g <- R g with full
 * marches (Algorithm 1).  For SWR_V_NONLINEAR the interface operator R_nl is
 * nonlinear: FIXED_POINT runs g <- g - P^{-1}(g - R_nl g) with the plan's
 * preconditioner (Section 5), CLASSICAL runs g <- R_nl g, GMRES is rejected. */
enum { SWR_SOLVER_GMRES = 0, SWR_SOLVER_FIXED_POINT = 1, SWR_SOLVER_CLASSICAL = 2,
       SWR_SOLVER_CAUSAL = 3, SWR_SOLVER_BICGSTAB = 4 };
/* SWR_SOLVER_BICGSTAB (V(x), V(t,x)): right-preconditioned BiCGStab on (I - L) g = d,
 * the alternative Krylov method of Section 6 (Tables 6-7), same preconditioners and
 * true-residual stopping test as GMRES; iterations counts BiCGStab steps (two operator
 * applications each). */
/* SWR_SOLVER_CAUSAL (static V only): no Krylov iteration.  The blocks of L are
 * causal Toeplitz in time (Props. 3-4), so (I - L) g = d is solved by block
 * forward substitution in time, g = P^{-1} d with the CAUSAL preconditioner's
 * substitution (in its window form the same-step coupling of neighbouring
 * interfaces is solved exactly, so P = I - L to rounding), then refined,
 * g += P^{-1} (d - (I - L) g), while the true residual is >= tol_abs (at most
 * maxit substitutions; iterations counts them). */
/* Preconditioners for GMRES (right preconditioning):
 *   NONE;
 *   ZERO_POTENTIAL: P = I - L_0, the interface operator with V = 0 (Section 5);
 *   CAUSAL: P = I - L itself (V = V(x) only), whose blocks are causal Toeplitz
 *           (Props. 3-4) so that P^{-1} is a block forward substitution in time;
 *   MEAN_POTENTIAL: P = I - L_Vbar, the interface operator of the time-averaged
 *           potential Vbar(x) = mean_n V(t_n, x) (V0 for NONLINEAR): the
 *           zero-potential construction of Section 5 keeping the static part of V,
 *           for potentials too strong for L_0. */
enum { SWR_PC_NONE = 0, SWR_PC_ZERO_POTENTIAL = 1, SWR_PC_CAUSAL = 2, SWR_PC_MEAN_POTENTIAL = 3 };

typedef struct swr_desc {
    int32_t nx;                 /* P1 nodes on (a0, b0), nx >= 3                       */
    double a0, b0;              /* domain; h = (b0 - a0)/(nx - 1)                      */
    int32_t nt;                 /* time steps, T = nt * dt                             */
    double dt;
    int32_t nsub;               /* N >= 2 subdomains                                   */
    const int32_t *node_off;    /* HOST, nsub+1 increasing offsets, off[0] = 0,        */
                                /* off[N] = nx-1; subdomain j = nodes off[j]..off[j+1] */
                                /* (interface nodes are shared); each holds >= 3 nodes */
                                /* NULL: equal partition, the first (nx-1) mod N get   */
                                /* one extra element                                  */
    int32_t vkind;              /* SWR_V_*                                             */
    int32_t tc;                 /* SWR_TC_*                                            */
    double tc_re, tc_im;        /* Robin parameter p (S-bar v = p v); unused by S_0^2  */
    int32_t solver;             /* SWR_SOLVER_*                                        */
    int32_t restart;            /* GMRES restart length m (default 30 if <= 0, at most 200)      */
    int32_t maxit;              /* iteration cap (default 2000 if <= 0)                */
    double tol_abs;             /* stop when ||d - (I-L) g||_2 < tol_abs (default 1e-10) */
    int32_t precond;            /* SWR_PC_*                                            */
    int32_t nl_maxit;           /* nonlinear inner fixed point cap (default 50)        */
    double nl_tol;              /* inner stop: max|dz| <= nl_tol max(1,max|z|) (1e-13) */
    double nl_coef;             /* f(u) = nl_coef |u|^2 (default 1 if 0)               */
    int32_t pc_sweeps;          /* block-Jacobi sweeps resolving the same-step coupling  */
                                /* of neighbouring interfaces in the causal substitution */
                                /* (CAUSAL / ZERO_POTENTIAL preconditioners), 0..16;    */
                                /* < 0: chosen by the library (CAUSAL, static V, after  */
                                /* the first build: the exact window form when the       */
                                /* corner couplings decay within 8 interfaces, see       */
                                /* swr_stats.causal_window; else 1 sweep)               */
} swr_desc;

/* Execution choices of a plan (no counterpart in the paper: they change how the
 * library runs the method, never what it computes beyond rounding).  Zero-filled
 * means "library default" for every field; swr_tuning_defaults writes the defaults
 * explicitly.  A plan takes its copy at creation (swr_plan_ex / swr_plan_batch_ex);
 * swr_plan / swr_plan_batch use the defaults. */
typedef struct swr_tuning {
    int32_t chunk_L;            /* chunk length of the partitioned marches: 0 (default)  */
                                /* chosen per launch; 4, 8, 12 or 16 fixed; the         */
                                /* nonlinear march takes 2, 4 or 8 (2: nonlinear only)  */
    int32_t autotune;           /* launch shapes: 0 (default) measured by probe marches  */
                                /* at the first build; -1 the modelled shape            */
    int32_t toeplitz_fft;       /* (I - L) x: 0 (default) FFT convolution for           */
                                /* 16 <= nt <= 2048; -1 direct causal sums              */
    int32_t superpose;          /* u(T), static V: 0 (default) by superposition of the   */
                                /* recorded impulse responses when they fit; -1 final   */
                                /* march                                                */
    int32_t long_march;         /* 0 (default): the grid-wide march only for subdomains */
                                /* longer than a cluster holds; 1 for every V(x) plan   */
    int32_t graph;              /* builds after the first: 0 (default) replayed as a     */
                                /* CUDA graph; -1 launched directly                     */
    int32_t tdep_precomp;       /* V(t,x): 0 (default) every step's factors computed once */
                                /* per build when they fit; -1 refactorised per step    */
    int32_t two_level;          /* systems spread over a cluster: 0 (default) two-level  */
                                /* separator solve (one cluster barrier per step) when   */
                                /* a system has <= 993 separators (the nonlinear         */
                                /* gradient's monodomain: <= 8161); -1 cluster-wide PCR  */
    int32_t debug;              /* 1: failing CUDA calls (2: also the launch-shape      */
                                /* probes) reported on stderr; 0 (default) silent        */
    int32_t history_fft;        /* causal substitution (CAUSAL preconditioner, direct   */
                                /* solver), single-instance plans with nt >= 64 and no   */
                                /* sweeps: 0 (default) the history sums of lags > 3 by   */
                                /* blocks of 32 steps, the far blocks as 64-point FFT    */
                                /* convolutions; -1 direct sums                         */
} swr_tuning;

typedef struct swr_info {
    int32_t iterations;         /* outer iterations (GMRES steps or fixed-point sweeps) */
    int32_t restarts;
    double residual;            /* final TRUE residual ||d - (I-L) g||_2                */
    double residual0;           /* ||d - (I-L) g0||_2                                   */
    double interface_jump;      /* max_j max_n |v_j(b_j) - v_{j+1}(a_{j+1})| in the     */
                                /* final march (diagnostic of the converged solution)  */
    double t_build_ms;          /* swr_build_interface time (device events)            */
    double t_solve_ms;          /* interface solve time                                 */
    double t_final_ms;          /* final march time                                     */
    int64_t march_point_steps;  /* point-steps marched inside swr_solve                */
} swr_info;

/* Cumulative device-time counters of a plan (CUDA events around each launch of
 * the named kernels on the plan's stream). */
typedef struct swr_stats {
    int64_t march_launches;     /* subdomain march kernel launches                     */
    int64_t march_point_steps;  /* nodes x time steps marched by those launches         */
    double march_ms;            /* summed device time of those launches                */
    int64_t toeplitz_launches;  /* (I - L) x applies from the Toeplitz first columns     */
    double toeplitz_ms;
    int64_t precond_calls;      /* block forward substitutions P^{-1} y                 */
    double precond_ms;
    int32_t march_variant;      /* kernel of the interface marches R g: 0 constant
                                 * matrix, 1 V(t,x) refactorised inside the march,
                                 * 2 nonlinear, 3 V(t,x) with every step's factors
                                 * computed once per build and streamed from HBM
                                 * (-1 before the first build)                          */
    int64_t march_factor_bytes_per_step; /* variant 3: factor bytes one R march reads
                                 * per time step (all subdomains); 0 otherwise           */
    int64_t march_point_iterations; /* nonlinear marches (swr_adjoint's included): nodes
                                 * x inner fixed-point iterations, summed over steps     */
    int64_t nl_march_launches;  /* of the march launches above, the nonlinear ones      */
    double nl_march_ms;         /* and their summed device time                         */
    int32_t superposed;         /* 1: swr_solve forms u(T) by superposition of the build
                                 * marches' recorded states (static V, Robin, enough free
                                 * memory, tuning.superpose >= 0) instead of a final march */
    int32_t toeplitz_fft_length; /* transform length M of the FFT Toeplitz applies (the
                                 * power of two >= 2 nt - 1, for 16 <= nt and M <= 4096,
                                 * tuning.toeplitz_fft >= 0); 0: direct causal sums      */
    int32_t causal_sweeps;      /* block-Jacobi sweeps of the causal substitution in use */
    int32_t causal_window;      /* H >= 1: the substitution solves the same-step coupling
                                 * exactly over a window of H interfaces each side; 0: sweeps */
    int64_t two_level_launches; /* march launches that took the two-level separator solve
                                 * (a system spread over a cluster)                     */
} swr_stats;

typedef struct swr_plan_s *swr_plan_t;

/* Validate d, copy the partition and allocate the plan on the current device.
 * stream: cudaStream_t (as void*) on which all later work of this plan runs.
 * Subdomains up to 69632 nodes are marched by thread-block clusters; a V(x) plan
 * with a longer subdomain is marched by the whole grid (one cooperative launch, the
 * state in device memory; swr_tuning.long_march = 1 forces it); V(t,x), nonlinear and batched
 * plans with such a subdomain return SWR_ERR_UNSUPPORTED.
 * Errors: SWR_ERR_ARG (bad field), SWR_ERR_UNSUPPORTED, SWR_ERR_NOMEM, SWR_ERR_CUDA.
 * *out is NULL on failure. */
swr_status swr_plan(const swr_desc *d, swr_plan_t *out, void *stream);

/* swr_plan with explicit execution choices (tuning may be NULL: the defaults).
 * Errors as swr_plan, and SWR_ERR_ARG for a tuning field out of range. */
swr_status swr_plan_ex(const swr_desc *d, const swr_tuning *tuning, swr_plan_t *out,
                       void *stream);

/* Fill *t with the library defaults (host-only, no device work). */
void swr_tuning_defaults(swr_tuning *t);

/* A batch of independent problem instances in one plan (no counterpart in the
 * paper, which solves one problem at a time).  descs[0..count-1] each give an
 * instance's grid (nx, a0, b0), step count nt and partition (nsub, node_off);
 * all other fields, the grid step h = (b0 - a0)/(nx - 1) (to 1e-12 relative)
 * and dt must agree (SWR_ERR_ARG otherwise), and vkind must be SWR_V_STATIC
 * (SWR_ERR_UNSUPPORTED otherwise).  Every launch of the plan (marches,
 * Toeplitz applies, GMRES vector kernels) covers all instances at once; the
 * causal substitution runs as few cooperative launches as hold whole instances.
 * The plan's arrays are the instances' arrays concatenated in order: V, u0, uT
 * (sum of nx), interface vectors (sum of (2 nsub - 2) nt, instance by
 * instance, blocks as for one instance) and first columns (sum of 4 nsub nt).
 * GMRES runs on the concatenated (block-diagonal) system, so its stopping test
 * bounds every instance's residual.  swr_adjoint is not available for batches. */
swr_status swr_plan_batch(const swr_desc *descs, int32_t count, swr_plan_t *out, void *stream);

/* swr_plan_batch with explicit execution choices (tuning may be NULL). */
swr_status swr_plan_batch_ex(const swr_desc *descs, int32_t count, const swr_tuning *tuning,
                             swr_plan_t *out, void *stream);

/* Assemble and factor the subdomain systems A_j - B_j (Eq. AvML) for potential
 * V and build the interface problem (Section 4.1):
 *   SWR_V_STATIC:    d = R 0 and the first columns of X^{j,1..4} (Props. 3-4),
 *                    i.e. L and d of Eq. chp1_ILgd explicitly (Algorithm 3);
 *   SWR_V_TIME:      d = R 0, and L_0 (L_Vbar) when precond == ZERO_POTENTIAL
 *                    (MEAN_POTENTIAL);
 *   SWR_V_NONLINEAR: L_0 (L_V0) when precond == ZERO_POTENTIAL (MEAN_POTENTIAL).
 * V:  double[nx] (STATIC; V0 for NONLINEAR) or double[(nt+1) * nx], row n = V(t_n, .)
 *     (TIME).  Copied into the plan.
 * u0: cplx[nx] initial value.  Copied into the plan.
 * Errors: SWR_ERR_SINGULAR (a pivot of A - B vanished), SWR_ERR_ARG, SWR_ERR_CUDA. */
swr_status swr_build_interface(swr_plan_t p, const double *V, const double *u0);

/* Solve the interface problem with the plan's solver, then form u(T) (last step
 * of Algorithms 1-3).  By default a final march of every subdomain with the
 * converged fluxes.  Static V with Robin transmission (p != 0): the march is
 * linear and time invariant, so swr_build_interface records the full states of
 * its impulse-driven marches (2 nt n_j complex per subdomain, when that takes at
 * most a quarter of the free device memory and tuning.superpose >= 0) and u(T)
 * is their superposition weighted by the converged fluxes plus the zero-flux
 * march's final state; info->interface_jump then comes from the final residual
 * (v_j(b_j) - v_{j+1}(a_{j+1}) = ((R g - g)[l_{j+1}] - (R g - g)[r_j]) / 2p).
 * SWR_V_NONLINEAR with Robin or Neumann ends (single instance): after a converged
 * solve the final march also records v_n of every step (nt x nx complex, allocated
 * once when that takes at most 1/8 of the free device memory, and kept for
 * swr_adjoint), so that a following swr_adjoint with one checkpoint segment runs only
 * the adjoint march.
 * g:    cplx[(2N-2) * nt]; on entry the initial guess g0 (ignored if
 *       g_is_initial == 0, then g0 = 0), on exit the converged interface vector.
 *       May be NULL (then g0 = 0 and the result is not returned).
 * uT:   cplx[nx] u at the final time; the interface node takes the left
 *       subdomain's value.  May be NULL.
 * info: HOST, may be NULL.
 * Returns SWR_ERR_NOT_CONVERGED when the cap is reached (outputs hold the last
 * iterate, info filled), SWR_ERR_STATE before swr_build_interface. */
swr_status swr_solve(swr_plan_t p, double *g, int32_t g_is_initial, double *uT,
                     swr_info *info);

/* One application of the interface operator R (Eq. interfacepbR): march every
 * subdomain with the fluxes g_in (and the plan's u0), then form the new fluxes
 * by Eq. TransmisionCond into g_out.  Both cplx[(2N-2) * nt], distinct buffers.
 * Requires swr_build_interface (it holds the factors and u0). */
swr_status swr_apply_R(swr_plan_t p, const double *g_in, double *g_out);

/* y = (I - L) x from the Toeplitz first columns (Eq. chp1_ILgd, Props. 3-4).
 * SWR_V_STATIC only.  x, y: cplx[(2N-2) * nt], distinct buffers. */
swr_status swr_apply_interface(swr_plan_t p, const double *x, double *y);

/* Copy the built interface problem out: d (cplx[(2N-2) * nt]) and the first
 * columns cols (cplx[4 N nt], column p-1 of subdomain j at (4j + p - 1) * nt,
 * zero where the block does not exist).  Either may be NULL. */
swr_status swr_get_interface(swr_plan_t p, double *d, double *cols);

/* x = P^{-1} y for the plan's preconditioner (ZERO_POTENTIAL or CAUSAL).
 * x, y: cplx[(2N-2) * nt], distinct buffers. */
swr_status swr_apply_precond(swr_plan_t p, const double *y, double *x);

/* Final-time misfit J = (u_T - u_target)^H M (u_T - u_target), M the P1 mass
 * matrix of the whole grid (not a passage of the paper: the objective of the
 * gradient below).  uT, u_target: cplx[nx] (device); ubar: cplx[nx] (device,
 * may be NULL) receives the M-weighted cotangent 2 (u_T - u_target), i.e.
 * dJ = Re(ubar^H M du_T); *J (host) receives J.  Synchronises the stream. */
swr_status swr_misfit(swr_plan_t p, const double *uT, const double *u_target, double *ubar,
                      double *J);

/* Gradient dJ/dV(x) of a final-time objective J through the converged SWR
 * solution (no counterpart in the paper, which has no adjoint).  Needs, after a
 * successful swr_solve (SWR_ERR_STATE otherwise), a single-instance plan with
 *   SWR_V_STATIC, Robin or S_0^2 transmission, any solver:   dJ/dV;
 *   SWR_V_TIME, Robin or S_0^2, every step's factors stored (swr_stats.march_variant
 *               3) with chunks of at most 8 nodes:          dJ/dV(t_m, x), m = 0..nt;
 *   SWR_V_NONLINEAR (any transmission condition and solver):  dJ/dV0;
 * SWR_ERR_UNSUPPORTED for other plans.
 *   dJ_duT:     cplx[nx] (device), the M-weighted cotangent ubar of J at u(T):
 *               dJ = Re(ubar^H M du_T) (swr_misfit returns it for the misfit);
 *   dJ_dV:      double[nx] (device), overwritten with dJ/dV_k for the nodal V;
 *               SWR_V_TIME: double[(nt + 1) nx], row m = dJ/dV(t_m, .) (the layout of V);
 *   ckpt_every: checkpoint interval K in time steps (<= 0: every step recorded in one
 *               segment when nt x nx complex take at most 1/8 of the free device memory
 *               or are already allocated, else 50).
 * Method (static V): the discrete adjoint of the Crank-Nicolson march,
 * conjugated and scaled, is the same march run from (dt/2i) conj(ubar); it is
 * solved by SWR on the plan's own interface problem (same Toeplitz columns and
 * preconditioner), then forward segments of K steps are recomputed from
 * checkpoints of u and the adjoint march over the mirrored steps accumulates
 *   dJ/dV_k = -2 Re sum_n (v^adj_{N-n+1})^T (dM_V/dV_k) v_n.
 * With S_0^2 the segment marches carry the ends' trace histories over the whole
 * time axis.  Method (V(t,x)): the adjoint march takes the step matrices A_N, ...,
 * A_1 in that order, so its SWR problem is the forward one with the time axis
 * reversed, solved matrix-free (Algorithm 2) with the plan's time-invariant
 * preconditioner; adjoint step n gives dJ/dW_n = -2 Re (v^adj)^T (dM_W/dW) v_n, which
 * enters dJ/dV(t_n) and dJ/dV(t_{n-1}) with weight 1/2 each (W_n = (V_n + V_{n-1})/2).
 * Method (nonlinear, Eq. CNS_NL with f = c|v|^2): the discrete adjoint of the
 * monodomain scheme, which the converged SWR solution reproduces.  Each adjoint
 * step solves the step's derivative, A0 w + M_{c|v|^2} w + 2c conj(v) .
 * Re(v^T (dM_W/dW_k) w) = (2i/dt) M z, by the march's inner fixed point about the
 * recorded forward v_n (relative test nl_tol, cap nl_maxit: SWR_ERR_NOT_CONVERGED
 * when reached), z <- 2 w - z, and dJ/dV0_k = -2 Re sum_n w_n^T (dM_V/dV_k) v_n.
 * With one segment (K = nt) the recorded v_n are the last swr_solve's final march
 * when it recorded them (see swr_solve: the converged SWR trajectory, equal to the
 * monodomain one to the solve's tolerance); otherwise, and with checkpoints, the
 * monodomain forward march recomputes them.
 * The whole grid is one system on a thread-block cluster (at most 16 CTAs of 256
 * threads: nx <= 20476, or 36856 with 8-node chunks; SWR_ERR_UNSUPPORTED above).
 * Device memory: (ceil(nt/K) + K + 5) nx complex plus two interface vectors.
 * Synchronises the stream. */
swr_status swr_adjoint(swr_plan_t p, const double *dJ_duT, double *dJ_dV,
                       int32_t ckpt_every);

/* Free everything the plan owns (after synchronising its stream).  NULL is a no-op. */
void swr_destroy(swr_plan_t p);

/* Copy the plan's cumulative counters into *out (host); reset them if reset != 0.
 * Synchronises the plan's stream. */
swr_status swr_get_stats(swr_plan_t p, swr_stats *out, int32_t reset);

/* x = (I - L)^{-1} y by the causal block forward substitution of the CAUSAL
 * preconditioner, WITHOUT allocating device memory.  The paper has no
 * counterpart: this is a deployment variant of swr_apply_precond.
 *
 * For callers that cannot allocate: applications that reserve all device memory
 * up front in their own pool, or latency-critical loops that cannot afford the
 * device-wide synchronisation cudaMalloc/cudaFree imply.  The caller provides
 * inputs and outputs; the substitution's working arrays live in a fixed
 * library-owned device array (about 260 KB, held on every GPU that loads the
 * library until the process exits).
 *   nsub:   N, 2 <= N <= 1024 (larger N: SWR_ERR_ARG; the array is sized for 1024)
 *   nt:     time steps, >= 1
 *   sweeps: block-Jacobi sweeps for the same-step coupling of neighbouring
 *           interfaces, 0..16 (swr_desc.pc_sweeps of a plan)
 *   cols:   cplx[4 N nt] Toeplitz first columns as returned by swr_get_interface
 *   y, x:   cplx[(2N-2) nt], distinct; x is overwritten
 *   stream: cudaStream_t (as void*) the work is enqueued on; the call
 *           synchronises it at the end to report a bounded-wait timeout.
 * The first call on a device looks up the device address of the library array
 * (cudaGetSymbolAddress, with that device current); make that first call before
 * any stream capture.  The lookup is repeated only when the device's context has
 * changed (e.g. after cudaDeviceReset).  Every call copies the status word to the
 * host and synchronises the stream before it returns.  All calls share the one
 * array: calls that overlap on the
 * GPU (other streams, other threads) race and give wrong results.  Each call
 * clears the array's progress counters and status word; the other entries are
 * written before they are read.
 * Errors: SWR_ERR_ARG (sizes, sweeps, NULL or aliased pointers),
 * SWR_ERR_UNSUPPORTED (device ordinal >= 64, or more interfaces than can be
 * resident at once), SWR_ERR_TIMEOUT (a bounded wait of the substitution gave
 * up; x is invalid), SWR_ERR_CUDA. */
swr_status swr_causal_solve_noalloc(int32_t nsub, int32_t nt, int32_t sweeps,
                                    const double *cols, const double *y, double *x,
                                    void *stream);

/* FP64 throughput probe: the denominator of the marches' roofline (no counterpart
 * in the paper; the march is FP64-bound on this part and its peak rate is measured,
 * not taken from a datasheet).  One timed launch of `blocks` CTAs of `threads`
 * threads (32..256, a multiple of 32) on stream (cudaStream_t as void*):
 *   kind 0: DFMA, each thread `iters` rounds of 8 independent fused multiply-add
 *           chains (2 flops each);
 *   kind 1: DMMA, each warp `iters` rounds of 4 independent
 *           mma.sync.aligned.m8n8k4 f64 products (512 flops each);
 *   kind 2: both in every round of every warp, equal flops (the 8 chains and one
 *           m8n8k4 product: 512 flops each per warp).
 * sink: double[blocks * threads] (device) receives the chains' values; *flops
 * (host) the flops executed; *ms (host) the launch's device time from CUDA events
 * on the stream.  Synchronises the stream.
 * Errors: SWR_ERR_ARG (kind, sizes, NULL pointers), SWR_ERR_CUDA. */
swr_status swr_fp64_peak(int32_t kind, int64_t iters, int32_t blocks, int32_t threads,
                         double *sink, double *flops, float *ms, void *stream);

/* TEST HOOK of the bounded device waits (no counterpart in the paper; off by
 * default, for failure-detection tests).  The causal substitution (CAUSAL
 * preconditioner, SWR_SOLVER_CAUSAL, swr_causal_solve_noalloc) hands values between
 * the CTAs of one cooperative launch through progress counters, and every wait on a
 * counter gives up after a bounded number of polls (about 1-2 s), raising
 * SWR_ERR_TIMEOUT.  On the current device this sets
 *   max_polls: the poll limit of those waits (<= 0: the default);
 *   withhold:  an interface (global index) whose CTA never publishes its progress,
 *              so that its neighbours' waits run out (< 0: none, the default).
 * Affects launches enqueued after the call; restore with (0, -1).
 * Errors: SWR_ERR_CUDA. */
swr_status swr_test_wait_hook(int64_t max_polls, int32_t withhold);

/* Number of CUDA kernels this library has launched in this process, over all
 * plans (a monotonically increasing counter; host-only, no device work). */
int64_t swr_kernel_launch_count(void);

/* Static, human-readable name of a status code. */
const char *swr_status_string(swr_status s);

#ifdef __cplusplus
}
#endif
#endif /* SWR_H */
