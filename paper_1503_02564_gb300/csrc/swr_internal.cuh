// Internal declarations shared by the CUDA translation units of libswr.
// Complex FP64 values are double2 (x = re, y = im).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/swr.h"

// ---------------------------------------------------------------------------
// complex helpers (each complex multiply-add is 4 FP64 pipe operations)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ double2 cmk(double re, double im) { return make_double2(re, im); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// c + a*b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(-a.y, b.y, fma(a.x, b.x, c.x)), fma(a.y, b.x, fma(a.x, b.y, c.y)));
}
// c - a*b
__device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.y, b.y, fma(-a.x, b.x, c.x)), fma(-a.y, b.x, fma(-a.x, b.y, c.y)));
}
// conj(a)*b
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ double2 crcp(double2 a) {
    double s = 1.0 / fma(a.x, a.x, a.y * a.y);
    return make_double2(a.x * s, -a.y * s);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ bool cfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }
// c ? a : b as one selp per component.  Picking one element of an unrolled
// register array under a runtime condition (the last interior node of a chunk)
// is otherwise rewritten by the compiler into an indexed read, which moves the
// whole array to local memory.
__device__ __forceinline__ double2 csel(bool c, double2 a, double2 b) {
    double2 r;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %4, 0;\n\t"
        "selp.f64 %0, %2, %5, q;\n\tselp.f64 %1, %3, %6, q;\n\t}"
        : "=d"(r.x), "=d"(r.y)
        : "d"(a.x), "d"(a.y), "r"((unsigned)c), "d"(b.x), "d"(b.y));
    return r;
}

// S_0^2 history sum of one end, sum_{s=0}^{t-1} beta_{t-s} hist[s], by one full
// warp: lanes strided over s, then a fixed butterfly (lane 0's value is the same
// from run to run).
__device__ __forceinline__ double2 s02_history(const double* __restrict__ beta,
                                               const double2* hist, int t, int lane) {
    double2 acc = make_double2(0.0, 0.0);
    for (int s = lane; s < t; s += 32) {
        const double b = beta[t - s];
        const double2 v = hist[s];
        acc.x = fma(b, v.x, acc.x);
        acc.y = fma(b, v.y, acc.y);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    return acc;
}

// The same for a transmission operator with a complex kernel per end (S_0^3, S_0^4,
// S_1^2, S_1^4 for V(x)): o1 = sum_{s<t} k1[t-s] hist[s] (the end's own operator, for
// its boundary row) and o2 = sum_{s<t} k2[t-s] hist[s] (the flux update's operator).
__device__ __forceinline__ void conv_history2(const double2* __restrict__ k1,
                                              const double2* __restrict__ k2,
                                              const double2* hist, int t, int lane,
                                              double2& o1, double2& o2) {
    double2 a1 = make_double2(0.0, 0.0), a2 = a1;
    for (int s = lane; s < t; s += 32) {
        const double2 v = hist[s];
        const double2 c1 = k1[t - s], c2 = k2[t - s];
        a1.x = fma(c1.x, v.x, fma(-c1.y, v.y, a1.x));
        a1.y = fma(c1.x, v.y, fma(c1.y, v.x, a1.y));
        a2.x = fma(c2.x, v.x, fma(-c2.y, v.y, a2.x));
        a2.y = fma(c2.x, v.y, fma(c2.y, v.x, a2.y));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a1.x += __shfl_xor_sync(0xffffffffu, a1.x, off);
        a1.y += __shfl_xor_sync(0xffffffffu, a1.y, off);
        a2.x += __shfl_xor_sync(0xffffffffu, a2.x, off);
        a2.y += __shfl_xor_sync(0xffffffffu, a2.y, off);
    }
    o1 = a1;
    o2 = a2;
}

// ---------------------------------------------------------------------------
// device status word bits
// ---------------------------------------------------------------------------
enum : int {
    ST_SINGULAR = 1,
    ST_NONFINITE = 2,
    ST_TIMEOUT = 4,
    ST_NL_NOCONV = 8,
};

// ---------------------------------------------------------------------------
// March systems.  One "system" is one right-hand side of one subdomain:
// its u0 (given or zero) and its flux inputs (from an interface vector, a unit
// impulse at t_1, or zero).  The march emits the new fluxes of Eq. TransmisionCond.
// ---------------------------------------------------------------------------
enum : int {
    SYS_ZERO_U0 = 1,     // start from u0 = 0
    SYS_IMP_L = 2,       // l_{j,1} = 1, other l = 0
    SYS_IMP_R = 4,       // r_{j,1} = 1, other r = 0
    SYS_WRITE_UT = 8,    // write u(T) into the nodal output
    SYS_TRACE = 16,      // write v_n at both ends into the trace buffer
    // record states for u(T) by superposition (a.urec set; local node order):
    SYS_REC_U = 32,      // u after every step t at urec[rec + (t-1) n_j + node]
    SYS_REC_LAST = 64,   // u after the system's last step at urec[rec + node]
};

struct MarchSys {
    int sub;             // subdomain index
    int flags;           // SYS_*
    int nt;              // time steps of this system (its problem instance)
    int in_l, in_r;      // offset (complex entries) in gin of l_j / r_j at step 1 (or -1)
    int out_a, out_b;    // offset in gout of -l + 2 S v(a) / -r + 2 S v(b) at step 1 (or -1)
    long long rec;       // SYS_REC_*: offset (complex entries) of its states in urec
};

// Chunked (partitioned) factorisation of the subdomain matrices for one chunk
// length LMAX.  Subdomain j, chunk p (0 <= p < P), separators 0..P.
struct FactorSet {
    int L = 0;           // LMAX (template parameter of the march kernel)
    int P = 0;           // chunks per subdomain (padded to the maximum)
    int levels = 0;      // PCR levels over P+1 separators
    int* sub_P = nullptr;          // [N]   real chunks of subdomain j
    int* sep_pos = nullptr;        // [N][P+1] local node index of separator p
    unsigned char* clen = nullptr; // [N][P] interior nodes of chunk p (0 = dummy)
    double2* fac = nullptr;        // [N][L][4][P]  (q, c, a, b) per interior node
    double2* tips = nullptr;       // [N][P][4]     (a_first, b_first, a_last, b_last)
    double2* sep = nullptr;        // [N][3][P+1]   (E_left, E_right, 1/delta)
    double2* pcr = nullptr;        // [N][levels][2][P+1] (alpha, gamma)
    double2* red = nullptr;        // [N][6][P+1]   scratch for the PCR coefficient run
    // Per-step factorisations (V(t,x) tabulated, Eq. AvML with W at t_{n-1/2}):
    // fac, sep and pcr hold nsteps consecutive copies, step n-1 at n-1 times the
    // stride; tips, red and the assembled dg/od are scratch for a batch of steps.
    int nsteps = 1, batch = 1;
    long long fstride = 0, sstride = 0, pstride = 0;   // elements per step (0: one set)
    double2* dgb = nullptr;        // [batch][ldd] assembled diagonal (nsteps > 1)
    double2* odb = nullptr;        // [batch][ldd] assembled coupling
    long long ldd = 0;
    // Two-level separator solve for systems spread over a cluster (constant matrix,
    // P < kTlMaxSep): separators in warp blocks of 32, lane 0 of every block (and the
    // system's last separator) a super-separator, lanes 1..31 a super-chunk solved by
    // PCR with warp shuffles; the super-separators form a tridiagonal reduced system
    // of at most 32 unknowns, solved by one warp (tl_rs = 32, tl_rl = 5).  On request
    // (swr_launch_factor_tl with wide) up to kTlMaxSepWide separators: the reduced
    // system then has up to tl_rs = 256 unknowns, solved by PCR over a whole CTA
    // (the nonlinear march only).  Layout, per subdomain:
    //   tl_pcr  [N][5][2][P+1]  super-chunk PCR coefficients (alpha, gamma), zero off it
    //   tl_aux  [N][3][P+1]     1/delta after the last level, spikes a (left), b (right)
    //   tl_red  [N][2 tl_rl + 3][tl_rs]  reduced system: tl_rl levels of (alpha, gamma),
    //                           1/delta, and the weights of y_last(q-1), y_first(q) in
    //                           its right-hand side
    double2* tl_pcr = nullptr;
    double2* tl_aux = nullptr;
    double2* tl_red = nullptr;
    int tl_rs = 32, tl_rl = 5;
    bool tl_ok = false;
};
constexpr int kTlMaxSep = 993;        // P + 1 <= 993: at most 32 super-separators
constexpr int kTlMaxSepWide = 8161;   // P + 1 <= 8161: at most 256 super-separators

struct MarchArgs {
    int nt, P, levels, C, G, T, nsys;
    const MarchSys* sys;
    const int* sub_n;     // nodes of subdomain j
    const int* sub_goff;  // global index of its first node
    const int* sub_tc;    // bit0: left end carries a transmission condition, bit1: right
    const int* sub_P;
    const int* sep_pos;
    const unsigned char* clen;
    const double2* fac;
    const double2* sep;
    const double2* pcr;
    const double2* u0;    // nodal initial value (global)
    const double2* gin;   // interface vector input (blocks of nt)
    double2* gout;        // output blocks
    double2* uT;          // nodal output
    double2* trace;       // [nsys][2][nt]
    double2* urec;        // states of the SYS_REC_* systems (NULL: none recorded)
    // Transmission operators with a kernel per end (S_0^3, S_0^4, S_1^2, S_1^4; NULL:
    // Robin or S_0^2 from the scalars below).  End e = 2 sub + side:
    //   kap[e kstride + m]:  the end's own operator, S-bar v_n = sum_s kap[n-s] h_s
    //                        (kap[0] is its boundary matrix entry);
    //   kout[e kstride + m]: the flux update's operator (the two sides' sum);
    //   rho[e]: h_0 = rho v_0 (the gauge strategy's phase at s = 0), h_s = v_s.
    const double2* kap;
    const double2* kout;
    const double2* rho;
    int kstride;
    long long fstride, sstride, pstride;   // per-step factor strides (0: constant matrix)
    int stage;            // staging of streamed factors in shared memory (0, 1, 2)
    // Ragged packing (C == 1): CTA b holds the systems rag[rag_start[b] .. rag_start[b+1])
    // as (system index, first thread) pairs, each with exactly P_j + 1 threads and no
    // padding; NULL: G systems of P + 1 threads per CTA.
    const int* rag_start;
    const int2* rag;
    // A launch may march a segment of the time axis: its step t is step t0 + t of the
    // flux blocks, whose stride is gstride (the whole problem's nt).
    int t0;
    long long gstride;
    // Adjoint support (segment marches of the gradient):
    //   record mode: v of every step into vrec[(t-1) * nxrec + global node];
    //   gradient mode: with x = this march's v and y = vfwd[(nt - t) * nxrec + node],
    //   accumulate Re x^T (dM_W/dW_k) y per node k into gint (interior nodes of a
    //   chunk), gl (a separator, from the element on its right) and gr (a separator,
    //   from the element on its left); h12 = h / 12.
    long long nxrec;
    double2* vrec;
    const double2* vfwd;
    double* gint;
    double* gl;
    double* gr;
    double h12;
    // S_0^2 transmission condition (Section 2.2): S-bar v_n = c2 sum_{s<=n} beta_{n-s} v_s.
    // The current-step term sits in the matrix (sigma0 = c2 beta_0) and in two_sigma;
    // the history b_n = c2 sum_{s<n} beta_{n-s} v_s enters the end rows and the fluxes.
    int s02;
    const double* beta;   // [nt+1]
    double2* hist;        // [nsys][2][hstride] end traces v_0..v_nt (v_0 = u0 at the end)
    int hstride;          // entries per trace (0: nt + 1)
    int ht0;              // absolute step before this launch's step 1: a segment march
                          // continues the traces that earlier segments wrote (0: v_0 = u0)
    double2 c2_ik;        // c2 / (i kappa)
    double2 two_c2;       // 2 c2
    double2 two_sigma;    // 2 p (Robin): 2 S-tilde v = 2 p v
    double2 inv_ik;       // 1/(i kappa), kappa = (2/dt)(h/6): the system is scaled by it
    int* status;
    // two-level separator solve of cluster-spread systems (FactorSet.tl_*; NULL: off)
    const double2* tl_pcr;
    const double2* tl_aux;
    const double2* tl_red;
    int tl_rs, tl_rl;     // reduced system: stride (32, or up to 256 wide) and PCR levels
    int two_level;        // 0: keep the cluster-wide PCR even when the data exists
    // per-step factors (V(t,x)): index of the factor set of this launch's step 1, and
    // frev != 0 to walk them backwards (the adjoint's time-reversed march)
    int fstep0;
    int frev;
};

// One problem instance of a batched plan.  The instances' subdomains, interface
// blocks and Toeplitz first columns are concatenated; the interface kernels take
// an InstInfo table plus a block -> instance (or interface -> instance) map, or
// NULL for a single instance described by their (N, nt) arguments.
struct InstInfo {
    int N;            // subdomains
    int nt;           // time steps
    int sub0;         // first subdomain (global index)
    int if0;          // first interface (global index; its interfaces are k = 0..N-2)
    int blk0;         // first interface block (global index; 2N-2 blocks)
    int pad;
    long long foff;   // offset (complex entries) of its interface vector (blocks of nt)
    long long coff;   // offset of its first columns (4N slots of nt)
};

// Process-wide count of kernels launched by this library (swr_capi.cu).
void swr_count_launch(int n);

// Host-side launchers (swr_march.cu)
int swr_launch_assemble_static(const double* V, int N, const int* d_n, const int* d_goff,
                               const int* d_loff, const int* d_tc, int ntot, double h, double dt,
                               double2 sigma0, double2 inv_ik, double2* dg, double2* od,
                               cudaStream_t s, const double2* kap = nullptr, int kstride = 0);
// Per-end kernels of S_0^3, S_0^4, S_1^2, S_1^4 (tc = SWR_TC_*) from V(x): kap (the end's
// own operator), kout (the flux update's: both sides' sum) for m < kstride, rho (s = 0).
int swr_launch_tc_kernels(int tc, const double* V, int N, const int* d_n, const int* d_goff,
                          const int* d_tc, int kstride, double h, double dt, const double* beta,
                          double2 c2, double2* kap, double2* kout, double2* rho, cudaStream_t s);
int swr_launch_row_mean(const double* V, int nrows, long long nx, double* out, cudaStream_t s);
int swr_factor_alloc(FactorSet& fs, int N, int L, int P, cudaStream_t s, int nsteps = 1,
                     long long ldd = 0);
size_t swr_factor_step_bytes(int N, int L, int P);
// Assemble and factor the matrices of steps 1..fs.nsteps of a tabulated V(t,x)
// (row t of V at t * vstride), W = (V(t_{n-1}) + V(t_n)) / 2 at step n.
int swr_launch_factor_steps(FactorSet& fs, int N, const int* d_n, const int* d_goff,
                            const int* d_loff, const int* d_tc, int nmax, const double* V,
                            long long vstride, double h, double dt, double2 sigma0,
                            double2 inv_ik, int* status, cudaStream_t s);
void swr_factor_free(FactorSet& fs);
int swr_launch_factor(FactorSet& fs, int N, const int* d_n, const int* d_loff, const double2* dg,
                      const double2* od, int* status, cudaStream_t s);
// The two-level separator data (FactorSet.tl_*) after swr_launch_factor, for a constant
// matrix with P + 1 <= kTlMaxSep (wide: kTlMaxSepWide; the arrays are allocated here when
// swr_factor_alloc did not).  0, -1 (CUDA error) or -2 (not applicable).
int swr_launch_factor_tl(FactorSet& fs, int N, const int* d_loff, const double2* dg,
                         const double2* od, int* status, cudaStream_t s, bool wide = false);
int swr_launch_march(const FactorSet& fs, MarchArgs a, int nsys_groups, cudaStream_t s,
                     int mode = 0);
int swr_launch_march_nl(const FactorSet& fs, MarchArgs a, double cw, double coef, double tol,
                        int maxit, int* iters, int ngroups, cudaStream_t s, int mode = 0,
                        unsigned long long* pit = nullptr);
int swr_launch_march_tdep(const FactorSet& fs, MarchArgs a, const double* V, long long vstride,
                          double h, double kappa, double2 sig_ik, int ngroups, cudaStream_t s);
int swr_march_smem_bytes(int T, int G, int stage_slots = 0);
int swr_march_tl_smem_bytes(int T);

// Interface algebra launchers (swr_krylov.cu)
int swr_launch_toeplitz(int N, int nt, const double2* cols, const double2* x, const double2* add,
                        double2* y, int mode, cudaStream_t s, const InstInfo* inst = nullptr,
                        const int* blk_inst = nullptr, int nblk_total = 0, int ntmax = 0);
int swr_launch_dots(const double2* V, long long ldv, int nvec, const double2* w, long long n,
                    double2* partial, int nblocks, double2* out, cudaStream_t s);
int swr_launch_gemv_sub(const double2* V, long long ldv, int nvec, const double2* h, double2* w,
                        long long n, double sign, cudaStream_t s);
int swr_launch_axpby(double2* y, const double2* x, long long n, double2 a, double2 b,
                     cudaStream_t s);
int swr_launch_scale_by_rnorm(double2* v, const double2* w, long long n, const double2* hdiag,
                              cudaStream_t s);
int swr_launch_givens(double2* H, int ldh, double2* cs, double2* sn, double2* sv, int j,
                      double* res_out, cudaStream_t s);
int swr_launch_lsq(const double2* H, int ldh, const double2* sv, int k, double2* y,
                   cudaStream_t s);
int swr_launch_causal(int N, int nt, const double2* cols, const double2* lag0,
                      const double2* y, double2* x, int sweeps, void* scratch, int* status,
                      cudaStream_t s, const InstInfo* inst = nullptr, const int* if_inst = nullptr,
                      int k0 = 0, int nif_group = 0, int nif_total = 0,
                      const double2* Gw = nullptr, int H = 0, double2* P = nullptr,
                      const double2* hspec = nullptr, double2* xspec = nullptr);
// FFT form of the substitution's history sums (single instance, nt >= kHistFftMinNt):
// column-segment spectra hspec and the launch's block spectra xspec, each
// 4 (N-1) swr_hist_blocks(nt) 64 complex.
constexpr int kHistFftMinNt = 64;
int swr_hist_blocks(int nt);
int swr_launch_hist_spectra(int N, int nt, const double2* cols, double2* hspec, cudaStream_t s);
// Long subdomains (beyond one cluster): the whole grid marches every system of the list
// (L = 16 factors), state in the scratch of swr_long_scratch_bytes(nsys, 16, P).
size_t swr_long_scratch_bytes(int nsys, int L, int P);
int swr_launch_march_long(const FactorSet& fs, MarchArgs a, void* scratch, size_t scratch_bytes,
                          int nsm, cudaStream_t s);
// Rows of the lag-0 inverse for the window form of the substitution, |j - k| <= H
// (1 <= H <= 8): Gw[nif][2H+1][4].
int swr_launch_lag0_window(int N, int nt, const double2* cols, const double2* lag0, double2* Gw,
                           int H, cudaStream_t s, const InstInfo* inst = nullptr,
                           const int* if_inst = nullptr, int nif_total = 0);
int swr_causal_capacity(int nt);
// Progress counters of the causal substitution sit kProgStride ints apart (one per
// 128-byte line: every counter is polled by many CTAs and written by one).
constexpr int kProgStride = 32;
// Test hook of the substitution's bounded waits on the current device: poll limit
// (<= 0: the default, about 1-2 s) and an interface whose progress is never
// published (< 0: none).  Returns 0 or -1 (CUDA error).
int swr_set_wait_hook(long long max_polls, int withhold);
size_t swr_causal_scratch_bytes(int N);
int swr_launch_lag0_setup(int N, int nt, const double2* cols, double2* lag0, cudaStream_t s,
                          const InstInfo* inst = nullptr, const int* if_inst = nullptr,
                          int nif_total = 0);
int swr_launch_jump(const double2* trace, const MarchSys* sys, int N, int nt, double* out,
                    cudaStream_t s, const InstInfo* inst = nullptr, const int* if_inst = nullptr,
                    int nif_total = 0);
// Toeplitz apply through the FFT (transform length M, a power of two >= 2 nt - 1;
// W[k] = exp(-2 pi i k / M), k < M/2): spectra of the 4 N first columns once per
// build, then applies as swr_launch_toeplitz.
int swr_launch_col_spectra(int nsub_total, int nt, const double2* cols, double2* spec, int M,
                           const double2* W, cudaStream_t s, const InstInfo* inst = nullptr,
                           int ninst = 0);
int swr_launch_toeplitz_fft(int N, int nt, const double2* spec, const double2* x,
                            const double2* add, double2* y, int mode, int M, const double2* W,
                            cudaStream_t s, const InstInfo* inst = nullptr,
                            const int* blk_inst = nullptr, int nblk_total = 0);
// The same for convolution operators (S_0^2: kout NULL, K = 2 c2 beta; the higher-order
// ones: the flux kernels kout); nt <= 4259 (trace, kernel and data in shared memory).
int swr_launch_jump_conv(const double2* w, const double2* g, int N, int nt, const double2* kout,
                         int kstride, double2 c2, const double* beta, double* out,
                         cudaStream_t s, const InstInfo* inst = nullptr,
                         const int* if_inst = nullptr, int nif_total = 0);
// u(T) by superposition of the recorded build-march states (static V): subdomain j's
// states at urec + rec_base[j] (impulse-l responses, impulse-r responses, each nt rows of
// n_j, then the zero-flux final state); sys[j] gives its flux blocks and step count.
int swr_launch_superpose(const double2* urec, const long long* rec_base, const MarchSys* sys,
                         int N, const int* sub_n, const int* sub_goff, const int* sub_tc,
                         int nmax, const double2* g, double2* uT, cudaStream_t s);
// Interface mismatch from R(g) = L g + d (w) and g: max |(w-g)[l_{k+1}] - (w-g)[r_k]| * scale.
int swr_launch_jump_res(const double2* w, const double2* g, int N, int nt, double scale,
                        double* out, cudaStream_t s, const InstInfo* inst = nullptr,
                        const int* if_inst = nullptr, int nif_total = 0);
int swr_launch_misfit(const double2* u, const double2* tgt, long long n, double h, double2* ubar,
                      double* part, double* out, cudaStream_t s);
int swr_launch_adj_seed(const double2* ubar, double half_dt, long long n, double2* y,
                        cudaStream_t s);
int swr_launch_grad_combine(const double* gint, const double* gl, const double* gr, long long n,
                            double* out, cudaStream_t s);
// Time-dependent potential: one adjoint step's potential-form sums (gint, gl, gr) give
// dJ/dW_n = -2 (gint + gl + gr), which enters dJ/dV_n and dJ/dV_{n-1} with weight 1/2
// each (W_n = (V_n + V_{n-1}) / 2); adds them to rows n and n-1 of out (nx each) and
// clears the sums.
int swr_launch_grad_step_tdep(double* gint, double* gl, double* gr, long long nx, int n,
                              double* out, cudaStream_t s);
