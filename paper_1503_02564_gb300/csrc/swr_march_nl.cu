// Nonlinear subdomain march (Besse & Xing, Eq. CNS_NL / AvMNL): the Durán–Sanz-Serna
// scheme with f(v) = c |v|^2 on top of a static potential V0.  The matrix
// (2i/dt) M - S + M_{V0} - B is constant, so the chunked factorisation of the
// static march is reused; every time step runs the fixed point
//     (A - B) zeta^{s+1} = (2i/dt) M u_{n-1} - b_f(zeta^s) - Q^T (l_n, r_n)^T,
//     zeta^0 = v_{n-1},   b_f(zeta) = M_{c|zeta|^2} zeta,
// until max |zeta^{s+1} - zeta^s| <= tol max(1, max |zeta^s|) over the subdomain
// (checked per system with shared-memory, or cluster, max-reductions), then
// v_n = zeta, u_n = 2 v_n - u_{n-1}.  Each inner iteration is one partitioned
// solve (chunk LU sweeps, separator PCR with precomputed coefficients, spike
// correction) with the generalised-mass term recomputed from the iterate.
#include <cooperative_groups.h>

#include "swr_internal.cuh"

namespace cg = cooperative_groups;

struct NlArgs {
    MarchArgs m;
    double cw;        // (h/12)/kappa: scale of b_f after the 1/(i kappa) pre-scaling
    double coef;      // f(u) = coef |u|^2
    double tol;       // inner tolerance
    int maxit;        // inner cap
    int* iters;       // optional: max inner iterations over steps, per system
    unsigned long long* pit;   // optional: += nodes x inner iterations, summed over steps
};

// sum of the P1 element weights times zeta around a node: s such that
// b_f = (h/12) s; W = coef |zeta|^2 at the three nodes (left/right may be absent)
__device__ __forceinline__ double2 bf_sum(bool hasl, bool hasr, double2 zl, double2 z0,
                                          double2 zr, double Wl, double W0, double Wr) {
    double2 s = make_double2(0.0, 0.0);
    if (hasl) {
        const double a = Wl + 3.0 * W0, b = Wl + W0;
        s.x = fma(a, z0.x, fma(b, zl.x, s.x));
        s.y = fma(a, z0.y, fma(b, zl.y, s.y));
    }
    if (hasr) {
        const double a = 3.0 * W0 + Wr, b = W0 + Wr;
        s.x = fma(a, z0.x, fma(b, zr.x, s.x));
        s.y = fma(a, z0.y, fma(b, zr.y, s.y));
    }
    return s;
}
// rhs - s * (h/12) / (i kappa) = rhs - s * (-i cw) = rhs + (-cw s.y, cw s.x)
__device__ __forceinline__ double2 sub_bf(double2 rhs, double2 s, double cw) {
    return make_double2(fma(-cw, s.y, rhs.x), fma(cw, s.x, rhs.y));
}
__device__ __forceinline__ double nrm2(double2 a) { return fma(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ double rmul(double2 a, double2 b) { return a.x * b.x - a.y * b.y; }
// Adjoint of the nonlinear step: the real-linear part of the linearised |v|^2 v,
// 2c conj(v_k) Re(v^T (dM_W/dW_k) w) / (h/12), from the element(s) at node k
// (values at k-1, k, k+1 of the forward v and of the iterate w).
__device__ __forceinline__ double2 lin_term(bool hasl, bool hasr, double2 vl, double2 v0,
                                            double2 vr, double2 wl, double2 w0, double2 wr,
                                            double coef) {
    double r = 0.0;
    if (hasl) r += rmul(vl, wl) + rmul(vl, w0) + rmul(v0, wl) + 3.0 * rmul(v0, w0);
    if (hasr) r += 3.0 * rmul(v0, w0) + rmul(v0, wr) + rmul(vr, w0) + rmul(vr, wr);
    const double s = 2.0 * coef * r;
    return make_double2(s * v0.x, -s * v0.y);
}
__device__ __forceinline__ unsigned long long dbits(double v) {
    return (unsigned long long)__double_as_longlong(v);
}

int swr_march_nl_smem_bytes(int T, int G) {
    return (int)sizeof(double2) * (4 * (T + G) + 6 * T + 2 * G) +
           (int)sizeof(unsigned long long) * (4 * G + 4);
}

// MODE 0: march; 1: also record v of every step (a.vrec); 2: adjoint of the
// nonlinear step (see swr_adjoint): the inner fixed point solves
//     (A - B) w + M_{c|v|^2} w + 2c conj(v) . Re(v^T dM w) = (2i/dt) M rho
// with v the recorded forward midpoint value of the mirrored step (a.vfwd), and
// the potential form of w against v is accumulated as in the constant-matrix march.
// The adjoint is linear in its data, so its inner test is relative:
// max |dw| <= tol max |w| (the march tests max |dzeta| <= tol max(1, max |zeta|)).
template <int L, int MODE>
__global__ void __launch_bounds__(256, 1) k_march_nl(const NlArgs na) {
    const MarchArgs& a = na.m;
    extern __shared__ double2 sm[];
    const int T = a.T, G = a.G, P = a.P, C = a.C, nt = a.nt, levels = a.levels;
    const int S = T + G;
    double2* usep = sm;
    double2* zsep = sm + S;
    double2* dA = sm + 2 * S;
    double2* dB = sm + 3 * S;
    double2* ufst = sm + 4 * S;
    double2* ulst = ufst + T;
    double2* zfst = ulst + T;
    double2* zlst = zfst + T;
    double2* yfst = zlst + T;
    double2* ylst = yfst + T;
    // reductions: red[slot][g][0] = max |dz|^2, red[slot][g][1] = max |z|^2; cnt[slot]
    unsigned long long* red = reinterpret_cast<unsigned long long*>(ylst + T);
    unsigned long long* cnt = red + 4 * G;
    double2* hsum = reinterpret_cast<double2*>(cnt + 4);   // [2G] S_0^2 history sums
    // the previous step's converged iterate (chunk nodes [L][T], separators SEP layout),
    // for the extrapolated start of the inner fixed point
    double2* zpc = hsum + 2 * G;
    double2* zps = zpc + L * T;
    // the converged iterates of the two steps before that (zeta_{n-3}, zeta_{n-4}; chunk
    // nodes [L][T] and separators, as zpc / zps) for the cubic start below
    double2* zh1c = zps + (T + G);
    double2* zh1s = zh1c + L * T;
    double2* zh2c = zh1s + (T + G);
    double2* zh2s = zh2c + L * T;
    // MODE 2: forward values of this step: chunk nodes [L][T] (element-major),
    // separators (SEP layout) and the chunk ends (CHK layout) for the neighbours
    double2* vfc = zh2s + (T + G);
    double2* vfsep = vfc + L * T;
    double2* vffst = vfsep + (T + G);
    double2* vflst = vffst + T;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (C > 1) ? (int)cl.block_rank() : 0;
    const int tid = threadIdx.x;
    int g, p, sidx;
    if (C == 1) {
        g = tid / (P + 1);
        p = tid - g * (P + 1);
        sidx = blockIdx.x * G + g;
        if (g >= G) p = -1;
    } else {
        g = 0;
        p = rank * T + tid;
        sidx = blockIdx.x / C;
        if (p > P) p = -1;
    }
    const bool valid = (p >= 0) && (sidx < a.nsys);
    auto SEP = [&](double2* arr, int ps) -> double2* {
        if (C == 1) return arr + g * (P + 1) + ps;
        const int home = ps / T;
        double2* base = (home == rank) ? arr : cl.map_shared_rank(arr, home);
        return base + (ps - home * T);
    };
    auto CHK = [&](double2* arr, int pc) -> double2* {
        if (C == 1) return arr + g * P + pc;
        const int home = pc / T;
        double2* base = (home == rank) ? arr : cl.map_shared_rank(arr, home);
        return base + (pc - home * T);
    };
    // per-CTA partial maxima (local atomics only); a system spread over a cluster
    // reads the partials of all its CTAs after the barrier
    auto RED = [&](int slot, int q) -> unsigned long long* { return red + (slot * G + g) * 2 + q; };
    auto RED_ALL = [&](int slot, int q) -> unsigned long long {
        if (C == 1) return *RED(slot, q);
        unsigned long long m = 0ull;
        for (int r = 0; r < C; ++r) {
            const unsigned long long* b = (r == rank) ? red : cl.map_shared_rank(red, r);
            const unsigned long long v = b[(slot * G + g) * 2 + q];
            m = v > m ? v : m;
        }
        return m;
    };
    auto CNT = [&](int slot) -> unsigned long long* { return cnt + slot; };
    auto SYNC = [&]() {
        if (C == 1)
            __syncthreads();
        else
            cl.sync();
    };
    const double2 zero = make_double2(0.0, 0.0);
    MarchSys sy = {0, 0, 0, -1, -1, -1, -1, 0};
    int j = 0, Pj = 0, Lp = 0, sp = 0, goff = 0, tcf = 0;
    if (valid) {
        sy = a.sys[sidx];
        j = sy.sub;
        Pj = a.sub_P[j];
        goff = a.sub_goff[j];
        tcf = a.sub_tc[j];
        Lp = (p < P) ? a.clen[j * P + p] : 0;
        sp = a.sep_pos[j * (P + 1) + p];
    }
    const bool zero_u0 = (sy.flags & SYS_ZERO_U0) != 0;
    const bool realsep = valid && (p <= Pj);
    const double2* F = a.fac + (size_t)j * L * 4 * P + (p < P ? p : 0);
    const double2* sE_l = a.sep + (size_t)(j * 3 + 0) * (P + 1);
    const double2* sE_r = a.sep + (size_t)(j * 3 + 1) * (P + 1);
    const double2* sbinv = a.sep + (size_t)(j * 3 + 2) * (P + 1);
    const double2* pcr = a.pcr + (size_t)j * levels * 2 * (P + 1);
    const double cw = na.cw, coef = na.coef;

    double2 u[L], z[L], f[L], y[L];
#pragma unroll
    for (int i = 0; i < L; ++i) {
        u[i] = (valid && i < Lp && !zero_u0) ? a.u0[goff + sp + 1 + i] : zero;
        z[i] = u[i];                                  // zeta^0 of step 1 is v_0 = u_0
        f[i] = zero;
        y[i] = zero;
    }
    if (valid) {
        const double2 u0s = (realsep && !zero_u0) ? a.u0[goff + sp] : zero;
        *SEP(usep, p) = u0s;
        *SEP(zsep, p) = u0s;
    }
    for (int q = tid; q < 4 * G + 4; q += blockDim.x) red[q] = 0ull;   // slots and counters
    // S_0^2: the end traces start with v_0 = u_0 at the end
    const bool hl = a.s02 && realsep && p == 0 && (tcf & 1);
    const bool hr = a.s02 && realsep && p == Pj && (tcf & 2);
    double2* hist_l = a.s02 ? a.hist + ((size_t)sidx * 2 + 0) * (nt + 1) : nullptr;
    double2* hist_r = a.s02 ? a.hist + ((size_t)sidx * 2 + 1) * (nt + 1) : nullptr;
    if (hl) hist_l[0] = zero_u0 ? zero : a.u0[goff + sp];
    if (hr) hist_r[0] = zero_u0 ? zero : a.u0[goff + sp];
    const int hs_l = (C == 1) ? 2 * g : 0, hs_r = hs_l + 1;
    SYNC();

    double2 lin = zero, rin = zero, fs = zero;
    int itmax = 0;
    unsigned long long itsum = 0;   // inner iterations summed over the steps
    bool nl_fail = false;
    double ga_int[MODE == 2 ? L : 1], ga_l = 0.0, ga_r = 0.0;   // MODE 2 sums
#pragma unroll
    for (int i = 0; i < (MODE == 2 ? L : 1); ++i) ga_int[i] = 0.0;
    for (int t = 1; t <= nt; ++t) {
        // ---- step-constant right-hand side (2i/dt) M u_{n-1} - fluxes, scaled ----
        if (valid && Lp > 0) {
            const double2 uL = *SEP(usep, p), uR = *SEP(usep, p + 1);
            double2 uf = zero, ul = zero;
#pragma unroll
            for (int i = 0; i < L; ++i) {
                if (i < Lp) {
                    const double2 left = (i == 0) ? uL : u[i - 1];
                    double2 right;
                    if (i + 1 < L)
                        right = (i == Lp - 1) ? uR : u[i + 1];
                    else
                        right = uR;
                    f[i] = make_double2(fma(4.0, u[i].x, left.x + right.x),
                                        fma(4.0, u[i].y, left.y + right.y));
                    if (i == 0) uf = u[i];
                    ul = csel(i == Lp - 1, u[i], ul);
                }
            }
            *CHK(ufst, p) = uf;
            *CHK(ulst, p) = ul;
        }
        if (a.s02) {
            // history sums of the ends this CTA holds, one warp per end
            const int lane = tid & 31, w = tid >> 5, nw = T >> 5;
            if (C == 1) {
                for (int e = w; e < 2 * G; e += nw) {
                    const int gs = blockIdx.x * G + (e >> 1), side = e & 1;
                    if (gs < a.nsys && (a.sub_tc[a.sys[gs].sub] & (1 << side))) {
                        const double2 hsv = s02_history(
                            a.beta, a.hist + ((size_t)gs * 2 + side) * (nt + 1), t, lane);
                        if (lane == 0) hsum[e] = hsv;
                    }
                }
            } else {
                const int Pe = a.sub_P[a.sys[sidx].sub];
                const int tce = a.sub_tc[a.sys[sidx].sub];
                if (w == 0 && rank == 0 && (tce & 1)) {
                    const double2 hsv = s02_history(a.beta, hist_l, t, lane);
                    if (lane == 0) hsum[0] = hsv;
                }
                if (w == (nw > 1 ? 1 : 0) && rank == Pe / T && (tce & 2)) {
                    const double2 hsv = s02_history(a.beta, hist_r, t, lane);
                    if (lane == 0) hsum[1] = hsv;
                }
            }
        }
        if constexpr (MODE == 2) {   // forward values of the mirrored step
            const double2* vrow = a.vfwd + (size_t)(nt - t) * a.nxrec + goff + sp;
            if (valid && Lp > 0) {
#pragma unroll
                for (int i = 0; i < L; ++i)
                    if (i < Lp) vfc[i * T + tid] = vrow[1 + i];
                *CHK(vffst, p) = vrow[1];
                *CHK(vflst, p) = vrow[Lp];
            }
            if (realsep) *SEP(vfsep, p) = vrow[0];
        }
        // reduction slot 0 serves the first inner iteration of this step
        for (int q = tid; q < 2 * G; q += blockDim.x) red[q] = 0ull;
        if (tid == 0) *CNT(0) = 0ull;
        SYNC();
        if (realsep) {
            const double2 us = *SEP(usep, p);
            const bool le = (p == 0), re = (p == Pj);
            const double2 um = le ? zero : *CHK(ulst, p - 1);
            const double2 up = re ? zero : *CHK(ufst, p);
            if (le)
                fs = make_double2(fma(2.0, us.x, up.x), fma(2.0, us.y, up.y));
            else if (re)
                fs = make_double2(fma(2.0, us.x, um.x), fma(2.0, us.y, um.y));
            else
                fs = make_double2(fma(4.0, us.x, um.x + up.x), fma(4.0, us.y, um.y + up.y));
            if (le && (tcf & 1)) {
                if (sy.flags & SYS_IMP_L)
                    lin = (t == 1) ? make_double2(1.0, 0.0) : zero;
                else
                    lin = (sy.in_l >= 0 && a.gin) ? a.gin[(size_t)sy.in_l + t - 1] : zero;
                fs = cfms(lin, a.inv_ik, fs);
                if (a.s02) fs = cfma(hsum[hs_l], a.c2_ik, fs);
            }
            if (re && (tcf & 2)) {
                if (sy.flags & SYS_IMP_R)
                    rin = (t == 1) ? make_double2(1.0, 0.0) : zero;
                else
                    rin = (sy.in_r >= 0 && a.gin) ? a.gin[(size_t)sy.in_r + t - 1] : zero;
                fs = cfms(rin, a.inv_ik, fs);
                if (a.s02) fs = cfma(hsum[hs_r], a.c2_ik, fs);
            }
        }
        // ---- inner fixed point (Eq. AvMNL) ------------------------------------
        // start: zeta^0 = 2 v_{n-1} - v_{n-2} (the paper starts from v_{n-1}; both reach the
        // same fixed point to the inner tolerance, the extrapolation in fewer iterations);
        // step 1 starts from v_0 = u_0.  Each thread updates its own nodes and separator;
        // neighbours read the separators only after the first barrier below.
        // start: cubic extrapolation of the last four steps' converged iterates,
        // zeta^0 = 4 z_{n-1} - 6 z_{n-2} + 4 z_{n-3} - z_{n-4} (t >= 5; linear for t = 2..4;
        // step 1 starts from v_0 = u_0).  The paper starts from v_{n-1}; every start
        // reaches the same fixed point to the inner tolerance, this one (about 1e-9 of
        // |zeta| on the nonlinear workload, against 2e-5 for the linear one) in fewest
        // iterations.  Each thread updates its own nodes and separator; neighbours read the
        // separators only after the first barrier below.
        auto predict = [&](double2 z1, double2 z2, double2 z3, double2 z4) -> double2 {
            if (t >= 5)
                return make_double2(fma(4.0, z1.x + z3.x, fma(-6.0, z2.x, -z4.x)),
                                    fma(4.0, z1.y + z3.y, fma(-6.0, z2.y, -z4.y)));
            if (t >= 2) return make_double2(fma(2.0, z1.x, -z2.x), fma(2.0, z1.y, -z2.y));
            return z1;
        };
        if (valid && Lp > 0) {
#pragma unroll
            for (int i = 0; i < L; ++i) {
                if (i < Lp) {
                    const double2 z2 = zpc[i * T + tid], z3 = zh1c[i * T + tid],
                                  z4 = zh2c[i * T + tid];
                    zh2c[i * T + tid] = z3;
                    zh1c[i * T + tid] = z2;
                    zpc[i * T + tid] = z[i];
                    z[i] = predict(z[i], z2, z3, z4);
                }
            }
        }
        if (realsep) {
            double2* zs = SEP(zsep, p);
            double2* q0 = SEP(zps, p);
            double2* q1 = SEP(zh1s, p);
            double2* q2 = SEP(zh2s, p);
            const double2 z1 = *zs, z2 = *q0, z3 = *q1, z4 = *q2;
            *q2 = z3;
            *q1 = z2;
            *q0 = z1;
            *zs = predict(z1, z2, z3, z4);
        }
        bool active = valid;
        int used = na.maxit;
        // The test on max |zeta^{s+1} - zeta^s|^2 = dm against tol^2 max(1, max |zeta|^2)
        // (MODE 2, linear in w: against tol^2 max |w|^2).  The iteration contracts by a
        // factor rho near the fixed point; from the second iteration on rho is estimated
        // as sqrt(dm / dm_prev) and, when below 1/4, the distance of the new iterate from
        // the fixed point, at most rho / (1 - rho) of the last difference, is what is
        // tested: that saves the iteration that would only confirm the last one.
        double dm_prev = 0.0;
        auto converged = [&](double dm, double zm, double dmp, int itn) -> bool {
            const double lim = na.tol * na.tol * (MODE == 2 ? zm : fmax(1.0, zm));
            if (dm <= lim) return true;
            if (itn >= 1 && dmp > 0.0 && dm < 0.0625 * dmp) {
                const double rho = sqrt(dm / dmp);
                const double q = rho / (1.0 - rho);
                return dm * q * q <= lim;
            }
            return false;
        };
        for (int it = 0; it < na.maxit; ++it) {
            const int slot = it & 1, nslot = slot ^ 1;
            if (valid && Lp > 0) {
                double2 zf = zero, zl = zero;
#pragma unroll
                for (int i = 0; i < L; ++i) {
                    if (i == 0) zf = z[i];
                    zl = csel(i == Lp - 1, z[i], zl);
                }
                *CHK(zfst, p) = zf;
                *CHK(zlst, p) = zl;
            }
            SYNC();
            for (int q = tid; q < 2 * G; q += blockDim.x) red[nslot * 2 * G + q] = 0ull;
            if (tid == 0) *CNT(nslot) = 0ull;
            // chunk: right-hand side with b_f(zeta), local LU sweeps
            if (active && Lp > 0) {
                const double2 zL = *SEP(zsep, p), zR = *SEP(zsep, p + 1);
                double Wprev = coef * nrm2(zL);
                double W0 = coef * nrm2(z[0]);
                double2 vL = zero, vR = zero;
                if constexpr (MODE == 2) {   // W from the forward values
                    vL = *SEP(vfsep, p);
                    vR = *SEP(vfsep, p + 1);
                    Wprev = coef * nrm2(vL);
                    W0 = coef * nrm2(vfc[tid]);
                }
                double2 zprev = zero, cprev = zero;
#pragma unroll
                for (int i = 0; i < L; ++i) {
                    if (i < Lp) {
                        const double2 zl_ = (i == 0) ? zL : z[i - 1];
                        double2 zr_;
                        if (i + 1 < L)
                            zr_ = (i == Lp - 1) ? zR : z[i + 1];
                        else
                            zr_ = zR;
                        double Wr;
                        double2 sx;
                        if constexpr (MODE == 2) {
                            const double2 vl = (i == 0) ? vL : vfc[(i > 0 ? i - 1 : 0) * T + tid];
                            const double2 v0 = vfc[i * T + tid];
                            const double2 vr = (i + 1 < L && i != Lp - 1)
                                                   ? vfc[(i + 1 < L ? i + 1 : 0) * T + tid] : vR;
                            Wr = coef * nrm2(vr);
                            sx = cadd(bf_sum(true, true, zl_, z[i], zr_, Wprev, W0, Wr),
                                      lin_term(true, true, vl, v0, vr, zl_, z[i], zr_, coef));
                        } else {
                            Wr = coef * nrm2(zr_);
                            sx = bf_sum(true, true, zl_, z[i], zr_, Wprev, W0, Wr);
                        }
                        const double2 rhs = sub_bf(f[i], sx, cw);
                        const double2 zz = (i == 0) ? rhs : cfms(cprev, zprev, rhs);
                        y[i] = zz;
                        zprev = zz;
                        cprev = F[(i * 4 + 1) * P];
                        Wprev = W0;
                        W0 = Wr;
                    }
                }
                double2 ynext = zero, yl = zero;
#pragma unroll
                for (int i = L - 1; i >= 0; --i) {
                    if (i < Lp) {
                        double2 yi = cmul(F[(i * 4 + 0) * P], y[i]);
                        if (i != Lp - 1) yi = cfms(F[(i * 4 + 1) * P], ynext, yi);
                        else yl = yi;
                        y[i] = yi;
                        ynext = yi;
                    }
                }
                *CHK(yfst, p) = y[0];
                *CHK(ylst, p) = yl;
            }
            SYNC();
            // separator: reduced right-hand side
            if (valid) {
                double2 d = zero;
                if (active && realsep) {
                    const bool hasl = (p > 0), hasr = (p < Pj);
                    const double2 zs = *SEP(zsep, p);
                    const double2 zl_ = hasl ? *CHK(zlst, p - 1) : zero;
                    const double2 zr_ = hasr ? *CHK(zfst, p) : zero;
                    double2 sb;
                    if constexpr (MODE == 2) {
                        const double2 vs = *SEP(vfsep, p);
                        const double2 vl = hasl ? *CHK(vflst, p - 1) : zero;
                        const double2 vr = hasr ? *CHK(vffst, p) : zero;
                        sb = cadd(bf_sum(hasl, hasr, zl_, zs, zr_, coef * nrm2(vl), coef * nrm2(vs),
                                         coef * nrm2(vr)),
                                  lin_term(hasl, hasr, vl, vs, vr, zl_, zs, zr_, coef));
                    } else {
                        sb = bf_sum(hasl, hasr, zl_, zs, zr_, coef * nrm2(zl_), coef * nrm2(zs),
                                    coef * nrm2(zr_));
                    }
                    d = sub_bf(fs, sb, cw);
                    if (hasl) d = cfms(sE_l[p], *CHK(ylst, p - 1), d);
                    if (hasr) d = cfms(sE_r[p], *CHK(yfst, p), d);
                }
                *SEP(dA, p) = d;
            }
            SYNC();
            double2* src = dA;
            double2* dst = dB;
            for (int k = 0; k < levels; ++k) {
                const int st = 1 << k;
                if (valid) {
                    const double2* al = pcr + (size_t)(k * 2 + 0) * (P + 1);
                    const double2* ga = pcr + (size_t)(k * 2 + 1) * (P + 1);
                    double2 dd = *SEP(src, p);
                    if (p - st >= 0) dd = cfma(al[p], *SEP(src, p - st), dd);
                    if (p + st <= P) dd = cfma(ga[p], *SEP(src, p + st), dd);
                    if (k == levels - 1) dd = cmul(dd, sbinv[p]);
                    *SEP(dst, p) = dd;
                }
                SYNC();
                double2* tmp = src;
                src = dst;
                dst = tmp;
            }
            // correction, change of the iterate, per-system max reductions
            double dmax = 0.0, zmax = 0.0;
            double2 zsn = zero;
            if (active && Lp > 0) {
                const double2 vL = *SEP(src, p), vR = *SEP(src, p + 1);
#pragma unroll
                for (int i = 0; i < L; ++i) {
                    if (i < Lp) {
                        double2 v = cfms(F[(i * 4 + 2) * P], vL, y[i]);
                        v = cfms(F[(i * 4 + 3) * P], vR, v);
                        dmax = fmax(dmax, nrm2(csub(v, z[i])));
                        zmax = fmax(zmax, nrm2(z[i]));
                        y[i] = v;                       // new iterate, kept in y
                    }
                }
            }
            if (active && realsep) {
                zsn = *SEP(src, p);
                const double2 zs = *SEP(zsep, p);
                dmax = fmax(dmax, nrm2(csub(zsn, zs)));
                zmax = fmax(zmax, nrm2(zs));
            }
            if (active) {
                atomicMax(RED(slot, 0), dbits(dmax));
                atomicMax(RED(slot, 1), dbits(zmax));
            }
            SYNC();
            // C > 1: every thread of the cluster (padding threads included) evaluates the
            // one system's test on the same partials, so the exit below is uniform
            bool conv_all = false;
            if (C > 1) {
                const double dm = __longlong_as_double((long long)RED_ALL(slot, 0));
                const double zm = __longlong_as_double((long long)RED_ALL(slot, 1));
                conv_all = converged(dm, zm, dm_prev, it);
            }
            if (active) {
                const double dm = __longlong_as_double((long long)RED_ALL(slot, 0));
                const double zm = __longlong_as_double((long long)RED_ALL(slot, 1));
#pragma unroll
                for (int i = 0; i < L; ++i)
                    if (i < Lp) z[i] = y[i];
                if (realsep) *SEP(zsep, p) = zsn;
                if (converged(dm, zm, dm_prev, it)) {
                    active = false;
                    used = it + 1;
                } else if (C == 1 && p == 0) {
                    atomicAdd(CNT(slot), 1ull);
                }
            }
            if (active || C > 1)   // the next test's previous difference (this system's)
                dm_prev = __longlong_as_double((long long)RED_ALL(slot, 0));
            // C == 1: stop when no system of the CTA is still iterating.  C > 1: one
            // system, whose decision every thread of the cluster computed identically.
            bool more;
            if (C == 1) {
                __syncthreads();
                more = (*CNT(slot) != 0ull);
            } else {
                more = !conv_all;
                cl.sync();           // every CTA has read the partials before any reset
            }
            if (!more) break;
        }
        if (active) nl_fail = true;      // cap reached without convergence
        if (valid && used > itmax) itmax = used;
        itsum += (unsigned long long)used;
        if constexpr (MODE == 1) {   // record v_n (an interface node by its left subdomain)
            double2* row = a.vrec + (size_t)(t - 1) * a.nxrec + goff + sp;
            if (valid && Lp > 0) {
#pragma unroll
                for (int i = 0; i < L; ++i)
                    if (i < Lp) row[1 + i] = z[i];
            }
            if (realsep && !(p == 0 && (tcf & 1))) row[0] = *SEP(zsep, p);
        }
        if constexpr (MODE == 2) {
            // potential form of w (this march) against the forward v, elements from
            // separator p to separator p+1 (as in the constant-matrix march)
            if (valid && p < Pj) {
                const double2 xL = *SEP(zsep, p), xR = *SEP(zsep, p + 1);
                const double2 yL = *SEP(vfsep, p), yR = *SEP(vfsep, p + 1);
                const double h12 = a.h12;
#pragma unroll
                for (int e = 0; e <= L; ++e) {
                    if (e <= Lp) {
                        const int im = e > 0 ? e - 1 : 0, ic = e < L ? e : 0;
                        const double2 xa = (e == 0) ? xL : z[im];
                        const double2 ya = (e == 0) ? yL : vfc[im * T + tid];
                        const double2 xb = (e < L) ? csel(e < Lp, z[ic], xR) : xR;
                        const double2 yb = (e < L && e < Lp) ? vfc[ic * T + tid] : yR;
                        const double sa = rmul(xa, ya), sb = rmul(xb, yb);
                        const double c = rmul(xa, yb) + rmul(xb, ya);
                        const double toa = h12 * (3.0 * sa + c + sb);
                        const double tob = h12 * (sa + c + 3.0 * sb);
                        if (e == 0) ga_l += toa;
                        else ga_int[im] += toa;
                        if (e < Lp) ga_int[ic] += tob;
                        else ga_r += tob;
                    }
                }
            }
        }
        // ---- v_n = zeta: CN update and fluxes ---------------------------------
#pragma unroll
        for (int i = 0; i < L; ++i)
            if (valid && i < Lp) u[i] = make_double2(fma(2.0, z[i].x, -u[i].x), fma(2.0, z[i].y, -u[i].y));
        if (realsep) {
            const double2 v = *SEP(zsep, p);
            double2* us = SEP(usep, p);
            const double2 uo = *us;
            *us = make_double2(fma(2.0, v.x, -uo.x), fma(2.0, v.y, -uo.y));
            if (p == 0) {
                if (hl) hist_l[t] = v;
                if ((tcf & 1) && sy.out_a >= 0 && a.gout) {
                    double2 o = csub(cmul(a.two_sigma, v), lin);
                    if (a.s02) o = cfma(a.two_c2, hsum[hs_l], o);
                    a.gout[(size_t)sy.out_a + t - 1] = o;
                }
                if ((sy.flags & SYS_TRACE) && a.trace) a.trace[((size_t)sidx * 2 + 0) * nt + t - 1] = v;
            }
            if (p == Pj) {
                if (hr) hist_r[t] = v;
                if ((tcf & 2) && sy.out_b >= 0 && a.gout) {
                    double2 o = csub(cmul(a.two_sigma, v), rin);
                    if (a.s02) o = cfma(a.two_c2, hsum[hs_r], o);
                    a.gout[(size_t)sy.out_b + t - 1] = o;
                }
                if ((sy.flags & SYS_TRACE) && a.trace) a.trace[((size_t)sidx * 2 + 1) * nt + t - 1] = v;
            }
        }
        SYNC();
    }
    if constexpr (MODE == 2) {   // add this segment's sums (one writer per entry)
        if (valid && p < Pj) {
#pragma unroll
            for (int i = 0; i < L; ++i)
                if (i < Lp) a.gint[goff + sp + 1 + i] += ga_int[i];
            a.gl[goff + sp] += ga_l;
            a.gr[goff + sp + Lp + 1] += ga_r;
        }
    }
    bool bad = false;
    if (valid) {
#pragma unroll
        for (int i = 0; i < L; ++i)
            if (i < Lp) bad |= !cfinite(u[i]);
        if ((sy.flags & SYS_WRITE_UT) && a.uT) {
#pragma unroll
            for (int i = 0; i < L; ++i)
                if (i < Lp) a.uT[goff + sp + 1 + i] = u[i];
        }
        if (realsep) {
            const double2 us = *SEP(usep, p);
            bad |= !cfinite(us);
            if ((sy.flags & SYS_WRITE_UT) && a.uT && (sp > 0 || !(tcf & 1))) a.uT[goff + sp] = us;
        }
        if (p == 0 && na.iters) atomicMax(na.iters + sidx, itmax);
        if (p == 0 && na.pit) atomicAdd(na.pit, itsum * (unsigned long long)a.sub_n[j]);
    }
    if (bad) atomicOr(a.status, ST_NONFINITE);
    if (nl_fail) atomicOr(a.status, ST_NL_NOCONV);
    if (C > 1) cl.sync();
}

// ---------------------------------------------------------------------------
// The nonlinear march of one system spread over a cluster of C > 1 CTAs with the
// two-level separator solve of the constant-matrix march (FactorSet.tl_*): every inner
// iteration solves its separators with warp-shuffle PCR in blocks of 32 and a reduced
// system of the super-separators that every CTA solves redundantly (at most 32 unknowns:
// warp 0 with shuffles; a wide system of up to tl_rs <= T unknowns: the whole CTA, one
// barrier per PCR level), with one cluster barrier, and a second one for the convergence
// test, where the cluster-wide PCR took one per level.  MODE 0; 1 also records v_n of
// every step into a.vrec; 2 is the adjoint step of the nonlinear gradient (as k_march_nl:
// the linearised term about the recorded forward values a.vfwd, a relative test, the
// potential-form sums added to a.gint, a.gl, a.gr).  Robin or Neumann ends.  Thread
// p = rank T + tid owns separator p and chunk p; T is a multiple of 32.  Per step: the
// step-constant right-hand sides, the start of the fixed point, then per inner iteration
//   A  chunk right-hand sides with b_f(zeta), local LU solves;
//   B  separator right-hand sides: a separator's own part (its right element) and the
//      part of its left element, formed by the thread of the chunk on its left (the
//      same thread's neighbour in the warp, or lane 31 of the warp before for a
//      super-separator, which publishes it);
//   C  super-chunk PCR in registers, publication, cluster barrier;
//   D  the reduced system in every CTA (every CTA holds the new iterate at all
//      super-separators), CTA barrier;
//   E  super-chunk values; F  chunk values, change of the iterate, partial maxima;
//   G  cluster barrier, the convergence test on all CTAs' partials (the same decision
//      everywhere).
// After the fixed point: v_n = zeta, u_n = 2 v_n - u_{n-1}, fluxes.
// Shared memory: see swr_march_nl_tl_smem_bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 nl_shup(double2 v, int d) {
    return make_double2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ double2 nl_shdn(double2 v, int d) {
    return make_double2(__shfl_down_sync(0xffffffffu, v.x, d),
                        __shfl_down_sync(0xffffffffu, v.y, d));
}

int swr_march_nl_tl_smem_bytes(int L, int T, int RS, int mode) {
    const int W = T / 32;
    // usep zsep xv ulst ylst zlst [T] each; pub [2][W][5]; usup [RS], zsb [2][RS]; step
    // histories: chunk nodes [3][L][T], own separators [3][T], replicas [3][RS]; the wide
    // reduced PCR [2][RS]; MODE 2: forward values vfc [L][T], vfsep and vflst [T], vfsup
    // [RS], and the potential-form sums [L + 2][T] (doubles); partial maxima [2][2]
    int n2 = 6 * T + 2 * W * 5 + 3 * RS + 3 * L * T + 3 * T + 3 * RS + 2 * RS;
    if (mode == 2) n2 += L * T + 2 * T + RS;
    return (int)sizeof(double2) * n2 + (mode == 2 ? (int)sizeof(double) * (L + 2) * T : 0) +
           (int)sizeof(unsigned long long) * 4;
}

template <int L, int MODE>
__global__ void __launch_bounds__(256, 1) k_march_nl_tl(const NlArgs na) {
    const MarchArgs& a = na.m;
    extern __shared__ double2 sm[];
    const int T = a.T, P = a.P, C = a.C, nt = a.nt;
    const int W = T / 32;
    const int RS = a.tl_rs, RLv = a.tl_rl;   // reduced system: 32 (one warp) or wide
    double2* usep = sm;              // [T] u at my separators
    double2* zsep = usep + T;        // [T] the iterate at my separators
    double2* xv = zsep + T;          // [T] the separators' new iterate (this iteration)
    double2* ulst = xv + T;          // [T] chunk ends (last node): u, y, zeta
    double2* ylst = ulst + T;
    double2* zlst = ylst + T;
    double2* pub = zlst + T;         // [2][W][5]
    double2* usup = pub + 2 * W * 5; // [RS] u at the super-separators (every CTA)
    double2* zsb = usup + RS;        // [2][RS] the iterate at the super-separators (ping-pong)
    double2* hc = zsb + 2 * RS;      // [3][L][T] chunk iterates of steps n-2, n-3, n-4
    double2* hs = hc + 3 * L * T;    // [3][T] own separators' iterates, same steps
    double2* hq = hs + 3 * T;        // [3][RS] super-separators' iterates, same steps
    double2* rA = hq + 3 * RS;       // [2][RS] wide reduced PCR (ping-pong)
    double2* rB = rA + RS;
    double2* vfc = rB + RS;          // MODE 2 [L][T] forward values of my chunk's nodes
    double2* vfsep = vfc + L * T;    // MODE 2 [T] at my separators, [T] at my chunk's end,
    double2* vflst = vfsep + T;      //        [RS] at the super-separators
    double2* vfsup = vflst + T;
    double* gsm = reinterpret_cast<double*>(vfsup + RS);   // MODE 2 [L + 2][T] sums
    unsigned long long* red = reinterpret_cast<unsigned long long*>(
        MODE == 2 ? (void*)(gsm + (L + 2) * T) : (void*)vfc);   // [2][2]
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, wl = tid >> 5;
    const int p = rank * T + tid;
    const int sidx = blockIdx.x / C;
    const double2 zero = make_double2(0.0, 0.0);
    const bool valid = (p <= P) && (sidx < a.nsys);
    MarchSys sy = {0, 0, 0, -1, -1, -1, -1, 0};
    int j = 0, Pj = 0, Lp = 0, sp = 0, goff = 0, tcf = 0;
    if (sidx < a.nsys) {
        sy = a.sys[sidx];
        j = sy.sub;
        Pj = a.sub_P[j];
        goff = a.sub_goff[j];
        tcf = a.sub_tc[j];
    }
    if (valid) {
        Lp = (p < P) ? a.clen[j * P + p] : 0;
        sp = a.sep_pos[j * (P + 1) + p];
    }
    const int Q = (Pj + 31) / 32;
    const int q = p >> 5;
    const bool zero_u0 = (sy.flags & SYS_ZERO_U0) != 0;
    const bool realsep = valid && (p <= Pj);
    const bool sup = realsep && (lane == 0 || p == Pj);
    const int qsup = (p == Pj) ? Q : q;
    const int m = (32 * q < Pj) ? min(31, Pj - 1 - 32 * q) : 0;
    const bool member = realsep && lane >= 1 && lane <= m;
    const int rsup = (p + 1 == Pj) ? Q : (((p + 1) & 31) == 0 ? (p + 1) >> 5 : -1);
    const size_t S = P + 1;
    const double2* F = a.fac + (size_t)j * L * 4 * P + (p < P ? p : 0);
    const double2* sE_l = a.sep + (size_t)(j * 3 + 0) * S;
    const double2* sE_r = a.sep + (size_t)(j * 3 + 1) * S;
    const double2* tpc = a.tl_pcr + (size_t)j * 10 * S + (valid ? p : 0);
    const double2* tax = a.tl_aux + (size_t)j * 3 * S + (valid ? p : 0);
    const double2* trow = a.tl_red + (size_t)j * (2 * RLv + 3) * RS;
    const double2* tred = trow + lane;   // one-warp reduced system (RS = 32)
    const double cw = na.cw, coef = na.coef;
    const bool le = (p == 0), re = (p == Pj);
    const bool own_left = realsep && !le && lane != 0;   // the chunk on the left is in my warp

    double2 u[L], z[L], f[L], y[L];
#pragma unroll
    for (int i = 0; i < L; ++i) {
        u[i] = (valid && i < Lp && !zero_u0) ? a.u0[goff + sp + 1 + i] : zero;
        z[i] = u[i];                                  // zeta^0 of step 1 is v_0 = u_0
        f[i] = zero;
        y[i] = zero;
    }
    {
        const double2 u0s = (realsep && !zero_u0) ? a.u0[goff + sp] : zero;
        usep[tid] = u0s;
        zsep[tid] = u0s;
    }
    if (tid <= Q && sidx < a.nsys) {
        const int ps = (tid < Q) ? 32 * tid : Pj;
        const double2 us = zero_u0 ? zero : a.u0[goff + a.sep_pos[j * S + ps]];
        usup[tid] = us;
        zsb[tid] = us;
    }
    if constexpr (MODE == 2) {
#pragma unroll
        for (int i = 0; i < L + 2; ++i) gsm[i * T + tid] = 0.0;
    }
    if (tid < 4) red[tid] = 0ull;
    cl.sync();

    int cur = 0;                     // zsb + RS cur: the super-separators' current iterate
    int itg = 0;                     // inner iterations so far (parity of pub and red)
    int itmax = 0;
    unsigned long long itsum = 0;
    bool nl_fail = false;
    double2 lin = zero, rin = zero;
    for (int t = 1; t <= nt; ++t) {
        if constexpr (MODE == 2) {   // forward values of the mirrored step
            const double2* vrow = a.vfwd + (size_t)(nt - t) * a.nxrec + goff;
            if (valid && Lp > 0) {
#pragma unroll
                for (int i = 0; i < L; ++i)
                    if (i < Lp) vfc[i * T + tid] = vrow[sp + 1 + i];
                vflst[tid] = vrow[sp + Lp];
            }
            if (realsep) vfsep[tid] = vrow[sp];
            if (tid <= Q && sidx < a.nsys)
                vfsup[tid] = vrow[a.sep_pos[j * S + ((tid < Q) ? 32 * tid : Pj)]];
        }
        // ---- step-constant right-hand sides: chunks, and my separator's own part ------
        double2 uf = zero, ul = zero;
        if (valid && Lp > 0) {
            const double2 uL = usep[tid];
            const double2 uR = (rsup >= 0) ? usup[rsup] : usep[tid + 1];
#pragma unroll
            for (int i = 0; i < L; ++i) {
                if (i < Lp) {
                    const double2 left = (i == 0) ? uL : u[i - 1];
                    double2 right;
                    if (i + 1 < L)
                        right = (i == Lp - 1) ? uR : u[i + 1];
                    else
                        right = uR;
                    f[i] = make_double2(fma(4.0, u[i].x, left.x + right.x),
                                        fma(4.0, u[i].y, left.y + right.y));
                    if (i == 0) uf = u[i];
                    ul = csel(i == Lp - 1, u[i], ul);
                }
            }
            ulst[tid] = ul;
        }
        __syncwarp();
        // own part: (2 or 4) u_s + u of the right chunk's first node, boundary data; the
        // left chunk's last node joins it here (own_left) or through lane 31's part
        double2 fown = zero;
        if (realsep) {
            const double2 us = usep[tid];
            const double cs = (le || re) ? 2.0 : 4.0;
            fown = make_double2(fma(cs, us.x, re ? 0.0 : uf.x), fma(cs, us.y, re ? 0.0 : uf.y));
            if (own_left) fown = cadd(fown, ulst[tid - 1]);
            if (le && (tcf & 1)) {
                if (sy.flags & SYS_IMP_L)
                    lin = (t == 1) ? make_double2(1.0, 0.0) : zero;
                else
                    lin = (sy.in_l >= 0 && a.gin) ? a.gin[(size_t)sy.in_l + t - 1] : zero;
                fown = cfms(lin, a.inv_ik, fown);
            }
            if (re && (tcf & 2)) {
                if (sy.flags & SYS_IMP_R)
                    rin = (t == 1) ? make_double2(1.0, 0.0) : zero;
                else
                    rin = (sy.in_r >= 0 && a.gin) ? a.gin[(size_t)sy.in_r + t - 1] : zero;
                fown = cfms(rin, a.inv_ik, fown);
            }
        }
        // ---- start of the fixed point: cubic extrapolation (t >= 5), linear (t = 2..4)
        auto predict = [&](double2 z1, double2 z2, double2 z3, double2 z4) -> double2 {
            if (t >= 5)
                return make_double2(fma(4.0, z1.x + z3.x, fma(-6.0, z2.x, -z4.x)),
                                    fma(4.0, z1.y + z3.y, fma(-6.0, z2.y, -z4.y)));
            if (t >= 2) return make_double2(fma(2.0, z1.x, -z2.x), fma(2.0, z1.y, -z2.y));
            return z1;
        };
        if (valid && Lp > 0) {
#pragma unroll
            for (int i = 0; i < L; ++i) {
                if (i < Lp) {
                    double2* h = hc + (size_t)i * T + tid;        // steps n-2, n-3, n-4
                    const double2 z2 = h[0], z3 = h[(size_t)L * T], z4 = h[(size_t)2 * L * T];
                    h[(size_t)2 * L * T] = z3;
                    h[(size_t)L * T] = z2;
                    h[0] = z[i];
                    z[i] = predict(z[i], z2, z3, z4);
                }
            }
        }
        if (realsep) {
            const double2 z1 = zsep[tid], z2 = hs[tid], z3 = hs[T + tid], z4 = hs[2 * T + tid];
            hs[2 * T + tid] = z3;
            hs[T + tid] = z2;
            hs[tid] = z1;
            zsep[tid] = predict(z1, z2, z3, z4);
        }
        if (tid <= Q) {
            double2* zc = zsb + RS * cur;
            const double2 z1 = zc[tid], z2 = hq[tid], z3 = hq[RS + tid], z4 = hq[2 * RS + tid];
            hq[2 * RS + tid] = z3;
            hq[RS + tid] = z2;
            hq[tid] = z1;
            zc[tid] = predict(z1, z2, z3, z4);
        }
        __syncthreads();
        // ---- inner fixed point (Eq. AvMNL), the stopping rule of k_march_nl ------------
        int used = na.maxit;
        double dm_prev = 0.0;
        bool done = false;
        for (int it = 0; it < na.maxit; ++it, ++itg) {
            const int slot = (itg & 1) * W * 5, rs = itg & 1;
            const double2* zc = zsb + RS * cur;       // current iterate, super-separators
            double2* zn = zsb + RS * (cur ^ 1);       // the new one (phase D)
            // A: chunk right-hand side with b_f(zeta), local LU sweeps
            double2 zl_own = zero;
            if (valid && Lp > 0) {
                const double2 zL = zsep[tid];
                const double2 zR = (rsup >= 0) ? zc[rsup] : zsep[tid + 1];
                double Wprev = coef * nrm2(zL);
                double W0 = coef * nrm2(z[0]);
                double2 vL = zero, vR = zero;
                if constexpr (MODE == 2) {   // W from the forward values
                    vL = vfsep[tid];
                    vR = (rsup >= 0) ? vfsup[rsup] : vfsep[tid + 1];
                    Wprev = coef * nrm2(vL);
                    W0 = coef * nrm2(vfc[tid]);
                }
                double2 zprev = zero, cprev = zero;
#pragma unroll
                for (int i = 0; i < L; ++i) {
                    if (i < Lp) {
                        const double2 zl_ = (i == 0) ? zL : z[i - 1];
                        double2 zr_;
                        if (i + 1 < L)
                            zr_ = (i == Lp - 1) ? zR : z[i + 1];
                        else
                            zr_ = zR;
                        double Wr;
                        double2 sx;
                        if constexpr (MODE == 2) {
                            const double2 vl = (i == 0) ? vL : vfc[(i > 0 ? i - 1 : 0) * T + tid];
                            const double2 v0 = vfc[i * T + tid];
                            const double2 vr = (i + 1 < L && i != Lp - 1)
                                                   ? vfc[(i + 1 < L ? i + 1 : 0) * T + tid] : vR;
                            Wr = coef * nrm2(vr);
                            sx = cadd(bf_sum(true, true, zl_, z[i], zr_, Wprev, W0, Wr),
                                      lin_term(true, true, vl, v0, vr, zl_, z[i], zr_, coef));
                        } else {
                            Wr = coef * nrm2(zr_);
                            sx = bf_sum(true, true, zl_, z[i], zr_, Wprev, W0, Wr);
                        }
                        const double2 rhs = sub_bf(f[i], sx, cw);
                        const double2 zz = (i == 0) ? rhs : cfms(cprev, zprev, rhs);
                        y[i] = zz;
                        zprev = zz;
                        cprev = F[(i * 4 + 1) * P];
                        Wprev = W0;
                        W0 = Wr;
                        zl_own = csel(i == Lp - 1, z[i], zl_own);
                    }
                }
                double2 ynext = zero, yl = zero;
#pragma unroll
                for (int i = L - 1; i >= 0; --i) {
                    if (i < Lp) {
                        double2 yi = cmul(F[(i * 4 + 0) * P], y[i]);
                        if (i != Lp - 1) yi = cfms(F[(i * 4 + 1) * P], ynext, yi);
                        else yl = yi;
                        y[i] = yi;
                        ynext = yi;
                    }
                }
                ylst[tid] = yl;
                zlst[tid] = zl_own;
            }
            __syncwarp();
            // B: separator right-hand sides.  Right element of separator p: nodes (p, first
            // of chunk p); left element: (last of chunk p - 1, p).
            double2 d = zero;
            if (realsep) {
                const double2 zs = zsep[tid];
                double2 vs = zs;                      // W at the separator: iterate or forward
                if constexpr (MODE == 2) vs = vfsep[tid];
                const double W0 = coef * nrm2(vs);
                double2 sb = zero;
                if (!re) {
                    const double2 zr_ = z[0];
                    if constexpr (MODE == 2) {
                        const double2 vr = vfc[tid];
                        sb = cadd(bf_sum(false, true, zero, zs, zr_, 0.0, W0, coef * nrm2(vr)),
                                  lin_term(false, true, zero, vs, vr, zero, zs, zr_, coef));
                    } else {
                        sb = bf_sum(false, true, zero, zs, zr_, 0.0, W0, coef * nrm2(zr_));
                    }
                }
                if (own_left) {
                    const double2 zl_ = zlst[tid - 1];
                    if constexpr (MODE == 2) {
                        const double2 vl = vflst[tid - 1];
                        sb = cadd(sb, cadd(bf_sum(true, false, zl_, zs, zero, coef * nrm2(vl), W0,
                                                  0.0),
                                           lin_term(true, false, vl, vs, zero, zl_, zs, zero,
                                                    coef)));
                    } else {
                        sb = cadd(sb, bf_sum(true, false, zl_, zs, zero, coef * nrm2(zl_), W0,
                                             0.0));
                    }
                }
                d = sub_bf(fown, sb, cw);
                if (own_left) d = cfms(sE_l[p], ylst[tid - 1], d);
                if (!re) d = cfms(sE_r[p], y[0], d);
            }
            // lane 31: its chunk's part of the next super-separator's row (left element)
            double2 p1 = zero;
            if (valid && lane == 31 && p + 1 <= Pj) {
                const double2 zs1 = zc[rsup];        // p + 1 is a super-separator
                double2 sl;
                if constexpr (MODE == 2) {
                    const double2 vl = vflst[tid], vs1 = vfsup[rsup];
                    sl = cadd(bf_sum(true, false, zl_own, zs1, zero, coef * nrm2(vl),
                                     coef * nrm2(vs1), 0.0),
                              lin_term(true, false, vl, vs1, zero, zl_own, zs1, zero, coef));
                } else {
                    sl = bf_sum(true, false, zl_own, zs1, zero, coef * nrm2(zl_own),
                                coef * nrm2(zs1), 0.0);
                }
                p1 = cfms(sE_l[p + 1], ylst[tid], sub_bf(ulst[tid], sl, cw));
            }
            // C: super-chunk PCR in registers, publication, cluster barrier
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const int st = 1 << k;
                const double2 dm = nl_shup(d, st), dp = nl_shdn(d, st);
                if (member) d = cfma(tpc[(2 * k + 1) * S], dp, cfma(tpc[(2 * k) * S], dm, d));
            }
            if (member) d = cmul(d, tax[0]);
            {
                double2* pb = pub + slot + wl * 5;
                if (lane == 0 && realsep) pb[0] = d;
                if (lane == 31) pb[1] = p1;
                if (lane == 1 && member) pb[2] = d;
                if (member && lane == m) pb[3] = d;
                if (p == Pj && lane != 0 && valid) pb[4] = d;
            }
            cl.sync();
            if (tid == 0) {   // the next iteration's partial maxima start at zero
                red[2 * (rs ^ 1) + 0] = 0ull;
                red[2 * (rs ^ 1) + 1] = 0ull;
            }
            // D: the reduced system (every CTA holds the new iterate at all
            // super-separators): row i's right-hand side from the published values
            auto pubof = [&](int qq) -> const double2* {
                const int home = (32 * qq) / T;
                double2* base = (home == rank) ? pub : cl.map_shared_rank(pub, home);
                return base + slot + ((32 * qq) % T) / 32 * 5;
            };
            auto reduced_rhs = [&](int i) -> double2 {
                double2 r;
                if (i == Q && (Pj & 31) != 0) {
                    r = pubof(Q - 1)[4];
                } else {
                    r = pubof(i)[0];
                    if (i >= 1) r = cadd(r, pubof(i - 1)[1]);
                }
                const double2 cL = trow[(2 * RLv + 1) * RS + i], cU = trow[(2 * RLv + 2) * RS + i];
                if (i >= 1 && (cL.x != 0.0 || cL.y != 0.0)) r = cfms(cL, pubof(i - 1)[3], r);
                if (i < Q && (cU.x != 0.0 || cU.y != 0.0)) r = cfms(cU, pubof(i)[2], r);
                return r;
            };
            if (RS == 32) {   // warp 0: PCR by shuffles
                if (wl == 0 && sidx < a.nsys) {
                    double2 r = zero;
                    if (lane <= Q) r = reduced_rhs(lane);
#pragma unroll
                    for (int k = 0; k < 5; ++k) {
                        const int st = 1 << k;
                        if (st > Q) break;   // no neighbour within the Q + 1 unknowns
                        const double2 rm = nl_shup(r, st), rp = nl_shdn(r, st);
                        if (lane <= Q)
                            r = cfma(tred[(2 * k + 1) * 32], rp, cfma(tred[(2 * k) * 32], rm, r));
                    }
                    if (lane <= Q) zn[lane] = cmul(r, tred[10 * 32]);
                }
            } else {          // wide: PCR over the CTA, one barrier per level (T >= RS)
                double2 r = zero;
                if (tid <= Q && sidx < a.nsys) r = reduced_rhs(tid);
                if (tid < RS) rA[tid] = r;
                __syncthreads();
                double2* src = rA;
                double2* dst = rB;
                for (int k = 0; k < RLv; ++k) {
                    const int st = 1 << k;
                    if (st > Q) break;
                    if (tid <= Q) {
                        double2 v = src[tid];
                        if (tid >= st) v = cfma(trow[(2 * k) * RS + tid], src[tid - st], v);
                        if (tid + st <= Q) v = cfma(trow[(2 * k + 1) * RS + tid], src[tid + st], v);
                        dst[tid] = v;
                    }
                    __syncthreads();
                    double2* tmp = src;
                    src = dst;
                    dst = tmp;
                }
                if (tid <= Q) zn[tid] = cmul(src[tid], trow[(2 * RLv) * RS + tid]);
            }
            __syncthreads();
            // E: separator values of the new iterate
            double2 v = zero;
            if (member) {
                v = cfms(tax[S], zn[q], d);
                v = cfms(tax[2 * S], zn[q + 1], v);
            } else if (sup) {
                v = zn[qsup];
            }
            xv[tid] = v;
            __syncwarp();
            // F: chunk values of the new iterate, the change, partial maxima
            double dmax = 0.0, zmax = 0.0;
            if (valid && Lp > 0) {
                const double2 vR = (rsup >= 0) ? zn[rsup] : xv[tid + 1];
#pragma unroll
                for (int i = 0; i < L; ++i) {
                    if (i < Lp) {
                        double2 vi = cfms(F[(i * 4 + 2) * P], v, y[i]);
                        vi = cfms(F[(i * 4 + 3) * P], vR, vi);
                        dmax = fmax(dmax, nrm2(csub(vi, z[i])));
                        zmax = fmax(zmax, nrm2(z[i]));
                        z[i] = vi;
                    }
                }
            }
            if (realsep) {
                const double2 zs = zsep[tid];
                dmax = fmax(dmax, nrm2(csub(v, zs)));
                zmax = fmax(zmax, nrm2(zs));
                zsep[tid] = v;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
                zmax = fmax(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
            }
            if (lane == 0) {
                atomicMax(red + 2 * rs + 0, dbits(dmax));
                atomicMax(red + 2 * rs + 1, dbits(zmax));
            }
            // G: every CTA's partials, the same decision in every thread of the cluster
            cl.sync();
            double dm = 0.0, zm = 0.0;
            for (int r = 0; r < C; ++r) {
                const unsigned long long* b = (r == rank) ? red : cl.map_shared_rank(red, r);
                dm = fmax(dm, __longlong_as_double((long long)b[2 * rs + 0]));
                zm = fmax(zm, __longlong_as_double((long long)b[2 * rs + 1]));
            }
            cur ^= 1;                                  // the new iterate is current
            // MODE 2 (linear in w): relative to max |w|^2, as in k_march_nl
            const double lim = na.tol * na.tol * (MODE == 2 ? zm : fmax(1.0, zm));
            bool conv = dm <= lim;
            if (!conv && it >= 1 && dm_prev > 0.0 && dm < 0.0625 * dm_prev) {
                const double rho = sqrt(dm / dm_prev);
                const double qf = rho / (1.0 - rho);
                conv = dm * qf * qf <= lim;
            }
            dm_prev = dm;
            if (conv) {
                used = it + 1;
                done = true;
                ++itg;
                break;
            }
        }
        if (!done) nl_fail = true;      // cap reached without convergence
        if (used > itmax) itmax = used;
        itsum += (unsigned long long)used;
        if constexpr (MODE == 2) {
            // potential form of w (this march) against the forward v, elements from
            // separator p to separator p + 1 (as k_march_nl)
            if (valid && p < Pj) {
                const double2* zcv = zsb + RS * cur;
                const double2 xL = zsep[tid], xR = (rsup >= 0) ? zcv[rsup] : zsep[tid + 1];
                const double2 yL = vfsep[tid], yR = (rsup >= 0) ? vfsup[rsup] : vfsep[tid + 1];
                const double h12 = a.h12;
                double* g = gsm + tid;   // rows 0..L-1 interior nodes, L left end, L+1 right
#pragma unroll
                for (int e = 0; e <= L; ++e) {
                    if (e <= Lp) {
                        const int im = e > 0 ? e - 1 : 0, ic = e < L ? e : 0;
                        const double2 xa = (e == 0) ? xL : z[im];
                        const double2 ya = (e == 0) ? yL : vfc[im * T + tid];
                        const double2 xb = (e < L) ? csel(e < Lp, z[ic], xR) : xR;
                        const double2 yb = (e < L && e < Lp) ? vfc[ic * T + tid] : yR;
                        const double sa = rmul(xa, ya), sb = rmul(xb, yb);
                        const double c = rmul(xa, yb) + rmul(xb, ya);
                        const double toa = h12 * (3.0 * sa + c + sb);
                        const double tob = h12 * (sa + c + 3.0 * sb);
                        if (e == 0) g[L * T] += toa;
                        else g[im * T] += toa;
                        if (e < Lp) g[ic * T] += tob;
                        else g[(L + 1) * T] += tob;
                    }
                }
            }
        }
        if constexpr (MODE == 1) {   // record v_n (an interface node by its left subdomain)
            double2* row = a.vrec + (size_t)(t - 1) * a.nxrec + goff + sp;
            if (valid && Lp > 0) {
#pragma unroll
                for (int i = 0; i < L; ++i)
                    if (i < Lp) row[1 + i] = z[i];
            }
            if (realsep && !(p == 0 && (tcf & 1))) row[0] = zsep[tid];
        }
        // ---- v_n = zeta: CN update and fluxes -----------------------------------------
#pragma unroll
        for (int i = 0; i < L; ++i)
            if (valid && i < Lp) u[i] = make_double2(fma(2.0, z[i].x, -u[i].x), fma(2.0, z[i].y, -u[i].y));
        if (realsep) {
            const double2 v = zsep[tid];
            const double2 uo = usep[tid];
            usep[tid] = make_double2(fma(2.0, v.x, -uo.x), fma(2.0, v.y, -uo.y));
            if (p == 0) {
                if ((tcf & 1) && sy.out_a >= 0 && a.gout)
                    a.gout[(size_t)sy.out_a + t - 1] = csub(cmul(a.two_sigma, v), lin);
                if ((sy.flags & SYS_TRACE) && a.trace) a.trace[((size_t)sidx * 2 + 0) * nt + t - 1] = v;
            }
            if (p == Pj) {
                if ((tcf & 2) && sy.out_b >= 0 && a.gout)
                    a.gout[(size_t)sy.out_b + t - 1] = csub(cmul(a.two_sigma, v), rin);
                if ((sy.flags & SYS_TRACE) && a.trace) a.trace[((size_t)sidx * 2 + 1) * nt + t - 1] = v;
            }
        }
        if (tid <= Q) {
            const double2 v = zsb[RS * cur + tid], uo = usup[tid];
            usup[tid] = make_double2(fma(2.0, v.x, -uo.x), fma(2.0, v.y, -uo.y));
        }
        __syncthreads();
    }
    if constexpr (MODE == 2) {   // add this segment's sums (one writer per entry)
        if (valid && p < Pj) {
            const double* g = gsm + tid;
#pragma unroll
            for (int i = 0; i < L; ++i)
                if (i < Lp) a.gint[goff + sp + 1 + i] += g[i * T];
            a.gl[goff + sp] += g[L * T];
            a.gr[goff + sp + Lp + 1] += g[(L + 1) * T];
        }
    }
    // ---- final state ----------------------------------------------------------------
    bool bad = false;
    if (valid) {
#pragma unroll
        for (int i = 0; i < L; ++i)
            if (i < Lp) bad |= !cfinite(u[i]);
        if ((sy.flags & SYS_WRITE_UT) && a.uT) {
#pragma unroll
            for (int i = 0; i < L; ++i)
                if (i < Lp) a.uT[goff + sp + 1 + i] = u[i];
        }
        if (realsep) {
            const double2 us = usep[tid];
            bad |= !cfinite(us);
            if ((sy.flags & SYS_WRITE_UT) && a.uT && (sp > 0 || !(tcf & 1))) a.uT[goff + sp] = us;
        }
        if (p == 0 && rank == 0) {
            if (na.iters) atomicMax(na.iters + sidx, itmax);
            if (na.pit) atomicAdd(na.pit, itsum * (unsigned long long)a.sub_n[j]);
        }
    }
    if (bad) atomicOr(a.status, ST_NONFINITE);
    if (nl_fail && p == 0 && valid) atomicOr(a.status, ST_NL_NOCONV);
    cl.sync();   // keep this CTA's shared memory alive until every CTA of the cluster is done
}

template <int L>
static int launch_nl_t(NlArgs na, int ngroups, cudaStream_t s, int mode) {
    // the previous three steps' iterates ([L][T] and separators each)
    int smem = swr_march_nl_smem_bytes(na.m.T, na.m.G) +
               3 * (int)sizeof(double2) * (L * na.m.T + na.m.T + na.m.G);
    if (mode == 2)   // forward values of the step: [L][T], separators, chunk ends
        smem += (int)sizeof(double2) * (L * na.m.T + (na.m.T + na.m.G) + 2 * na.m.T);
    void (*kern)(const NlArgs) = k_march_nl<L, 0>;
    if (mode == 1) kern = k_march_nl<L, 1>;
    if (mode == 2) kern = k_march_nl<L, 2>;
    // one system spread over a cluster with its two-level separator data: the two-level
    // solve (Robin or Neumann ends).  A system alone in its CTA keeps the CTA-wide PCR,
    // which measured faster there (its levels cost a CTA barrier, not a cluster one).
    const MarchArgs& m = na.m;
    if (m.tl_pcr && m.two_level && !m.s02 && !m.kap && m.C > 1 && (m.T & 31) == 0 &&
        (m.tl_rs == 32 || m.T >= m.tl_rs)) {
        kern = (mode == 2) ? k_march_nl_tl<L, 2>
                           : ((mode == 1) ? k_march_nl_tl<L, 1> : k_march_nl_tl<L, 0>);
        smem = swr_march_nl_tl_smem_bytes(L, m.T, m.tl_rs, mode);
    }
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
        return -1;
    if (na.m.C > 8 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return -1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ngroups * na.m.C);
    cfg.blockDim = dim3(na.m.T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = na.m.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    swr_count_launch(1);
    return cudaLaunchKernelEx(&cfg, kern, na) == cudaSuccess ? 0 : -1;
}

int swr_launch_march_nl(const FactorSet& fs, MarchArgs a, double cw, double coef, double tol,
                        int maxit, int* iters, int ngroups, cudaStream_t s, int mode,
                        unsigned long long* pit) {
    if (mode != 0 && a.s02) return -2;   // the adjoint modes: Robin or Neumann ends
    if (a.kap) return -2;                // higher-order conditions: V(x) only
    a.P = fs.P;
    a.levels = fs.levels;
    a.sub_P = fs.sub_P;
    a.sep_pos = fs.sep_pos;
    a.clen = fs.clen;
    a.fac = fs.fac;
    a.sep = fs.sep;
    a.pcr = fs.pcr;
    a.tl_pcr = fs.tl_ok ? fs.tl_pcr : nullptr;
    a.tl_aux = fs.tl_aux;
    a.tl_red = fs.tl_red;
    a.tl_rs = fs.tl_rs;
    a.tl_rl = fs.tl_rl;
    NlArgs na{a, cw, coef, tol, maxit, iters, pit};
    switch (fs.L) {
        case 2: return launch_nl_t<2>(na, ngroups, s, mode);
        case 4: return launch_nl_t<4>(na, ngroups, s, mode);
        case 8: return launch_nl_t<8>(na, ngroups, s, mode);
        default: return -2;
    }
}
