// Subdomain Crank-Nicolson marches of the SWR method (Besse & Xing, Section 2.2).
//
// Each march solves, for n = 1..nt, the subdomain system of Eq. AvML
//     (A_j - B_j) v_n = (2i/dt) M_j u_{n-1} - Q_j^T (l_n, r_n)^T,   u_n = 2 v_n - u_{n-1},
// with the Robin boundary matrix B_j = p Q_j^T Q_j at ends that carry a
// transmission condition, and emits the fluxes of Eq. TransmisionCond
//     r_{j-1,n} = -l_{j,n} + 2 p v_n(a_j),      l_{j+1,n} = -r_{j,n} + 2 p v_n(b_j).
//
// GB300 design.  FP64 on this part runs at about 1/64 of the FP32 rate and a
// partially filled warp costs the FP64 pipe as much as a full one, so the march
// is FP64-ALU bound and needs many full warps.  One thread per right-hand side
// (plain Thomas) gives at most a few thousand threads; instead every tridiagonal
// system is cut into P chunks of <= L interior nodes separated by single
// separator nodes (a SPIKE-type partition):
//   * the chunk state u (L complex values) lives in registers for all nt steps;
//   * each chunk is solved with its own precomputed LU (2 complex factors per
//     node) and corrected with two precomputed spikes (the chunk's responses to
//     its two separators);
//   * the P+1 separator unknowns form a tridiagonal Schur complement with a
//     constant matrix, solved each step by parallel cyclic reduction (PCR) whose
//     per-level coefficients are precomputed, so a step only updates right-hand
//     sides (2 complex FMAs per separator and level);
//   * a CTA carries G systems (short subdomains) or one system is spread over a
//     thread-block cluster of C CTAs (long subdomains), the separators being read
//     through distributed shared memory.
// The system is pre-scaled by 1/(i kappa), kappa = (2/dt)(h/6), so that the
// right-hand side (2i/dt) M u becomes the integer stencil u_{i-1} + 4 u_i + u_{i+1}.
#include <cooperative_groups.h>

#include <algorithm>

#include "swr_internal.cuh"

namespace cg = cooperative_groups;

__device__ __forceinline__ void prefetch_l2(const void* ptr) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
}
// 16-byte asynchronous global -> shared copy (bypassing L1) and its group control
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Assembly of A_j - B_j (P1 elements, generalised mass by exact quadrature of the
// P1 interpolant of W), scaled by 1/(i kappa).  dg[loff_j + i] is the diagonal,
// od[loff_j + i] the coupling of local nodes i and i+1.
// ---------------------------------------------------------------------------
__global__ void k_assemble_static(const double* __restrict__ V, long long vstride,
                                  const int* __restrict__ n_, const int* __restrict__ goff_,
                                  const int* __restrict__ loff_, const int* __restrict__ tc_,
                                  double h, double dt, double2 sigma0, double2 inv_ik,
                                  double2* __restrict__ dg, double2* __restrict__ od,
                                  long long ldd, const double2* __restrict__ kap = nullptr,
                                  int kstride = 0) {
    const int j = blockIdx.y;
    const int n = n_[j];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // batch entry z: W = (V row z + V row z+1) / 2 (vstride = 0: the single row V)
    const double* V0 = V ? V + (size_t)blockIdx.z * vstride : nullptr;
    const double* V1 = V ? V0 + vstride : nullptr;
    auto W = [&](int gg) -> double { return V ? 0.5 * (V0[gg] + V1[gg]) : 0.0; };
    dg += (size_t)blockIdx.z * ldd;
    od += (size_t)blockIdx.z * ldd;
    const int g = goff_[j] + i;
    const int lo = loff_[j] + i;
    const int tc = tc_[j];
    const double W0 = W(g);
    double md = 0.0, sd = 0.0, wd = 0.0;
    if (i > 0) {
        const double Wm = W(g - 1);
        md += h / 3.0;
        sd += 1.0 / h;
        wd += h / 12.0 * (Wm + 3.0 * W0);
    }
    if (i < n - 1) {
        const double Wp = W(g + 1);
        md += h / 3.0;
        sd += 1.0 / h;
        wd += h / 12.0 * (3.0 * W0 + Wp);
    }
    double2 D = make_double2(-sd + wd, 2.0 / dt * md);
    // the end's boundary entry: sigma0, or the lag-0 entry of its own kernel
    if (i == 0 && (tc & 1)) D = csub(D, kap ? kap[(size_t)(2 * j + 0) * kstride] : sigma0);
    if (i == n - 1 && (tc & 2)) D = csub(D, kap ? kap[(size_t)(2 * j + 1) * kstride] : sigma0);
    dg[lo] = cmul(D, inv_ik);
    if (i < n - 1) {
        const double Wp = W(g + 1);
        const double2 E = make_double2(1.0 / h + h / 12.0 * (W0 + Wp), 2.0 / dt * (h / 6.0));
        od[lo] = cmul(E, inv_ik);
    } else {
        od[lo] = make_double2(0.0, 0.0);
    }
}

// Kernels of the higher-order transmission operators for V(x) (Section 2.2).  End
// e = 2 j + side of subdomain j sits on node g with potential W = V[g] and outward
// derivative d_nW = +-(V[g+1] - V[g-1]) / 2h (+ at the right end).  For V(x) every
// operator is a convolution of the end trace, S-bar v_n = sum_s k[n-s] h_s, with
// h_s = v_s (s >= 1) and h_0 = rho v_0:
//   S_0^3: k_m = c2 beta_m - e^{i pi/4} sqrt(dt/2) (W/2) alpha_m,            rho = 1;
//   S_0^4: S_0^3's k_m - i (d_nW/4) (dt/2) gamma_m,                          rho = 1;
//   S_1^2: k_m = c2 beta_m e^{i m dt W}, since e^{i Wc_n} e^{-i Wc_s} = e^{i (n-s) dt W}
//          for s >= 1 (Wc_n = (n - 1/2) dt W) and e^{i n dt W} e^{-i dt W/2} for s = 0
//          (Wc_0 = 0):                                                      rho = e^{-i dt W/2};
//   S_1^4: k_m = [c2 beta_m - i (d_nW/4) (dt/2) gamma_m] e^{i m dt W}: sgn(d_nW) times the
//          product of the two sqrt(|d_nW|)/2 factors is d_nW/4;              rho as S_1^2.
// alpha_m = |beta_m|, gamma = (1, 2, 2, ...).  kout is the flux update's operator, the
// sum of this end's kernel and the neighbour's at the same node (same W, opposite
// d_nW).  One thread per (end, m).
__device__ __forceinline__ double2 tc_kernel_entry(int tc, int m, double b, double W, double dn,
                                                   double dt, double2 c2) {
    const double al = fabs(b), ga = (m == 0) ? 1.0 : 2.0;
    double2 k = make_double2(c2.x * b, c2.y * b);
    if (tc == 2 || tc == 3) {   // S_0^3, S_0^4
        const double r = sqrt(0.5 * dt) * 0.5 * W * al;   // e^{i pi/4} = (1 + i) / sqrt(2)
        k.x -= r * 0.70710678118654752440;
        k.y -= r * 0.70710678118654752440;
        if (tc == 3) k.y -= 0.25 * dn * 0.5 * dt * ga;   // - i (d_nW/4)(dt/2) gamma
        return k;
    }
    if (tc == 5) k.y -= 0.25 * dn * 0.5 * dt * ga;      // S_1^4
    double sn, cs;
    sincos((double)m * dt * W, &sn, &cs);
    return make_double2(k.x * cs - k.y * sn, k.x * sn + k.y * cs);
}

__global__ void k_tc_kernels(int tc, const double* __restrict__ V, int N,
                             const int* __restrict__ n_, const int* __restrict__ goff_,
                             const int* __restrict__ tc_, int kstride, double h, double dt,
                             const double* __restrict__ beta, double2 c2,
                             double2* __restrict__ kap, double2* __restrict__ kout,
                             double2* __restrict__ rho) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int e = blockIdx.y;
    const int j = e >> 1, side = e & 1;
    if (m >= kstride || j >= N || !(tc_[j] & (1 << side))) return;
    const int g = goff_[j] + (side ? n_[j] - 1 : 0);    // an interior node of the whole grid
    const double W = V[g];
    const double dn = (V[g + 1] - V[g - 1]) / (2.0 * h) * (side ? 1.0 : -1.0);
    const double2 k1 = tc_kernel_entry(tc, m, beta[m], W, dn, dt, c2);
    const double2 k2 = tc_kernel_entry(tc, m, beta[m], W, -dn, dt, c2);
    kap[(size_t)e * kstride + m] = k1;
    kout[(size_t)e * kstride + m] = make_double2(k1.x + k2.x, k1.y + k2.y);
    if (m == 0) {
        if (tc >= 4) {
            double sn, cs;
            sincos(-0.5 * dt * W, &sn, &cs);
            rho[e] = make_double2(cs, sn);
        } else {
            rho[e] = make_double2(1.0, 0.0);
        }
    }
}

int swr_launch_tc_kernels(int tc, const double* V, int N, const int* d_n, const int* d_goff,
                          const int* d_tc, int kstride, double h, double dt, const double* beta,
                          double2 c2, double2* kap, double2* kout, double2* rho, cudaStream_t s) {
    if (tc < 2 || tc > 5) return -2;
    dim3 grid((kstride + 255) / 256, 2 * N);
    k_tc_kernels<<<grid, 256, 0, s>>>(tc, V, N, d_n, d_goff, d_tc, kstride, h, dt, beta, c2, kap,
                                      kout, rho);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Vbar(x) = mean over the nrows rows of V (time average of a tabulated V(t,x)).
__global__ void k_row_mean(const double* __restrict__ V, int nrows, long long nx,
                           double* __restrict__ out) {
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    double acc = 0.0;
    for (int r = 0; r < nrows; ++r) acc += V[(size_t)r * nx + x];
    out[x] = acc / nrows;
}

int swr_launch_row_mean(const double* V, int nrows, long long nx, double* out, cudaStream_t s) {
    k_row_mean<<<(unsigned)((nx + 255) / 256), 256, 0, s>>>(V, nrows, nx, out);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int swr_launch_assemble_static(const double* V, int N, const int* d_n, const int* d_goff,
                               const int* d_loff, const int* d_tc, int nmax, double h, double dt,
                               double2 sigma0, double2 inv_ik, double2* dg, double2* od,
                               cudaStream_t s, const double2* kap, int kstride) {
    dim3 grid((nmax + 255) / 256, N);
    k_assemble_static<<<grid, 256, 0, s>>>(V, 0, d_n, d_goff, d_loff, d_tc, h, dt, sigma0, inv_ik,
                                           dg, od, 0, kap, kstride);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// Chunking, chunk LU and spikes.  One thread per (subdomain, chunk).
// Subdomain with n nodes: Pj = ceil((n-1)/(L+1)) chunks, separators at local
// nodes sep_0 = 0 < sep_1 < ... < sep_Pj = n-1, interior counts differing by at
// most one.  Chunks p >= Pj are dummies (no interior).
// ---------------------------------------------------------------------------
template <int L>
__global__ void k_factor_chunks(int N, int P, const int* __restrict__ n_,
                                const int* __restrict__ loff_, const double2* __restrict__ dg,
                                const double2* __restrict__ od, int* __restrict__ sub_P,
                                int* __restrict__ sep_pos, unsigned char* __restrict__ clen,
                                double2* __restrict__ fac, double2* __restrict__ tips,
                                int* status, long long ldd, long long fstride) {
    const int j = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    // batch entry z (per-step factorisations): its own dg/od, fac and tips
    const int z = blockIdx.z;
    dg += (size_t)z * ldd;
    od += (size_t)z * ldd;
    fac += (size_t)z * fstride;
    tips += (size_t)z * N * P * 4;
    const int n = n_[j];
    const int Pj = (n - 1 + L) / (L + 1);
    const int interior = n - 1 - Pj;
    const int q = interior / Pj, rem = interior % Pj;
    int Lp, sp;
    if (p < Pj) {
        Lp = q + (p < rem ? 1 : 0);
        sp = p + p * q + (p < rem ? p : rem);
    } else {
        Lp = 0;
        sp = n - 1;
    }
    if (z == 0) {
        if (p == 0) sub_P[j] = Pj;
        sep_pos[j * (P + 1) + p] = sp;
        if (p == P - 1) sep_pos[j * (P + 1) + P] = n - 1;
        clen[j * P + p] = (unsigned char)Lp;
    }
    const double2 zero = make_double2(0.0, 0.0);
    double2* F = fac + (size_t)j * L * 4 * P;
    if (Lp == 0) {
#pragma unroll
        for (int i = 0; i < L; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) F[(i * 4 + k) * P + p] = zero;
#pragma unroll
        for (int k = 0; k < 4; ++k) tips[((size_t)j * P + p) * 4 + k] = zero;
        return;
    }
    const double2* D = dg + loff_[j] + sp + 1;   // interior diagonal
    const double2* E = od + loff_[j] + sp + 1;   // E[i]: coupling i <-> i+1 (i = Lp-1: to sep p+1)
    const double2 Es = od[loff_[j] + sp];        // separator p <-> first interior
    double2 qv[L], cv[L];
    bool bad = false;
    double2 piv = D[0];
#pragma unroll
    for (int i = 0; i < L; ++i) {
        if (i < Lp) {
            if (i > 0) piv = cfms(E[i - 1], cv[i - 1], D[i]);
            bad |= !cfinite(piv) || (piv.x == 0.0 && piv.y == 0.0);
            qv[i] = crcp(piv);
            cv[i] = (i < Lp - 1) ? cmul(E[i], qv[i]) : zero;
        }
    }
    const double2 El = E[Lp - 1];
    // spike a = T^{-1}(Es e_0): forward z_0 = Es, z_i = -c_{i-1} z_{i-1}
    double2 za[L];
#pragma unroll
    for (int i = 0; i < L; ++i) {
        if (i < Lp) za[i] = (i == 0) ? Es : cfms(cv[i - 1], za[i - 1], zero);
    }
    double2 anext = zero, bnext = zero, a0 = zero, b0 = zero, aL = zero, bL = zero;
#pragma unroll
    for (int i = L - 1; i >= 0; --i) {
        if (i < Lp) {
            double2 ai, bi;
            if (i == Lp - 1) {
                ai = cmul(qv[i], za[i]);
                bi = cmul(qv[i], El);
                aL = ai;
                bL = bi;
            } else {
                ai = cfms(cv[i], anext, cmul(qv[i], za[i]));
                bi = cfms(cv[i], bnext, zero);
            }
            anext = ai;
            bnext = bi;
            if (i == 0) {
                a0 = ai;
                b0 = bi;
            }
            F[(i * 4 + 0) * P + p] = qv[i];
            F[(i * 4 + 1) * P + p] = cv[i];
            F[(i * 4 + 2) * P + p] = ai;
            F[(i * 4 + 3) * P + p] = bi;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) F[(i * 4 + k) * P + p] = zero;
        }
    }
    double2* tp = tips + ((size_t)j * P + p) * 4;
    tp[0] = a0;
    tp[1] = b0;
    tp[2] = aL;
    tp[3] = bL;
    if (bad) atomicOr(status, ST_SINGULAR);
}

// Reduced (separator) system and its PCR coefficients; one CTA per subdomain,
// threads strided over the separators, one barrier per PCR level.
// Row ps: E_{s-1} v_{s-1} + D_s v_s + E_s v_{s+1} = f_s with the neighbouring
// interiors eliminated through the chunk spikes:
//   delta = D_s - E_{s-1} b^{ps-1}_last - E_s a^{ps}_first,
//   lower = -E_{s-1} a^{ps-1}_last,  upper = -E_s b^{ps}_first,
//   rhs   = f_s - E_{s-1} y^{ps-1}_last - E_s y^{ps}_first.
// PCR (stride 2^k): alpha = -lower/delta_{p-st}, gamma = -upper/delta_{p+st}.
__global__ void k_reduce_pcr(int N, int P, int levels, const int* __restrict__ loff_,
                             const double2* __restrict__ dg, const double2* __restrict__ od,
                             const int* __restrict__ sub_P, const int* __restrict__ sep_pos,
                             const double2* __restrict__ tips, double2* __restrict__ sep,
                             double2* __restrict__ pcr, double2* __restrict__ red,
                             int* status, long long ldd, long long sstride, long long pstride) {
    const int j = blockIdx.x;
    if (j >= N) return;
    const int z = blockIdx.y;   // batch entry (per-step factorisations)
    dg += (size_t)z * ldd;
    od += (size_t)z * ldd;
    tips += (size_t)z * N * P * 4;
    sep += (size_t)z * sstride;
    pcr += (size_t)z * pstride;
    red += (size_t)z * N * 6 * (P + 1);
    const int Pj = sub_P[j];
    const int S = P + 1;
    const double2 zero = make_double2(0.0, 0.0);
    double2* lo = red + (size_t)(j * 6 + 0) * S;
    double2* dd = red + (size_t)(j * 6 + 1) * S;
    double2* up = red + (size_t)(j * 6 + 2) * S;
    double2* lo2 = red + (size_t)(j * 6 + 3) * S;
    double2* dd2 = red + (size_t)(j * 6 + 4) * S;
    double2* up2 = red + (size_t)(j * 6 + 5) * S;
    double2* sE_l = sep + (size_t)(j * 3 + 0) * S;
    double2* sE_r = sep + (size_t)(j * 3 + 1) * S;
    double2* sbinv = sep + (size_t)(j * 3 + 2) * S;
    const double2* T = tips + (size_t)j * P * 4;
    const int base = loff_[j];
    for (int ps = threadIdx.x; ps <= P; ps += blockDim.x) {
        if (ps <= Pj) {
            const int s = sep_pos[j * S + ps];
            double2 d = dg[base + s], l = zero, u = zero;
            double2 EL = zero, ER = zero;
            if (ps > 0) {
                EL = od[base + s - 1];
                d = cfms(EL, T[(ps - 1) * 4 + 3], d);
                l = cmul(make_double2(-EL.x, -EL.y), T[(ps - 1) * 4 + 2]);
            }
            if (ps < Pj) {
                ER = od[base + s];
                d = cfms(ER, T[ps * 4 + 0], d);
                u = cmul(make_double2(-ER.x, -ER.y), T[ps * 4 + 1]);
            }
            lo[ps] = l;
            dd[ps] = d;
            up[ps] = u;
            sE_l[ps] = EL;
            sE_r[ps] = ER;
        } else {
            lo[ps] = zero;
            dd[ps] = make_double2(1.0, 0.0);
            up[ps] = zero;
            sE_l[ps] = zero;
            sE_r[ps] = zero;
        }
    }
    __syncthreads();
    for (int k = 0; k < levels; ++k) {
        const int st = 1 << k;
        double2* al = pcr + ((size_t)(j * levels + k) * 2 + 0) * S;
        double2* ga = pcr + ((size_t)(j * levels + k) * 2 + 1) * S;
        for (int ps = threadIdx.x; ps <= P; ps += blockDim.x) {
            double2 a = zero, g = zero, nl = zero, nu = zero, nd = dd[ps];
            if (ps - st >= 0) {
                const double2 r = crcp(dd[ps - st]);
                a = cmul(make_double2(-lo[ps].x, -lo[ps].y), r);
                nl = cmul(a, lo[ps - st]);
                nd = cfma(a, up[ps - st], nd);
            }
            if (ps + st <= P) {
                const double2 r = crcp(dd[ps + st]);
                g = cmul(make_double2(-up[ps].x, -up[ps].y), r);
                nu = cmul(g, up[ps + st]);
                nd = cfma(g, lo[ps + st], nd);
            }
            al[ps] = a;
            ga[ps] = g;
            lo2[ps] = nl;
            dd2[ps] = nd;
            up2[ps] = nu;
        }
        __syncthreads();
        double2* t;
        t = lo; lo = lo2; lo2 = t;
        t = dd; dd = dd2; dd2 = t;
        t = up; up = up2; up2 = t;
    }
    bool bad = false;
    for (int ps = threadIdx.x; ps <= P; ps += blockDim.x) {
        const double2 d = dd[ps];
        bad |= !cfinite(d) || (d.x == 0.0 && d.y == 0.0);
        sbinv[ps] = crcp(d);
    }
    if (bad) atomicOr(status, ST_SINGULAR);
}

// ---------------------------------------------------------------------------
// Two-level separator solve (clusters).  One CTA of 1024 threads per subdomain,
// thread p = separator p (P + 1 <= 993).  The separator rows are those of
// k_reduce_pcr: lo x_{p-1} + dd x_p + up x_{p+1} = d_p.  Warp q holds separators
// 32q .. 32q+31; its lane 0 (s_q = 32q) and the last separator Pj are
// super-separators, the others (lanes 1..m_q, m_q = min(31, Pj - 1 - 32q)) form
// super-chunk q.  With the super-separators known, a super-chunk is the tridiagonal
// system A_q x = d - lo e_first x_{s_q} - up e_last x_{s_{q+1}}, solved as
// x = yhat - a x_{s_q} - b x_{s_{q+1}} (yhat = A_q^{-1} d by PCR, spikes a, b);
// substituting the neighbouring super-chunks' first/last rows into row s_q gives a
// tridiagonal system in the super-separators:
//   RL_q x_{s_{q-1}} + RD_q x_{s_q} + RU_q x_{s_{q+1}}
//       = d_{s_q} - cL_q yhat_last(q-1) - cU_q yhat_first(q),
//   RL = -lo a_{s-1} (lo when super-chunk q-1 is empty), RU = -up b_{s+1} (or up),
//   RD = dd - lo b_{s-1} - up a_{s+1} (terms of empty super-chunks dropped),
//   cL = lo, cU = up (0 for an empty super-chunk).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 shfl_up2(double2 v, int d) {
    return make_double2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ double2 shfl_down2(double2 v, int d) {
    return make_double2(__shfl_down_sync(0xffffffffu, v.x, d),
                        __shfl_down_sync(0xffffffffu, v.y, d));
}

// PCR coefficients of a tridiagonal system held one row per lane (rows outside
// [lo_lane, hi_lane] are absent): alpha/gamma of level k into co[(2k) cs], co[(2k+1) cs]
// (when `store`), and the decoupled diagonal into dfin.  Spike right-hand sides e1, e2
// are carried along.
__device__ void warp_pcr_coeffs(double2 L, double2 D, double2 U, int lane, int lo_lane,
                                int hi_lane, double2* co, size_t cs, bool store, double2& e1,
                                double2& e2, double2& dfin) {
    const double2 zero = make_double2(0.0, 0.0);
    const bool in = lane >= lo_lane && lane <= hi_lane;
    if (!in) {
        L = zero;
        U = zero;
        D = make_double2(1.0, 0.0);
        e1 = zero;
        e2 = zero;
    }
    for (int k = 0; k < 5; ++k) {
        const int st = 1 << k;
        const double2 Lm = shfl_up2(L, st), Dm = shfl_up2(D, st), Um = shfl_up2(U, st);
        const double2 Lp = shfl_down2(L, st), Dp = shfl_down2(D, st), Up = shfl_down2(U, st);
        const double2 e1m = shfl_up2(e1, st), e1p = shfl_down2(e1, st);
        const double2 e2m = shfl_up2(e2, st), e2p = shfl_down2(e2, st);
        double2 a = zero, g = zero;
        if (in && lane - st >= lo_lane) a = cmul(make_double2(-L.x, -L.y), crcp(Dm));
        if (in && lane + st <= hi_lane) g = cmul(make_double2(-U.x, -U.y), crcp(Dp));
        const double2 nL = cmul(a, Lm), nU = cmul(g, Up);
        const double2 nD = cfma(g, Lp, cfma(a, Um, D));
        e1 = cfma(g, e1p, cfma(a, e1m, e1));
        e2 = cfma(g, e2p, cfma(a, e2m, e2));
        if (store) {
            co[(size_t)(2 * k) * cs] = a;
            co[(size_t)(2 * k + 1) * cs] = g;
        }
        L = nL;
        D = nD;
        U = nU;
    }
    dfin = D;
}

// Two-level separator data of one system per CTA (blockIdx.x = subdomain j).  Warp w
// takes the warp blocks w, w + nw, ... of 32 separators: the separator rows (as
// k_reduce_pcr), the super-chunk PCR coefficients and spikes of each block, and the
// rows of its super-separator; then the reduced system over the Q + 1 super-separators:
// with RS = 32 (Q <= 31) by warp 0 with shuffles, otherwise by the whole CTA with one
// barrier per PCR level (RS <= blockDim.x).  tl_red [N][2 RL + 3][RS]: RL levels of
// (alpha, gamma), 1/delta, and the weights of y_last(q-1), y_first(q) in the rows.
// Dynamic shared memory: 13 RS double2.
__global__ void __launch_bounds__(1024, 1) k_factor_two_level(
    int N, int P, const int* __restrict__ loff_, const double2* __restrict__ dg,
    const double2* __restrict__ od, const int* __restrict__ sub_P,
    const int* __restrict__ sep_pos, const double2* __restrict__ tips,
    double2* __restrict__ tl_pcr, double2* __restrict__ tl_aux, double2* __restrict__ tl_red,
    int RS, int RL, int* status) {
    // per super-separator q: its row (lo, dd, up); per super-chunk q: the spikes at its
    // first member (af, bf) and last member (al, bl); wide reduced PCR: rows L, D, U
    extern __shared__ double2 fsm[];
    double2 *s_lo = fsm, *s_dd = s_lo + RS, *s_up = s_dd + RS, *s_af = s_up + RS;
    double2 *s_bf = s_af + RS, *s_al = s_bf + RS, *s_bl = s_al + RS;
    double2 *w_l = s_bl + RS, *w_d = w_l + RS, *w_u = w_d + RS;
    const int j = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int Pj = sub_P[j];
    const int S = P + 1;
    const int Q = (Pj + 31) / 32;
    const double2 zero = make_double2(0.0, 0.0), one = make_double2(1.0, 0.0);
    const double2* T = tips + (size_t)j * P * 4;
    const int base = loff_[j];
    bool bad = false;
    const int nblk = (S + 31) / 32;
    for (int q = wid; q < nblk; q += nw) {   // uniform per warp
        const int p = 32 * q + lane;
        // separator rows (as k_reduce_pcr); padding beyond Pj: identity rows
        double2 lo = zero, dd = one, up = zero;
        if (p <= Pj) {
            const int s = sep_pos[j * S + p];
            dd = dg[base + s];
            if (p > 0) {
                const double2 EL = od[base + s - 1];
                dd = cfms(EL, T[(p - 1) * 4 + 3], dd);
                lo = cmul(make_double2(-EL.x, -EL.y), T[(p - 1) * 4 + 2]);
            }
            if (p < Pj) {
                const double2 ER = od[base + s];
                dd = cfms(ER, T[p * 4 + 0], dd);
                up = cmul(make_double2(-ER.x, -ER.y), T[p * 4 + 1]);
            }
        }
        // super-separator rows: s_q = 32 q (q < Q) and s_Q = Pj
        if ((lane == 0 && q < Q) || p == Pj) {
            const int qi = (p == Pj) ? Q : q;
            s_lo[qi] = lo;
            s_dd[qi] = dd;
            s_up[qi] = up;
        }
        // super-chunk q: lanes 1..m
        const int m = (32 * q < Pj) ? min(31, Pj - 1 - 32 * q) : 0;
        double2 e1 = (lane == 1) ? lo : zero, e2 = (lane == m) ? up : zero, dfin;
        const bool keep = p < S;
        warp_pcr_coeffs(lo, dd, up, lane, 1, m, tl_pcr + (size_t)j * 10 * S + (keep ? p : 0),
                        (size_t)S, keep, e1, e2, dfin);
        const bool member = lane >= 1 && lane <= m;
        double2 binv = one, sa = zero, sb = zero;
        if (member) {
            bad |= !cfinite(dfin) || (dfin.x == 0.0 && dfin.y == 0.0);
            binv = crcp(dfin);
            sa = cmul(e1, binv);
            sb = cmul(e2, binv);
        }
        if (keep) {
            tl_aux[((size_t)j * 3 + 0) * S + p] = binv;
            tl_aux[((size_t)j * 3 + 1) * S + p] = sa;
            tl_aux[((size_t)j * 3 + 2) * S + p] = sb;
        }
        if (member && lane == 1) {
            s_af[q] = sa;
            s_bf[q] = sb;
        }
        if (member && lane == m) {
            s_al[q] = sa;
            s_bl[q] = sb;
        }
    }
    __syncthreads();
    // reduced row of super-separator i (identity beyond Q): lower, diagonal, upper, and
    // the weights of the neighbouring super-chunks' end values in its right-hand side
    auto reduced_row = [&](int i, double2& RL_, double2& RD_, double2& RU_, double2& cL,
                           double2& cU) {
        RL_ = zero;
        RD_ = one;
        RU_ = zero;
        cL = zero;
        cU = zero;
        if (i > Q) return;
        const int sq = (i < Q) ? 32 * i : Pj;
        const int mprev = (i >= 1) ? sq - 1 - 32 * (i - 1) : 0;   // members of block i-1
        const int mcur = (i < Q) ? min(31, Pj - 1 - sq) : 0;       // members of block i
        RD_ = s_dd[i];
        if (i >= 1) {
            if (mprev > 0) {
                RL_ = cmul(make_double2(-s_lo[i].x, -s_lo[i].y), s_al[i - 1]);
                RD_ = cfms(s_lo[i], s_bl[i - 1], RD_);
                cL = s_lo[i];
            } else {
                RL_ = s_lo[i];
            }
        }
        if (i < Q) {
            if (mcur > 0) {
                RU_ = cmul(make_double2(-s_up[i].x, -s_up[i].y), s_bf[i]);
                RD_ = cfms(s_up[i], s_af[i], RD_);
                cU = s_up[i];
            } else {
                RU_ = s_up[i];
            }
        }
    };
    double2* R = tl_red + (size_t)j * (2 * RL + 3) * RS;
    if (RS == 32) {
        if (wid == 0) {
            double2 RL_, RD_, RU_, cL, cU;
            reduced_row(lane, RL_, RD_, RU_, cL, cU);
            double2 z1 = zero, z2 = zero, rfin;
            warp_pcr_coeffs(RL_, RD_, RU_, lane, 0, Q, R + lane, 32, true, z1, z2, rfin);
            double2 rinv = one;
            if (lane <= Q) {
                bad |= !cfinite(rfin) || (rfin.x == 0.0 && rfin.y == 0.0);
                rinv = crcp(rfin);
            }
            R[10 * 32 + lane] = rinv;
            R[11 * 32 + lane] = cL;
            R[12 * 32 + lane] = cU;
        }
    } else {
        // wide: thread i < RS holds reduced row i (blockDim.x >= RS)
        const int i = tid;
        double2 RL_ = zero, RD_ = one, RU_ = zero, cL = zero, cU = zero;
        if (i < RS) {
            reduced_row(i, RL_, RD_, RU_, cL, cU);
            w_l[i] = RL_;
            w_d[i] = RD_;
            w_u[i] = RU_;
        }
        __syncthreads();
        for (int k = 0; k < RL; ++k) {
            const int st = 1 << k;
            double2 al = zero, ga = zero, nL = zero, nD = RD_, nU = zero;
            if (i < RS) {
                if (i <= Q && i - st >= 0) al = cmul(make_double2(-RL_.x, -RL_.y), crcp(w_d[i - st]));
                if (i <= Q && i + st <= Q) ga = cmul(make_double2(-RU_.x, -RU_.y), crcp(w_d[i + st]));
                if (i - st >= 0) {
                    nL = cmul(al, w_l[i - st]);
                    nD = cfma(al, w_u[i - st], nD);
                }
                if (i + st < RS) {
                    nU = cmul(ga, w_u[i + st]);
                    nD = cfma(ga, w_l[i + st], nD);
                }
                R[(size_t)(2 * k) * RS + i] = al;
                R[(size_t)(2 * k + 1) * RS + i] = ga;
            }
            __syncthreads();
            if (i < RS) {
                RL_ = nL;
                RD_ = nD;
                RU_ = nU;
                w_l[i] = nL;
                w_d[i] = nD;
                w_u[i] = nU;
            }
            __syncthreads();
        }
        if (i < RS) {
            double2 rinv = one;
            if (i <= Q) {
                bad |= !cfinite(RD_) || (RD_.x == 0.0 && RD_.y == 0.0);
                rinv = crcp(RD_);
            }
            R[(size_t)(2 * RL) * RS + i] = rinv;
            R[(size_t)(2 * RL + 1) * RS + i] = cL;
            R[(size_t)(2 * RL + 2) * RS + i] = cU;
        }
    }
    if (bad) atomicOr(status, ST_SINGULAR);
}

int swr_launch_factor_tl(FactorSet& fs, int N, const int* d_loff, const double2* dg,
                         const double2* od, int* status, cudaStream_t s, bool wide) {
    fs.tl_ok = false;
    if (fs.nsteps != 1) return -2;
    const int S = fs.P + 1;
    if (S > (wide ? kTlMaxSepWide : kTlMaxSep)) return -2;
    const int Qmax = (fs.P + 31) / 32;
    const int RS = (Qmax + 1 <= 32) ? 32 : ((Qmax + 1 + 31) / 32) * 32;
    int RL = 0;
    while ((1 << RL) < RS) ++RL;
    if (!fs.tl_pcr) {   // wide data of a system beyond kTlMaxSep separators: on request
        bool ok = cudaMalloc(&fs.tl_pcr, sizeof(double2) * (size_t)N * 10 * S) == cudaSuccess;
        ok &= cudaMalloc(&fs.tl_aux, sizeof(double2) * (size_t)N * 3 * S) == cudaSuccess;
        ok &= cudaMalloc(&fs.tl_red, sizeof(double2) * (size_t)N * (2 * RL + 3) * RS) ==
              cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return -1;
        }
    }
    fs.tl_rs = RS;
    fs.tl_rl = RL;
    const int threads = std::min(1024, std::max(RS, ((S + 31) / 32) * 32));
    k_factor_two_level<<<N, threads, sizeof(double2) * 13 * RS, s>>>(
        N, fs.P, d_loff, dg, od, fs.sub_P, fs.sep_pos, fs.tips, fs.tl_pcr, fs.tl_aux, fs.tl_red,
        RS, RL, status);
    swr_count_launch(1);
    if (cudaGetLastError() != cudaSuccess) return -1;
    fs.tl_ok = true;
    return 0;
}

static int ilog2ceil(int v) {
    int k = 0;
    while ((1 << k) < v) ++k;
    return k;
}

size_t swr_factor_step_bytes(int N, int L, int P) {
    const size_t S = P + 1;
    const int levels = std::max(1, ilog2ceil(P + 1));
    return sizeof(double2) * ((size_t)N * L * 4 * P + (size_t)N * 3 * S + (size_t)N * levels * 2 * S);
}

int swr_factor_alloc(FactorSet& fs, int N, int L, int P, cudaStream_t, int nsteps, long long ldd) {
    swr_factor_free(fs);
    fs.L = L;
    fs.P = P;
    fs.levels = ilog2ceil(P + 1);
    if (fs.levels < 1) fs.levels = 1;
    const size_t S = P + 1;
    fs.nsteps = std::max(1, nsteps);
    fs.batch = std::min(fs.nsteps, 64);
    const size_t fst = (size_t)N * L * 4 * P, sst = (size_t)N * 3 * S;
    const size_t pst = (size_t)N * fs.levels * 2 * S;
    if (fs.nsteps > 1) {
        fs.fstride = (long long)fst;
        fs.sstride = (long long)sst;
        fs.pstride = (long long)pst;
        fs.ldd = ldd;
    }
    const size_t ns = fs.nsteps, nb = fs.batch;
    bool ok = true;
    ok &= cudaMalloc(&fs.sub_P, sizeof(int) * N) == cudaSuccess;
    ok &= cudaMalloc(&fs.sep_pos, sizeof(int) * N * S) == cudaSuccess;
    ok &= cudaMalloc(&fs.clen, (size_t)N * P) == cudaSuccess;
    ok &= cudaMalloc(&fs.fac, sizeof(double2) * fst * ns) == cudaSuccess;
    ok &= cudaMalloc(&fs.tips, sizeof(double2) * (size_t)N * P * 4 * nb) == cudaSuccess;
    ok &= cudaMalloc(&fs.sep, sizeof(double2) * sst * ns) == cudaSuccess;
    ok &= cudaMalloc(&fs.pcr, sizeof(double2) * pst * ns) == cudaSuccess;
    ok &= cudaMalloc(&fs.red, sizeof(double2) * (size_t)N * 6 * S * nb) == cudaSuccess;
    if (fs.nsteps > 1) {
        ok &= cudaMalloc(&fs.dgb, sizeof(double2) * (size_t)ldd * nb) == cudaSuccess;
        ok &= cudaMalloc(&fs.odb, sizeof(double2) * (size_t)ldd * nb) == cudaSuccess;
    } else if (S <= (size_t)kTlMaxSep) {
        // the two-level separator data of cluster-spread systems
        ok &= cudaMalloc(&fs.tl_pcr, sizeof(double2) * (size_t)N * 10 * S) == cudaSuccess;
        ok &= cudaMalloc(&fs.tl_aux, sizeof(double2) * (size_t)N * 3 * S) == cudaSuccess;
        ok &= cudaMalloc(&fs.tl_red, sizeof(double2) * (size_t)N * 13 * 32) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();   // clear the allocation error
        swr_factor_free(fs);
        return -1;
    }
    return 0;
}

void swr_factor_free(FactorSet& fs) {
    cudaFree(fs.sub_P);
    cudaFree(fs.sep_pos);
    cudaFree(fs.clen);
    cudaFree(fs.fac);
    cudaFree(fs.tips);
    cudaFree(fs.sep);
    cudaFree(fs.pcr);
    cudaFree(fs.red);
    cudaFree(fs.dgb);
    cudaFree(fs.odb);
    cudaFree(fs.tl_pcr);
    cudaFree(fs.tl_aux);
    cudaFree(fs.tl_red);
    fs = FactorSet();
}

// One batch of nb steps (or the single constant matrix, nb = 1 and zero strides).
static int launch_factor_batch(FactorSet& fs, int N, const int* d_n, const int* d_loff,
                               const double2* dg, const double2* od, long long ldd, int t0,
                               int nb, int* status, cudaStream_t s) {
    dim3 grid((fs.P + 127) / 128, N, nb);
    double2* fac = fs.fac + (size_t)t0 * fs.fstride;
    switch (fs.L) {
        case 2:
            k_factor_chunks<2><<<grid, 128, 0, s>>>(N, fs.P, d_n, d_loff, dg, od, fs.sub_P,
                                                    fs.sep_pos, fs.clen, fac, fs.tips, status, ldd,
                                                    fs.fstride);
            break;
        case 4:
            k_factor_chunks<4><<<grid, 128, 0, s>>>(N, fs.P, d_n, d_loff, dg, od, fs.sub_P,
                                                    fs.sep_pos, fs.clen, fac, fs.tips, status, ldd,
                                                    fs.fstride);
            break;
        case 8:
            k_factor_chunks<8><<<grid, 128, 0, s>>>(N, fs.P, d_n, d_loff, dg, od, fs.sub_P,
                                                    fs.sep_pos, fs.clen, fac, fs.tips, status, ldd,
                                                    fs.fstride);
            break;
        case 12:
            k_factor_chunks<12><<<grid, 128, 0, s>>>(N, fs.P, d_n, d_loff, dg, od, fs.sub_P,
                                                     fs.sep_pos, fs.clen, fac, fs.tips, status,
                                                     ldd, fs.fstride);
            break;
        case 16:
            k_factor_chunks<16><<<grid, 128, 0, s>>>(N, fs.P, d_n, d_loff, dg, od, fs.sub_P,
                                                     fs.sep_pos, fs.clen, fac, fs.tips, status,
                                                     ldd, fs.fstride);
            break;
        default:
            return -2;
    }
    if (cudaGetLastError() != cudaSuccess) return -1;
    k_reduce_pcr<<<dim3(N, nb), 256, 0, s>>>(N, fs.P, fs.levels, d_loff, dg, od, fs.sub_P,
                                             fs.sep_pos, fs.tips, fs.sep + (size_t)t0 * fs.sstride,
                                             fs.pcr + (size_t)t0 * fs.pstride, fs.red, status, ldd,
                                             fs.sstride, fs.pstride);
    swr_count_launch(2);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int swr_launch_factor(FactorSet& fs, int N, const int* d_n, const int* d_loff, const double2* dg,
                      const double2* od, int* status, cudaStream_t s) {
    if (fs.nsteps != 1) return -2;
    return launch_factor_batch(fs, N, d_n, d_loff, dg, od, 0, 0, 1, status, s);
}

int swr_launch_factor_steps(FactorSet& fs, int N, const int* d_n, const int* d_goff,
                            const int* d_loff, const int* d_tc, int nmax, const double* V,
                            long long vstride, double h, double dt, double2 sigma0,
                            double2 inv_ik, int* status, cudaStream_t s) {
    if (fs.nsteps < 2 || !fs.dgb || !V) return -2;
    for (int t0 = 0; t0 < fs.nsteps; t0 += fs.batch) {
        const int nb = std::min(fs.batch, fs.nsteps - t0);
        dim3 grid((nmax + 255) / 256, N, nb);
        k_assemble_static<<<grid, 256, 0, s>>>(V + (size_t)t0 * vstride, vstride, d_n, d_goff,
                                               d_loff, d_tc, h, dt, sigma0, inv_ik, fs.dgb, fs.odb,
                                               fs.ldd);
        swr_count_launch(1);
        if (cudaGetLastError() != cudaSuccess) return -1;
        const int rc = launch_factor_batch(fs, N, d_n, d_loff, fs.dgb, fs.odb, fs.ldd, t0, nb,
                                           status, s);
        if (rc) return rc;
    }
    return 0;
}

// ---------------------------------------------------------------------------
// The march kernel.
// Each system has P+1 threads: thread p owns separator p and, for p < P, chunk p.
// C == 1: the CTA carries G systems, thread tid -> system g = tid / (P+1).
// C > 1:  one system per cluster, p = rank * T + tid.
// Shared memory (per CTA): separator values usep, PCR ping-pong dA/dB
// ([T+G] each) and, per chunk, the first/last interior u and y ([T] each).
// ---------------------------------------------------------------------------
int swr_march_smem_bytes(int T, int G, int stage_slots) {
    return (int)sizeof(double2) * (3 * (T + G) + 4 * T + 4 * G + stage_slots * T);
}

// MODE 0: march; 1: also record v of every step; 2: also accumulate the adjoint
// potential form against recorded forward values (see MarchArgs).
// GEN: the ends carry per-end kernels (a.kap, a.kout, a.rho: S_0^3, S_0^4, S_1^2, S_1^4),
// a separate instantiation so that Robin and S_0^2 marches keep their registers.
// LEAN: systems held by one CTA (C == 1) with Robin or Neumann ends (no S_0^2 history):
// the cluster and history paths compiled out, which halves the register spills of the
// 12-node chunks under their 168-register budget.
template <int L, int MODE, bool GEN = false, bool LEAN = false>
__global__ void __launch_bounds__((L == 16 || MODE == 2) ? 256 : 384, 1) k_march_static(const MarchArgs a) {
    extern __shared__ double2 sm[];
    const int T = a.T, G = a.G, P = a.P, nt = a.nt, levels = a.levels;
    const int C = LEAN ? 1 : a.C;
    const bool s02v = !LEAN && a.s02;   // S_0^2 history terms
    const int S = T + G;
    double2* usep = sm;
    double2* dA = usep + S;
    double2* dB = dA + S;
    double2* ufst = dB + S;
    double2* ulst = ufst + T;
    double2* yfst = ulst + T;
    double2* ylst = yfst + T;
    double2* hsum = ylst + T;        // [2G] S_0^2 history sums of this step (C > 1: [2])
    double2* hsum2 = hsum + 2 * G;   // [2G] flux-update history sums (per-end kernels)
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (C > 1) ? (int)cl.block_rank() : 0;
    const int tid = threadIdx.x;
    int g, p, sidx;
    // ragged packing: this CTA's systems and the first thread of each
    const bool ragged = (C == 1) && a.rag;
    int re0 = 0, rne = 0, rbase = 0;
    if (ragged) {
        re0 = a.rag_start[blockIdx.x];
        rne = a.rag_start[blockIdx.x + 1] - re0;
        g = -1;
        p = -1;
        sidx = a.nsys;
        for (int q = 0; q < rne; ++q) {
            const int2 en = a.rag[re0 + q];
            if (tid >= en.y) {
                g = q;
                sidx = en.x;
                rbase = en.y;
            }
        }
        if (g >= 0) p = tid - rbase;
    } else if (C == 1) {
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
    bool valid = (p >= 0) && (sidx < a.nsys);
    if (ragged && valid && p > a.sub_P[a.sys[sidx].sub]) valid = false;   // the next system's
    const int rcbase = rbase - (g > 0 ? g : 0);   // ragged chunk slots: sum of P_j before

    auto SEP = [&](double2* arr, int ps) -> double2* {
        if (ragged) return arr + rbase + ps;
        if (C == 1) return arr + g * (P + 1) + ps;
        const int home = ps / T;
        double2* base = (home == rank) ? arr : cl.map_shared_rank(arr, home);
        return base + (ps - home * T);
    };
    auto CHK = [&](double2* arr, int pc) -> double2* {
        if (ragged) return arr + rcbase + pc;
        if (C == 1) return arr + g * P + pc;
        const int home = pc / T;
        double2* base = (home == rank) ? arr : cl.map_shared_rank(arr, home);
        return base + (pc - home * T);
    };
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
    const bool realsep = valid && (p <= Pj);          // separators beyond Pj are padding
    // every step's state recorded (impulse responses for the superposed u(T))
    const bool rec_u = valid && a.urec && (sy.flags & SYS_REC_U);
    const int nj = valid ? a.sub_n[j] : 0;
    // Systems of a launch may have different step counts (a batch of problem
    // instances): the CTA runs to the longest of its systems (a cluster holds one
    // system), and a system past its own count neither reads fluxes, nor writes
    // outputs, nor advances its state.
    int ntc = 0;
    if (ragged) {
        for (int q = 0; q < rne; ++q) ntc = max(ntc, a.sys[a.rag[re0 + q].x].nt);
    } else if (C == 1) {
        for (int gg = 0; gg < G; ++gg) {
            const int si = blockIdx.x * G + gg;
            if (si < a.nsys) ntc = max(ntc, a.sys[si].nt);
        }
    } else {
        ntc = a.sys[blockIdx.x / C].nt;
    }
    ntc = min(ntc, nt);
    // factor pointers; with per-step factorisations they advance by one step's
    // stride per time step (the strides are zero for a constant matrix)
    const double2* F = a.fac + (size_t)j * L * 4 * P + (p < P ? p : 0);
    const double2* sE_l = a.sep + (size_t)(j * 3 + 0) * (P + 1);
    const double2* sE_r = a.sep + (size_t)(j * 3 + 1) * (P + 1);
    const double2* sbinv = a.sep + (size_t)(j * 3 + 2) * (P + 1);
    const double2* pcr = a.pcr + (size_t)j * levels * 2 * (P + 1);
    const bool stepped = a.fstride != 0;
    // Streamed per-step factors are staged one step ahead in shared memory by
    // asynchronous copies, each thread copying exactly the entries it reads
    // (element-major slots, slot k of thread tid at stg[k * T + tid]):
    //   stage 1: separator data (E_l, E_r, 1/delta, PCR coefficients);
    //   stage 2: also the chunk factors (q, c) and the spikes (a, b).
    // Every phase refills its buffer for step t+1 right after its last read at
    // step t, and waits (cp.async.wait_group 2) before its first read: the
    // groups are committed in the fixed order (q,c) | separator | (a,b).
    const int stage = a.stage;
    const int npc = 2 * levels + 3;
    double2* stg = hsum + 4 * G;
    auto issue_fa = [&](const double2* Fs) {   // Fs == nullptr: commit an empty group
        if (stage >= 2 && Fs && valid && Lp > 0) {
#pragma unroll
            for (int i = 0; i < L; ++i)
                if (i < Lp) {
                    cp_async16(stg + (npc + i * 2 + 0) * T + tid, Fs + (i * 4 + 0) * P);
                    cp_async16(stg + (npc + i * 2 + 1) * T + tid, Fs + (i * 4 + 1) * P);
                }
        }
        cp_async_commit();
    };
    auto issue_fd = [&](const double2* Fs) {
        if (stage >= 2 && Fs && valid && Lp > 0) {
#pragma unroll
            for (int i = 0; i < L; ++i)
                if (i < Lp) {
                    cp_async16(stg + (npc + 2 * L + i * 2 + 0) * T + tid, Fs + (i * 4 + 2) * P);
                    cp_async16(stg + (npc + 2 * L + i * 2 + 1) * T + tid, Fs + (i * 4 + 3) * P);
                }
        }
        cp_async_commit();
    };
    auto issue_pc = [&](bool on, long long sofs, long long pofs) {
        if (stage >= 1 && on && valid) {
            cp_async16(stg + 0 * T + tid, sE_l + sofs + p);
            cp_async16(stg + 1 * T + tid, sE_r + sofs + p);
            cp_async16(stg + 2 * T + tid, sbinv + sofs + p);
            for (int k = 0; k < 2 * levels; ++k)
                cp_async16(stg + (3 + k) * T + tid, pcr + pofs + (size_t)k * (P + 1) + p);
        }
        cp_async_commit();
    };
    // chunk factor (i, k) and separator datum k of the current step
    auto FAC = [&](int i, int k) -> double2 {
        if (stage >= 2)
            return stg[(npc + (k < 2 ? i * 2 + k : 2 * L + i * 2 + k - 2)) * T + tid];
        return F[(i * 4 + k) * P];
    };

    double2 u[L], y[L];
#pragma unroll
    for (int i = 0; i < L; ++i) {
        u[i] = (valid && i < Lp && !zero_u0) ? a.u0[goff + sp + 1 + i] : zero;
        y[i] = zero;
    }
    if (valid) *SEP(usep, p) = (realsep && !zero_u0) ? a.u0[goff + sp] : zero;
    // S_0^2: the end traces start with v_0 = u_0 at the end
    const bool hl = s02v && realsep && p == 0 && (tcf & 1);
    const bool hr = s02v && realsep && p == Pj && (tcf & 2);
    // end traces v_0..v_{nt} at absolute steps: a launch marching a segment of the time
    // axis (steps ht0 + 1 ..) extends the traces the earlier segments left
    const int hst = a.hstride > 0 ? a.hstride : nt + 1, ht0 = a.ht0;
    double2* hist_l = s02v ? a.hist + ((size_t)sidx * 2 + 0) * hst : nullptr;
    double2* hist_r = s02v ? a.hist + ((size_t)sidx * 2 + 1) * hst : nullptr;
    // per-end kernels: h_0 = rho v_0; the flux weight on v_n is kout[0]
    constexpr bool gen = GEN;
    if (hl && ht0 == 0) hist_l[0] = zero_u0 ? zero : (gen ? cmul(a.rho[2 * j + 0], a.u0[goff + sp]) : a.u0[goff + sp]);
    if (hr && ht0 == 0) hist_r[0] = zero_u0 ? zero : (gen ? cmul(a.rho[2 * j + 1], a.u0[goff + sp]) : a.u0[goff + sp]);
    const int hs_l = (C == 1) ? 2 * g : 0, hs_r = hs_l + 1;
    if (stage > 0) {   // step 1's factors
        issue_fa(F);
        issue_pc(true, 0, 0);
        issue_fd(F);
    }
    SYNC();

    // gradient mode: per-thread sums of the potential form (interior nodes of the
    // chunk, and the one-sided parts of its two separators)
    double ga_int[MODE == 2 ? L : 1], ga_l = 0.0, ga_r = 0.0;
#pragma unroll
    for (int i = 0; i < (MODE == 2 ? L : 1); ++i) ga_int[i] = 0.0;

    double2 lin = zero, rin = zero;
    for (int t = 1; t <= ntc; ++t) {
        const bool live = t <= sy.nt;
        if (stage == 0 && stepped && valid && t < nt) {
            // the next step's factors stream from HBM: request them into L2 now
            if (Lp > 0) {
#pragma unroll
                for (int i = 0; i < L; ++i)
                    if (i < Lp)
#pragma unroll
                        for (int k = 0; k < 4; ++k) prefetch_l2(F + a.fstride + (i * 4 + k) * P);
            }
            prefetch_l2(sE_l + a.sstride + p);
            prefetch_l2(sE_r + a.sstride + p);
            prefetch_l2(sbinv + a.sstride + p);
            for (int k = 0; k < 2 * levels; ++k) prefetch_l2(pcr + a.pstride + (size_t)k * (P + 1) + p);
        }
        // ---- phase A: chunk right-hand sides and local LU solves -------------
        if (stage >= 2) cp_async_wait<2>();
        if (valid && Lp > 0) {
            const double2 uL = *SEP(usep, p), uR = *SEP(usep, p + 1);
            double2 zprev = zero, cprev = zero, uf = zero, ul = zero;
#pragma unroll
            for (int i = 0; i < L; ++i) {
                if (i < Lp) {
                    const double2 left = (i == 0) ? uL : u[i - 1];
                    double2 right;
                    if (i + 1 < L)
                        right = (i == Lp - 1) ? uR : u[i + 1];
                    else
                        right = uR;
                    double2 f = make_double2(fma(4.0, u[i].x, left.x + right.x),
                                             fma(4.0, u[i].y, left.y + right.y));
                    const double2 z = (i == 0) ? f : cfms(cprev, zprev, f);
                    y[i] = z;
                    zprev = z;
                    cprev = FAC(i, 1);
                    if (i == 0) uf = u[i];
                    ul = csel(i == Lp - 1, u[i], ul);
                }
            }
            double2 ynext = zero, yl = zero;
#pragma unroll
            for (int i = L - 1; i >= 0; --i) {
                if (i < Lp) {
                    const double2 qi = FAC(i, 0);
                    double2 yi = cmul(qi, y[i]);
                    if (i != Lp - 1) yi = cfms(FAC(i, 1), ynext, yi);
                    else yl = yi;
                    y[i] = yi;
                    ynext = yi;
                }
            }
            *CHK(ufst, p) = uf;
            *CHK(ulst, p) = ul;
            *CHK(yfst, p) = y[0];
            *CHK(ylst, p) = yl;
        }
        if (stage > 0) issue_fa(t < nt ? F + a.fstride : nullptr);
        if (s02v) {
            // history sums of the ends this CTA holds, one warp per end
            const int lane = tid & 31, w = tid >> 5, nw = T >> 5;
            if (C == 1) {
                for (int e = w; e < 2 * (ragged ? rne : G); e += nw) {
                    const int gs = ragged ? a.rag[re0 + (e >> 1)].x : blockIdx.x * G + (e >> 1);
                    const int side = e & 1;
                    if (gs < a.nsys && (a.sub_tc[a.sys[gs].sub] & (1 << side))) {
                        const double2* hh = a.hist + ((size_t)gs * 2 + side) * hst;
                        if (gen) {
                            const size_t ke = (size_t)(2 * a.sys[gs].sub + side) * a.kstride;
                            double2 o1, o2;
                            conv_history2(a.kap + ke, a.kout + ke, hh, ht0 + t, lane, o1, o2);
                            if (lane == 0) {
                                hsum[e] = o1;
                                hsum2[e] = o2;
                            }
                        } else {
                            const double2 hsv = s02_history(a.beta, hh, ht0 + t, lane);
                            if (lane == 0) hsum[e] = hsv;
                        }
                    }
                }
            } else {
                const int Pe = a.sub_P[a.sys[sidx].sub];
                const int tce = a.sub_tc[a.sys[sidx].sub];
                const int se = a.sys[sidx].sub;
                if (w == 0 && rank == 0 && (tce & 1)) {
                    if (gen) {
                        const size_t ke = (size_t)(2 * se + 0) * a.kstride;
                        double2 o1, o2;
                        conv_history2(a.kap + ke, a.kout + ke, hist_l, ht0 + t, lane, o1, o2);
                        if (lane == 0) {
                            hsum[0] = o1;
                            hsum2[0] = o2;
                        }
                    } else {
                        const double2 hsv = s02_history(a.beta, hist_l, ht0 + t, lane);
                        if (lane == 0) hsum[0] = hsv;
                    }
                }
                if (w == (nw > 1 ? 1 : 0) && rank == Pe / T && (tce & 2)) {
                    if (gen) {
                        const size_t ke = (size_t)(2 * se + 1) * a.kstride;
                        double2 o1, o2;
                        conv_history2(a.kap + ke, a.kout + ke, hist_r, ht0 + t, lane, o1, o2);
                        if (lane == 0) {
                            hsum[1] = o1;
                            hsum2[1] = o2;
                        }
                    } else {
                        const double2 hsv = s02_history(a.beta, hist_r, ht0 + t, lane);
                        if (lane == 0) hsum[1] = hsv;
                    }
                }
            }
        }
        SYNC();
        // ---- phase B: reduced right-hand side at my separator ------------------
        if (stage >= 1) cp_async_wait<2>();
        if (valid) {
            double2 d = zero;
            if (realsep) {
                const double2 us = *SEP(usep, p);
                const bool le = (p == 0), re = (p == Pj);
                const double2 um = le ? zero : *CHK(ulst, p - 1);
                const double2 up = re ? zero : *CHK(ufst, p);
                double2 f;
                if (le)
                    f = make_double2(fma(2.0, us.x, up.x), fma(2.0, us.y, up.y));
                else if (re)
                    f = make_double2(fma(2.0, us.x, um.x), fma(2.0, us.y, um.y));
                else
                    f = make_double2(fma(4.0, us.x, um.x + up.x), fma(4.0, us.y, um.y + up.y));
                if (le && (tcf & 1)) {
                    if (sy.flags & SYS_IMP_L)
                        lin = (t == 1) ? make_double2(1.0, 0.0) : zero;
                    else
                        lin = (live && sy.in_l >= 0 && a.gin) ? a.gin[(size_t)sy.in_l + a.t0 + t - 1] : zero;
                    f = cfms(lin, a.inv_ik, f);
                    if (s02v) f = cfma(hsum[hs_l], gen ? a.inv_ik : a.c2_ik, f);
                }
                if (re && (tcf & 2)) {
                    if (sy.flags & SYS_IMP_R)
                        rin = (t == 1) ? make_double2(1.0, 0.0) : zero;
                    else
                        rin = (live && sy.in_r >= 0 && a.gin) ? a.gin[(size_t)sy.in_r + a.t0 + t - 1] : zero;
                    f = cfms(rin, a.inv_ik, f);
                    if (s02v) f = cfma(hsum[hs_r], gen ? a.inv_ik : a.c2_ik, f);
                }
                d = f;
                const double2 El = (stage >= 1) ? stg[0 * T + tid] : sE_l[p];
                const double2 Er = (stage >= 1) ? stg[1 * T + tid] : sE_r[p];
                if (!le) d = cfms(El, *CHK(ylst, p - 1), d);
                if (!re) d = cfms(Er, *CHK(yfst, p), d);
            }
            *SEP(dA, p) = d;
        }
        SYNC();
        // ---- phase C: PCR on the separators (coefficients precomputed) -------
        double2* src = dA;
        double2* dst = dB;
        for (int k = 0; k < levels; ++k) {
            const int st = 1 << k;
            if (valid) {
                const double2 alp = (stage >= 1) ? stg[(3 + 2 * k) * T + tid]
                                                 : pcr[(size_t)(k * 2 + 0) * (P + 1) + p];
                const double2 gap = (stage >= 1) ? stg[(4 + 2 * k) * T + tid]
                                                 : pcr[(size_t)(k * 2 + 1) * (P + 1) + p];
                double2 dd = *SEP(src, p);
                if (p - st >= 0) dd = cfma(alp, *SEP(src, p - st), dd);
                if (p + st <= (ragged ? Pj : P)) dd = cfma(gap, *SEP(src, p + st), dd);
                if (k == levels - 1) dd = cmul(dd, (stage >= 1) ? stg[2 * T + tid] : sbinv[p]);
                *SEP(dst, p) = dd;
            }
            SYNC();
            double2* tmp = src;
            src = dst;
            dst = tmp;
        }
        if (stage > 0) issue_pc(t < nt, a.sstride, a.pstride);
        // ---- phase D: spike correction, CN update, fluxes ---------------------
        if (stage >= 2) cp_async_wait<2>();
        double2 vv[MODE == 2 ? L : 1];
        if (valid && Lp > 0) {
            const double2 vL = *SEP(src, p), vR = *SEP(src, p + 1);
#pragma unroll
            for (int i = 0; i < L; ++i) {
                if (i < Lp) {
                    double2 v = cfms(FAC(i, 2), vL, y[i]);
                    v = cfms(FAC(i, 3), vR, v);
                    if constexpr (MODE == 1)
                        if (live) a.vrec[(size_t)(t - 1) * a.nxrec + goff + sp + 1 + i] = v;
                    if constexpr (MODE == 2) vv[i] = v;
                    if (live) u[i] = make_double2(fma(2.0, v.x, -u[i].x), fma(2.0, v.y, -u[i].y));
                }
            }
        }
        if constexpr (MODE == 2) {
            // elements e = 0..Lp from separator p (node sp) to separator p+1 (node
            // sp + Lp + 1); x = this march's v, y = the recorded forward v of the
            // mirrored step
            if (valid && live && p < Pj) {
                const double2* yrow = a.vfwd + (size_t)(nt - t) * a.nxrec + goff + sp;
                const double2 xL = *SEP(src, p), xR = *SEP(src, p + 1);
                const double h12 = a.h12;
#pragma unroll
                for (int e = 0; e <= L; ++e) {
                    if (e <= Lp) {
                        const double2 xa = (e == 0) ? xL : vv[e > 0 ? e - 1 : 0];
                        const double2 xb = (e < L) ? csel(e < Lp, vv[e < L ? e : 0], xR) : xR;
                        const double2 ya = yrow[e], yb = yrow[e + 1];
                        const double sa = xa.x * ya.x - xa.y * ya.y;
                        const double sb = xb.x * yb.x - xb.y * yb.y;
                        const double c = (xa.x * yb.x - xa.y * yb.y) + (xb.x * ya.x - xb.y * ya.y);
                        const double toa = h12 * (3.0 * sa + c + sb);
                        const double tob = h12 * (sa + c + 3.0 * sb);
                        if (e == 0) ga_l += toa;
                        else ga_int[e > 0 ? e - 1 : 0] += toa;
                        if (e < Lp) ga_int[e < L ? e : 0] += tob;
                        else ga_r += tob;
                    }
                }
            }
        }
        if (stage > 0) issue_fd(t < nt ? F + a.fstride : nullptr);
        if (realsep && live) {
            const double2 v = *SEP(src, p);
            if constexpr (MODE == 1) {   // an interface node is recorded by its left subdomain
                if (!(p == 0 && (tcf & 1))) a.vrec[(size_t)(t - 1) * a.nxrec + goff + sp] = v;
            }
            double2* us = SEP(usep, p);
            const double2 uo = *us;
            *us = make_double2(fma(2.0, v.x, -uo.x), fma(2.0, v.y, -uo.y));
            if (p == 0) {
                if (hl) hist_l[ht0 + t] = v;
                if ((tcf & 1) && sy.out_a >= 0 && a.gout) {
                    const double2 ts = gen ? a.kout[(size_t)(2 * j + 0) * a.kstride] : a.two_sigma;
                    double2 o = csub(cmul(ts, v), lin);
                    if (gen) o = cadd(o, hsum2[hs_l]);
                    else if (s02v) o = cfma(a.two_c2, hsum[hs_l], o);
                    a.gout[(size_t)sy.out_a + a.t0 + t - 1] = o;
                }
                if ((sy.flags & SYS_TRACE) && a.trace) a.trace[((size_t)sidx * 2 + 0) * nt + t - 1] = v;
            }
            if (p == Pj) {
                if (hr) hist_r[ht0 + t] = v;
                if ((tcf & 2) && sy.out_b >= 0 && a.gout) {
                    const double2 ts = gen ? a.kout[(size_t)(2 * j + 1) * a.kstride] : a.two_sigma;
                    double2 o = csub(cmul(ts, v), rin);
                    if (gen) o = cadd(o, hsum2[hs_r]);
                    else if (s02v) o = cfma(a.two_c2, hsum[hs_r], o);
                    a.gout[(size_t)sy.out_b + a.t0 + t - 1] = o;
                }
                if ((sy.flags & SYS_TRACE) && a.trace) a.trace[((size_t)sidx * 2 + 1) * nt + t - 1] = v;
            }
        }
        if (rec_u && live) {   // u_t of this system in local node order
            // streaming stores: the recorded states are read once, by the superposition,
            // and must not evict the factors the march rereads every step from L2
            double2* row = a.urec + sy.rec + (size_t)(t - 1) * nj;
#pragma unroll
            for (int i = 0; i < L; ++i)
                if (i < Lp) __stcs(row + sp + 1 + i, u[i]);
            if (realsep) __stcs(row + sp, *SEP(usep, p));
        }
        F += a.fstride;
        sE_l += a.sstride;
        sE_r += a.sstride;
        sbinv += a.sstride;
        pcr += a.pstride;
        SYNC();
    }
    if (stage > 0) cp_async_wait_all();   // no copy in flight past the loop
    if constexpr (MODE == 2) {
        // add this segment's sums; every entry has exactly one writer per launch
        if (valid && p < Pj) {
#pragma unroll
            for (int i = 0; i < L; ++i)
                if (i < Lp) a.gint[goff + sp + 1 + i] += ga_int[i];
            a.gl[goff + sp] += ga_l;
            a.gr[goff + sp + Lp + 1] += ga_r;
        }
    }
    // ---- final state ----------------------------------------------------------
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
            // the interface node belongs to the left subdomain
            if ((sy.flags & SYS_WRITE_UT) && a.uT && (sp > 0 || !(tcf & 1))) a.uT[goff + sp] = us;
            if ((sy.flags & SYS_REC_LAST) && a.urec) a.urec[sy.rec + sp] = us;
        }
        if ((sy.flags & SYS_REC_LAST) && a.urec) {
#pragma unroll
            for (int i = 0; i < L; ++i)
                if (i < Lp) a.urec[sy.rec + sp + 1 + i] = u[i];
        }
    }
    if (bad) atomicOr(a.status, ST_NONFINITE);
    // keep remote shared memory alive until every CTA of the cluster is done
    if (C > 1) cl.sync();
}

// ---------------------------------------------------------------------------
// The constant-matrix march of one system spread over a cluster of C CTAs (or alone
// in its CTA, C = 1) with the two-level separator solve (FactorSet.tl_*): one cluster
// barrier per time step instead of one per PCR level.  Thread p = rank T + tid owns separator p and chunk p
// as in k_march_static; T is a multiple of 32, so warp q of the system (separators
// 32q .. 32q+31) lies in one CTA, and the first separator of every CTA is a
// super-separator.  Per step:
//   A  chunk right-hand sides and local solves (the right separator's u comes from
//      the same warp or, for a super-separator, from this CTA's replica usup);
//   B  separator right-hand sides; a super-separator forms the part of its row it
//      owns, and lane 31 the part that its chunk contributes to the next warp's
//      super-separator;
//   C  super-chunk PCR in registers (warp shuffles), then each warp publishes its
//      super-separator data and the first/last super-chunk values (double-buffered
//      by step parity); one cluster barrier;
//   D  warp 0 of every CTA gathers the reduced right-hand sides (distributed shared
//      memory) and solves the reduced system by PCR, so every CTA holds all
//      super-separator values (xsup) and their u (usup); one CTA barrier;
//   E  super-chunk values x = yhat - a x_{s_q} - b x_{s_{q+1}};
//   F  spike correction of the chunks, CN update, fluxes (as k_march_static).
// Constant factors.  MODE 0; 1 also records v of every step (a.vrec), 2 accumulates the
// adjoint potential form against the recorded forward values (a.vfwd), both as
// k_march_static does (L <= 8, no S_0^2 history).
// ---------------------------------------------------------------------------
int swr_march_tl_smem_bytes(int T) {
    const int W = T / 32;
    return (int)sizeof(double2) * (6 * T + 2 * W * 5 + 2 * 33 + 8);
}

template <int L, bool GEN, int MODE = 0>
__global__ void __launch_bounds__((L == 16 || MODE == 2) ? 256 : 384, 1) k_march_tl(const MarchArgs a) {
    extern __shared__ double2 sm[];
    const int T = a.T, P = a.P, C = a.C, nt = a.nt;
    const int W = T / 32;
    double2* usep = sm;              // [T] u at my separators
    double2* xv = usep + T;          // [T] separator values of this step
    double2* ufst = xv + T;
    double2* ulst = ufst + T;
    double2* yfst = ulst + T;
    double2* ylst = yfst + T;
    double2* pub = ylst + T;         // [2][W][5] per warp: P0, P1, yhat_first, yhat_last, P4
    double2* xsup = pub + 2 * W * 5; // [33] super-separator values (every CTA)
    double2* usup = xsup + 33;       // [33] u at the super-separators (every CTA)
    double2* hsum = usup + 33;       // [2] S_0^2 / own-operator history of the two ends
    double2* hsum2 = hsum + 2;       // [2] flux-update history (per-end kernels)
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
    const bool sup = realsep && (lane == 0 || p == Pj);          // a super-separator
    const int qsup = (p == Pj) ? Q : q;                           // its index
    const int m = (32 * q < Pj) ? min(31, Pj - 1 - 32 * q) : 0;   // members of super-chunk q
    const bool member = realsep && lane >= 1 && lane <= m;
    // super-separator index of separator p + 1 (or -1 if it is a super-chunk member)
    const int rsup = (p + 1 == Pj) ? Q : (((p + 1) & 31) == 0 ? (p + 1) >> 5 : -1);
    const bool rec_u = valid && a.urec && (sy.flags & SYS_REC_U);
    const int nj = (sidx < a.nsys) ? a.sub_n[j] : 0;
    const int ntc = min(sy.nt, nt);
    const size_t S = P + 1;
    const double2* F = a.fac + (size_t)j * L * 4 * P + (p < P ? p : 0);
    const double2* sE_l = a.sep + (size_t)(j * 3 + 0) * S;
    const double2* sE_r = a.sep + (size_t)(j * 3 + 1) * S;
    const double2* tpc = a.tl_pcr + (size_t)j * 10 * S + (valid ? p : 0);
    const double2* tax = a.tl_aux + (size_t)j * 3 * S + (valid ? p : 0);
    const double2* tred = a.tl_red + (size_t)j * 13 * 32 + lane;
    // the separator solve's coefficients are re-read every step (L1-resident), which
    // keeps the chunk state in registers

    double2 u[L], y[L];
#pragma unroll
    for (int i = 0; i < L; ++i) {
        u[i] = (valid && i < Lp && !zero_u0) ? a.u0[goff + sp + 1 + i] : zero;
        y[i] = zero;
    }
    // MODE 2: per-thread sums of the potential form (interior nodes of the chunk, and the
    // one-sided parts of its two separators)
    double ga_int[MODE == 2 ? L : 1], ga_l = 0.0, ga_r = 0.0;
#pragma unroll
    for (int i = 0; i < (MODE == 2 ? L : 1); ++i) ga_int[i] = 0.0;
    usep[tid] = (realsep && !zero_u0) ? a.u0[goff + sp] : zero;
    // replicas of the super-separators' u in every CTA (warp 0)
    if (wl == 0 && lane <= Q && sidx < a.nsys) {
        const int ps = (lane < Q) ? 32 * lane : Pj;
        usup[lane] = zero_u0 ? zero : a.u0[goff + a.sep_pos[j * S + ps]];
    }
    const bool hl = a.s02 && realsep && p == 0 && (tcf & 1);
    const bool hr = a.s02 && realsep && p == Pj && (tcf & 2);
    // end traces v_0..v_{nt} at absolute steps: a launch marching a segment of the time
    // axis (steps ht0 + 1 ..) extends the traces the earlier segments left
    const int hst = a.hstride > 0 ? a.hstride : nt + 1, ht0 = a.ht0;
    double2* hist_l = a.s02 ? a.hist + ((size_t)sidx * 2 + 0) * hst : nullptr;
    double2* hist_r = a.s02 ? a.hist + ((size_t)sidx * 2 + 1) * hst : nullptr;
    constexpr bool gen = GEN;
    if (hl && ht0 == 0) hist_l[0] = zero_u0 ? zero : (gen ? cmul(a.rho[2 * j + 0], a.u0[goff + sp]) : a.u0[goff + sp]);
    if (hr && ht0 == 0) hist_r[0] = zero_u0 ? zero : (gen ? cmul(a.rho[2 * j + 1], a.u0[goff + sp]) : a.u0[goff + sp]);
    // the warps that hold the two ends form their history sums
    const bool wleft = a.s02 && (tcf & 1) && rank == 0 && wl == 0;
    const bool wright = a.s02 && (tcf & 2) && rank == Pj / T && wl == (Pj % T) / 32;
    cl.sync();

    double2 lin = zero, rin = zero;
    for (int t = 1; t <= ntc; ++t) {
        const int slot = (t & 1) * W * 5;
        // ---- A: chunk right-hand sides and local LU solves ---------------------
        if (valid && Lp > 0) {
            const double2 uL = usep[tid];
            const double2 uR = (rsup >= 0) ? usup[rsup] : usep[tid + 1];
            double2 zprev = zero, cprev = zero, uf = zero, ul = zero;
#pragma unroll
            for (int i = 0; i < L; ++i) {
                if (i < Lp) {
                    const double2 left = (i == 0) ? uL : u[i - 1];
                    double2 right;
                    if (i + 1 < L)
                        right = (i == Lp - 1) ? uR : u[i + 1];
                    else
                        right = uR;
                    double2 f = make_double2(fma(4.0, u[i].x, left.x + right.x),
                                             fma(4.0, u[i].y, left.y + right.y));
                    const double2 z = (i == 0) ? f : cfms(cprev, zprev, f);
                    y[i] = z;
                    zprev = z;
                    cprev = F[(i * 4 + 1) * P];
                    if (i == 0) uf = u[i];
                    ul = csel(i == Lp - 1, u[i], ul);
                }
            }
            double2 ynext = zero, yl = zero;
#pragma unroll
            for (int i = L - 1; i >= 0; --i) {
                if (i < Lp) {
                    const double2 qi = F[(i * 4 + 0) * P];
                    double2 yi = cmul(qi, y[i]);
                    if (i != Lp - 1) yi = cfms(F[(i * 4 + 1) * P], ynext, yi);
                    else yl = yi;
                    y[i] = yi;
                    ynext = yi;
                }
            }
            ufst[tid] = uf;
            ulst[tid] = ul;
            yfst[tid] = y[0];
            ylst[tid] = yl;
        }
        // history sums of the ends (the warps holding them; a system of at most 32
        // separators has both ends in warp 0 of its CTA, which then forms both sums)
        for (int side = 0; side < 2; ++side) {
            if (!(side == 0 ? wleft : wright)) continue;   // uniform over the warp
            const double2* hh = side == 0 ? hist_l : hist_r;
            if (gen) {
                const size_t ke = (size_t)(2 * j + side) * a.kstride;
                double2 o1, o2;
                conv_history2(a.kap + ke, a.kout + ke, hh, ht0 + t, lane, o1, o2);
                if (lane == 0) {
                    hsum[side] = o1;
                    hsum2[side] = o2;
                }
            } else {
                const double2 hsv = s02_history(a.beta, hh, ht0 + t, lane);
                if (lane == 0) hsum[side] = hsv;
            }
        }
        __syncwarp();
        // ---- B: separator right-hand sides --------------------------------------
        double2 d = zero;
        if (realsep) {
            const double2 us = usep[tid];
            const bool le = (p == 0), re = (p == Pj);
            // the chunk on the left is in this warp unless p is a warp's lane 0
            const bool own_left = !le && lane != 0;
            const double2 um = own_left ? ulst[tid - 1] : zero;
            const double2 up = re ? zero : ufst[tid];
            double2 f;
            if (le)
                f = make_double2(fma(2.0, us.x, up.x), fma(2.0, us.y, up.y));
            else if (re)
                f = make_double2(fma(2.0, us.x, um.x), fma(2.0, us.y, um.y));
            else
                f = make_double2(fma(4.0, us.x, um.x + up.x), fma(4.0, us.y, um.y + up.y));
            if (le && (tcf & 1)) {
                if (sy.flags & SYS_IMP_L)
                    lin = (t == 1) ? make_double2(1.0, 0.0) : zero;
                else
                    lin = (sy.in_l >= 0 && a.gin) ? a.gin[(size_t)sy.in_l + a.t0 + t - 1] : zero;
                f = cfms(lin, a.inv_ik, f);
                if (a.s02) f = cfma(hsum[0], gen ? a.inv_ik : a.c2_ik, f);
            }
            if (re && (tcf & 2)) {
                if (sy.flags & SYS_IMP_R)
                    rin = (t == 1) ? make_double2(1.0, 0.0) : zero;
                else
                    rin = (sy.in_r >= 0 && a.gin) ? a.gin[(size_t)sy.in_r + a.t0 + t - 1] : zero;
                f = cfms(rin, a.inv_ik, f);
                if (a.s02) f = cfma(hsum[1], gen ? a.inv_ik : a.c2_ik, f);
            }
            d = f;
            if (own_left) d = cfms(sE_l[p], ylst[tid - 1], d);
            if (!re) d = cfms(sE_r[p], yfst[tid], d);
        }
        // lane 31: this chunk's part of the next super-separator's row
        double2 p1 = zero;
        if (valid && lane == 31 && p + 1 <= Pj)
            p1 = cfms(sE_l[p + 1], ylst[tid], ulst[tid]);
        // ---- C: super-chunk PCR in registers ----------------------------------
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int st = 1 << k;
            const double2 dm = shfl_up2(d, st), dp = shfl_down2(d, st);
            if (member) d = cfma(tpc[(2 * k + 1) * S], dp, cfma(tpc[(2 * k) * S], dm, d));
        }
        if (member) d = cmul(d, tax[0]);
        {
            double2* pb = pub + slot + wl * 5;
            if (lane == 0 && realsep) pb[0] = d;                 // row s_q, own part
            if (lane == 31) pb[1] = p1;
            if (lane == 1 && member) pb[2] = d;                  // yhat of the first member
            if (member && lane == m) pb[3] = d;                  // yhat of the last member
            if (p == Pj && lane != 0 && valid) pb[4] = d;        // row Pj, complete
        }
        cl.sync();
        // ---- D: reduced system (warp 0 of every CTA) -----------------------------
        if (wl == 0 && sidx < a.nsys) {
            double2 r = zero;
            if (lane <= Q) {
                auto pubof = [&](int qq) -> const double2* {   // warp qq's published data
                    const int home = (32 * qq) / T;
                    double2* base = (home == rank) ? pub : cl.map_shared_rank(pub, home);
                    return base + slot + ((32 * qq) % T) / 32 * 5;
                };
                if (lane == Q && (Pj & 31) != 0) {
                    r = pubof(Q - 1)[4];
                } else {
                    r = pubof(lane)[0];
                    if (lane >= 1) r = cadd(r, pubof(lane - 1)[1]);
                }
                const double2 cL = tred[11 * 32], cU = tred[12 * 32];
                if (lane >= 1 && (cL.x != 0.0 || cL.y != 0.0))
                    r = cfms(cL, pubof(lane - 1)[3], r);
                if (lane < Q && (cU.x != 0.0 || cU.y != 0.0))
                    r = cfms(cU, pubof(lane)[2], r);
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const int st = 1 << k;
                const double2 rm = shfl_up2(r, st), rp = shfl_down2(r, st);
                if (lane <= Q) r = cfma(tred[(2 * k + 1) * 32], rp, cfma(tred[(2 * k) * 32], rm, r));
            }
            if (lane <= Q) {
                r = cmul(r, tred[10 * 32]);
                xsup[lane] = r;
                const double2 uo = usup[lane];
                usup[lane] = make_double2(fma(2.0, r.x, -uo.x), fma(2.0, r.y, -uo.y));
            }
        }
        __syncthreads();
        // ---- E: super-chunk values -----------------------------------------------
        double2 v = zero;
        if (member) {
            v = cfms(tax[S], xsup[q], d);
            v = cfms(tax[2 * S], xsup[q + 1], v);
        } else if (sup) {
            v = xsup[qsup];
        }
        xv[tid] = v;
        __syncwarp();
        // ---- F: spike correction, CN update, fluxes -------------------------------
        double2 vv[MODE == 2 ? L : 1];
        if (valid && Lp > 0) {
            const double2 vR = (rsup >= 0) ? xsup[rsup] : xv[tid + 1];
#pragma unroll
            for (int i = 0; i < L; ++i) {
                if (i < Lp) {
                    double2 vi = cfms(F[(i * 4 + 2) * P], v, y[i]);
                    vi = cfms(F[(i * 4 + 3) * P], vR, vi);
                    if constexpr (MODE == 1) a.vrec[(size_t)(t - 1) * a.nxrec + goff + sp + 1 + i] = vi;
                    if constexpr (MODE == 2) vv[i] = vi;
                    u[i] = make_double2(fma(2.0, vi.x, -u[i].x), fma(2.0, vi.y, -u[i].y));
                }
            }
            if constexpr (MODE == 2) {
                // elements e = 0..Lp from separator p (node sp) to separator p + 1 (node
                // sp + Lp + 1); x = this march's v, y = the recorded forward v of the
                // mirrored step
                if (p < Pj) {
                    const double2* yrow = a.vfwd + (size_t)(nt - t) * a.nxrec + goff + sp;
                    const double h12 = a.h12;
#pragma unroll
                    for (int e = 0; e <= L; ++e) {
                        if (e <= Lp) {
                            const double2 xa = (e == 0) ? v : vv[e > 0 ? e - 1 : 0];
                            const double2 xb = (e < L) ? csel(e < Lp, vv[e < L ? e : 0], vR) : vR;
                            const double2 ya = yrow[e], yb = yrow[e + 1];
                            const double sa = xa.x * ya.x - xa.y * ya.y;
                            const double sb = xb.x * yb.x - xb.y * yb.y;
                            const double c = (xa.x * yb.x - xa.y * yb.y) + (xb.x * ya.x - xb.y * ya.y);
                            const double toa = h12 * (3.0 * sa + c + sb);
                            const double tob = h12 * (sa + c + 3.0 * sb);
                            if (e == 0) ga_l += toa;
                            else ga_int[e > 0 ? e - 1 : 0] += toa;
                            if (e < Lp) ga_int[e < L ? e : 0] += tob;
                            else ga_r += tob;
                        }
                    }
                }
            }
        }
        if constexpr (MODE == 1) {   // an interface node is recorded by its left subdomain
            if (realsep && !(p == 0 && (tcf & 1)))
                a.vrec[(size_t)(t - 1) * a.nxrec + goff + sp] = v;
        }
        if (realsep) {
            const double2 uo = usep[tid];
            usep[tid] = make_double2(fma(2.0, v.x, -uo.x), fma(2.0, v.y, -uo.y));
            if (p == 0) {
                if (hl) hist_l[ht0 + t] = v;
                if ((tcf & 1) && sy.out_a >= 0 && a.gout) {
                    const double2 ts = gen ? a.kout[(size_t)(2 * j + 0) * a.kstride] : a.two_sigma;
                    double2 o = csub(cmul(ts, v), lin);
                    if (gen) o = cadd(o, hsum2[0]);
                    else if (a.s02) o = cfma(a.two_c2, hsum[0], o);
                    a.gout[(size_t)sy.out_a + a.t0 + t - 1] = o;
                }
                if ((sy.flags & SYS_TRACE) && a.trace) a.trace[((size_t)sidx * 2 + 0) * nt + t - 1] = v;
            }
            if (p == Pj) {
                if (hr) hist_r[ht0 + t] = v;
                if ((tcf & 2) && sy.out_b >= 0 && a.gout) {
                    const double2 ts = gen ? a.kout[(size_t)(2 * j + 1) * a.kstride] : a.two_sigma;
                    double2 o = csub(cmul(ts, v), rin);
                    if (gen) o = cadd(o, hsum2[1]);
                    else if (a.s02) o = cfma(a.two_c2, hsum[1], o);
                    a.gout[(size_t)sy.out_b + a.t0 + t - 1] = o;
                }
                if ((sy.flags & SYS_TRACE) && a.trace) a.trace[((size_t)sidx * 2 + 1) * nt + t - 1] = v;
            }
        }
        if (rec_u) {   // u_t of this system in local node order (streaming stores)
            double2* row = a.urec + sy.rec + (size_t)(t - 1) * nj;
#pragma unroll
            for (int i = 0; i < L; ++i)
                if (i < Lp) __stcs(row + sp + 1 + i, u[i]);
            if (realsep) __stcs(row + sp, usep[tid]);
        }
        __syncwarp();
    }
    if constexpr (MODE == 2) {
        // add this segment's sums; every entry has exactly one writer per launch
        if (valid && p < Pj) {
#pragma unroll
            for (int i = 0; i < L; ++i)
                if (i < Lp) a.gint[goff + sp + 1 + i] += ga_int[i];
            a.gl[goff + sp] += ga_l;
            a.gr[goff + sp + Lp + 1] += ga_r;
        }
    }
    // ---- final state ----------------------------------------------------------
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
            // the interface node belongs to the left subdomain
            if ((sy.flags & SYS_WRITE_UT) && a.uT && (sp > 0 || !(tcf & 1))) a.uT[goff + sp] = us;
            if ((sy.flags & SYS_REC_LAST) && a.urec) a.urec[sy.rec + sp] = us;
        }
        if ((sy.flags & SYS_REC_LAST) && a.urec) {
#pragma unroll
            for (int i = 0; i < L; ++i)
                if (i < Lp) a.urec[sy.rec + sp + 1 + i] = u[i];
        }
    }
    if (bad) atomicOr(a.status, ST_NONFINITE);
    // keep this CTA's shared memory alive until every CTA of the cluster is done
    cl.sync();
}

// ---------------------------------------------------------------------------
// Time-dependent potential (Eq. CNS_L with W_n = (V_n + V_{n-1})/2): the matrix
// A_{j,n} - B_j changes every step, so each step refactors in place.  Chunk
// thread: assemble its rows from W_n, LU, local solve and both spikes; the
// separator system (whose coefficients now change every step) is solved by PCR
// updating matrix and right-hand side together.  Entries are pre-scaled by
// 1/(i kappa): D = md/(h/6) + i (sd - wd)/kappa, E = 1 - i (1/h + wo)/kappa.
// ---------------------------------------------------------------------------
struct TdepArgs {
    MarchArgs m;
    const double* V;     // (nt+1) x nx, row n = V(t_n, .)
    long long vstride;   // nx
    double h, kappa;
    double2 sig_ik;      // sigma0 / (i kappa)
};

__device__ __forceinline__ double wat(const double* V0, const double* V1, int g) {
    return 0.5 * (V0[g] + V1[g]);
}

// Scaled diagonal and coupling (i <-> i+1) of local node i of a subdomain with n nodes.
__device__ __forceinline__ double2 tdep_diag(const double* V0, const double* V1, int g, int i,
                                             int n, int tc, double h, double kappa,
                                             double2 sig_ik) {
    const double W0 = wat(V0, V1, g);
    double md = 0.0, sd = 0.0, wd = 0.0;
    if (i > 0) {
        md += h / 3.0;
        sd += 1.0 / h;
        wd += h / 12.0 * (wat(V0, V1, g - 1) + 3.0 * W0);
    }
    if (i < n - 1) {
        md += h / 3.0;
        sd += 1.0 / h;
        wd += h / 12.0 * (3.0 * W0 + wat(V0, V1, g + 1));
    }
    double2 D = make_double2(md / (h / 6.0), (sd - wd) / kappa);
    if ((i == 0 && (tc & 1)) || (i == n - 1 && (tc & 2))) D = csub(D, sig_ik);
    return D;
}
__device__ __forceinline__ double2 tdep_off(const double* V0, const double* V1, int g, double h,
                                            double kappa) {
    const double wo = h / 12.0 * (wat(V0, V1, g) + wat(V0, V1, g + 1));
    return make_double2(1.0, -(1.0 / h + wo) / kappa);
}

template <int L>
__global__ void __launch_bounds__(256, 1) k_march_tdep(const TdepArgs ta) {
    const MarchArgs& a = ta.m;
    extern __shared__ double2 sm[];
    const int T = a.T, G = a.G, P = a.P, C = a.C, nt = a.nt, levels = a.levels;
    const int S = T + G;
    double2* usep = sm;
    // PCR buffers: set b (0/1), quantity q (0 lower, 1 diag, 2 upper, 3 rhs)
    auto PC = [&](int b, int q) -> double2* { return usep + S * (1 + b * 4 + q); };
    double2* cb = usep + S * 9;      // 8 per-chunk arrays of T
    double2* ufst = cb;
    double2* ulst = cb + T;
    double2* yfst = cb + 2 * T;
    double2* ylst = cb + 3 * T;
    double2* afst = cb + 4 * T;
    double2* bfst = cb + 5 * T;
    double2* alst = cb + 6 * T;
    double2* blst = cb + 7 * T;
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
    auto CHK = [&](double2* arr, int pcn) -> double2* {
        if (C == 1) return arr + g * P + pcn;
        const int home = pcn / T;
        double2* base = (home == rank) ? arr : cl.map_shared_rank(arr, home);
        return base + (pcn - home * T);
    };
    auto SYNC = [&]() {
        if (C == 1)
            __syncthreads();
        else
            cl.sync();
    };
    const double2 zero = make_double2(0.0, 0.0);
    MarchSys sy = {0, 0, 0, -1, -1, -1, -1, 0};
    int j = 0, Pj = 0, Lp = 0, sp = 0, goff = 0, tcf = 0, n = 0;
    if (valid) {
        sy = a.sys[sidx];
        j = sy.sub;
        Pj = a.sub_P[j];
        goff = a.sub_goff[j];
        tcf = a.sub_tc[j];
        n = a.sub_n[j];
        Lp = (p < P) ? a.clen[j * P + p] : 0;
        sp = a.sep_pos[j * (P + 1) + p];
    }
    const bool zero_u0 = (sy.flags & SYS_ZERO_U0) != 0;
    const bool realsep = valid && (p <= Pj);
    const double h = ta.h, kappa = ta.kappa;

    double2 u[L], y[L], av[L], bv[L];
#pragma unroll
    for (int i = 0; i < L; ++i) {
        u[i] = (valid && i < Lp && !zero_u0) ? a.u0[goff + sp + 1 + i] : zero;
        y[i] = zero;
        av[i] = zero;
        bv[i] = zero;
    }
    if (valid) *SEP(usep, p) = (realsep && !zero_u0) ? a.u0[goff + sp] : zero;
    SYNC();

    double2 lin = zero, rin = zero;
    for (int t = 1; t <= nt; ++t) {
        const double* V0 = ta.V + (size_t)(t - 1) * ta.vstride;
        const double* V1 = ta.V + (size_t)t * ta.vstride;
        // ---- phase A: assemble, factor, local solve and spikes -----------------
        if (valid && Lp > 0) {
            const double2 uL = *SEP(usep, p), uR = *SEP(usep, p + 1);
            const int g0 = goff + sp + 1;           // global index of the first interior node
            double2 qv[L], cv[L];
            double2 zprev = zero, zaprev = zero, cprev = zero, Eprev = zero, uf = zero, ul = zero;
            const double2 Es = tdep_off(V0, V1, g0 - 1, h, kappa);
            double2 Elast = zero;
#pragma unroll
            for (int i = 0; i < L; ++i) {
                if (i < Lp) {
                    const int li = sp + 1 + i;
                    const double2 Di = tdep_diag(V0, V1, g0 + i, li, n, tcf, h, kappa, ta.sig_ik);
                    const double2 Ei = tdep_off(V0, V1, g0 + i, h, kappa);   // i <-> i+1
                    const double2 piv = (i == 0) ? Di : cfms(Eprev, cprev, Di);
                    qv[i] = crcp(piv);
                    cv[i] = (i < Lp - 1) ? cmul(Ei, qv[i]) : zero;
                    Elast = csel(i == Lp - 1, Ei, Elast);
                    const double2 left = (i == 0) ? uL : u[i - 1];
                    double2 right;
                    if (i + 1 < L)
                        right = (i == Lp - 1) ? uR : u[i + 1];
                    else
                        right = uR;
                    const double2 f = make_double2(fma(4.0, u[i].x, left.x + right.x),
                                                   fma(4.0, u[i].y, left.y + right.y));
                    const double2 z = (i == 0) ? f : cfms(cprev, zprev, f);
                    const double2 za = (i == 0) ? Es : cfms(cprev, zaprev, zero);
                    y[i] = z;
                    av[i] = za;
                    zprev = z;
                    zaprev = za;
                    cprev = cv[i];
                    Eprev = Ei;
                    if (i == 0) uf = u[i];
                    ul = csel(i == Lp - 1, u[i], ul);
                }
            }
            double2 yn = zero, an = zero, bn = zero;
#pragma unroll
            for (int i = L - 1; i >= 0; --i) {
                if (i < Lp) {
                    double2 yi = cmul(qv[i], y[i]), ai = cmul(qv[i], av[i]), bi;
                    if (i == Lp - 1) {
                        bi = cmul(qv[i], Elast);
                    } else {
                        yi = cfms(cv[i], yn, yi);
                        ai = cfms(cv[i], an, ai);
                        bi = cfms(cv[i], bn, zero);
                    }
                    y[i] = yi;
                    av[i] = ai;
                    bv[i] = bi;
                    yn = yi;
                    an = ai;
                    bn = bi;
                }
            }
            *CHK(ufst, p) = uf;
            *CHK(ulst, p) = ul;
            *CHK(yfst, p) = y[0];
            double2 yl = zero, al = zero, bl = zero;
#pragma unroll
            for (int i = 0; i < L; ++i) {
                yl = csel(i == Lp - 1, y[i], yl);
                al = csel(i == Lp - 1, av[i], al);
                bl = csel(i == Lp - 1, bv[i], bl);
            }
            *CHK(ylst, p) = yl;
            *CHK(afst, p) = av[0];
            *CHK(bfst, p) = bv[0];
            *CHK(alst, p) = al;
            *CHK(blst, p) = bl;
        }
        SYNC();
        // ---- phase B: separator row of the reduced system ----------------------
        if (valid) {
            double2 lo = zero, dg = make_double2(1.0, 0.0), up = zero, r = zero;
            if (realsep) {
                const int gs = goff + sp;
                const bool le = (p == 0), re = (p == Pj);
                const double2 us = *SEP(usep, p);
                const double2 um = le ? zero : *CHK(ulst, p - 1);
                const double2 upv = re ? zero : *CHK(ufst, p);
                double2 f;
                if (le)
                    f = make_double2(fma(2.0, us.x, upv.x), fma(2.0, us.y, upv.y));
                else if (re)
                    f = make_double2(fma(2.0, us.x, um.x), fma(2.0, us.y, um.y));
                else
                    f = make_double2(fma(4.0, us.x, um.x + upv.x), fma(4.0, us.y, um.y + upv.y));
                if (le && (tcf & 1)) {
                    if (sy.flags & SYS_IMP_L)
                        lin = (t == 1) ? make_double2(1.0, 0.0) : zero;
                    else
                        lin = (sy.in_l >= 0 && a.gin) ? a.gin[(size_t)sy.in_l + t - 1] : zero;
                    f = cfms(lin, a.inv_ik, f);
                }
                if (re && (tcf & 2)) {
                    if (sy.flags & SYS_IMP_R)
                        rin = (t == 1) ? make_double2(1.0, 0.0) : zero;
                    else
                        rin = (sy.in_r >= 0 && a.gin) ? a.gin[(size_t)sy.in_r + t - 1] : zero;
                    f = cfms(rin, a.inv_ik, f);
                }
                dg = tdep_diag(V0, V1, gs, sp, n, tcf, h, kappa, ta.sig_ik);
                r = f;
                if (!le) {
                    const double2 EL = tdep_off(V0, V1, gs - 1, h, kappa);
                    dg = cfms(EL, *CHK(blst, p - 1), dg);
                    lo = cmul(make_double2(-EL.x, -EL.y), *CHK(alst, p - 1));
                    r = cfms(EL, *CHK(ylst, p - 1), r);
                }
                if (!re) {
                    const double2 ER = tdep_off(V0, V1, gs, h, kappa);
                    dg = cfms(ER, *CHK(afst, p), dg);
                    up = cmul(make_double2(-ER.x, -ER.y), *CHK(bfst, p));
                    r = cfms(ER, *CHK(yfst, p), r);
                }
            }
            *SEP(PC(0, 0), p) = lo;
            *SEP(PC(0, 1), p) = dg;
            *SEP(PC(0, 2), p) = up;
            *SEP(PC(0, 3), p) = r;
        }
        SYNC();
        // ---- phase C: PCR with coefficient updates -----------------------------
        int cur = 0;
        for (int k = 0; k < levels; ++k) {
            const int st = 1 << k;
            if (valid) {
                double2 l0 = *SEP(PC(cur, 0), p), d0 = *SEP(PC(cur, 1), p);
                double2 u0v = *SEP(PC(cur, 2), p), r0 = *SEP(PC(cur, 3), p);
                double2 nl = zero, nu = zero, nd = d0, nr = r0;
                if (p - st >= 0) {
                    const double2 al = cmul(make_double2(-l0.x, -l0.y), crcp(*SEP(PC(cur, 1), p - st)));
                    nl = cmul(al, *SEP(PC(cur, 0), p - st));
                    nd = cfma(al, *SEP(PC(cur, 2), p - st), nd);
                    nr = cfma(al, *SEP(PC(cur, 3), p - st), nr);
                }
                if (p + st <= P) {
                    const double2 ga = cmul(make_double2(-u0v.x, -u0v.y), crcp(*SEP(PC(cur, 1), p + st)));
                    nu = cmul(ga, *SEP(PC(cur, 2), p + st));
                    nd = cfma(ga, *SEP(PC(cur, 0), p + st), nd);
                    nr = cfma(ga, *SEP(PC(cur, 3), p + st), nr);
                }
                *SEP(PC(cur ^ 1, 0), p) = nl;
                *SEP(PC(cur ^ 1, 1), p) = nd;
                *SEP(PC(cur ^ 1, 2), p) = nu;
                *SEP(PC(cur ^ 1, 3), p) = (k == levels - 1) ? cmul(nr, crcp(nd)) : nr;
            }
            SYNC();
            cur ^= 1;
        }
        double2* vs = PC(cur, 3);
        // ---- phase D: spike correction, CN update, fluxes ----------------------
        if (valid && Lp > 0) {
            const double2 vL = *SEP(vs, p), vR = *SEP(vs, p + 1);
#pragma unroll
            for (int i = 0; i < L; ++i) {
                if (i < Lp) {
                    double2 v = cfms(av[i], vL, y[i]);
                    v = cfms(bv[i], vR, v);
                    u[i] = make_double2(fma(2.0, v.x, -u[i].x), fma(2.0, v.y, -u[i].y));
                }
            }
        }
        if (realsep) {
            const double2 v = *SEP(vs, p);
            double2* us = SEP(usep, p);
            const double2 uo = *us;
            *us = make_double2(fma(2.0, v.x, -uo.x), fma(2.0, v.y, -uo.y));
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
        SYNC();
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
    }
    if (bad) atomicOr(a.status, ST_NONFINITE);
    if (C > 1) cl.sync();
}

int swr_march_tdep_smem_bytes(int T, int G) { return (int)sizeof(double2) * (9 * (T + G) + 8 * T); }

template <int L>
static int launch_tdep_t(TdepArgs ta, int ngroups, cudaStream_t s) {
    const int smem = swr_march_tdep_smem_bytes(ta.m.T, ta.m.G);
    auto kern = k_march_tdep<L>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
        return -1;
    if (ta.m.C > 8 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return -1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ngroups * ta.m.C);
    cfg.blockDim = dim3(ta.m.T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ta.m.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    swr_count_launch(1);
    return cudaLaunchKernelEx(&cfg, kern, ta) == cudaSuccess ? 0 : -1;
}

int swr_launch_march_tdep(const FactorSet& fs, MarchArgs a, const double* V, long long vstride,
                          double h, double kappa, double2 sig_ik, int ngroups, cudaStream_t s) {
    if (a.s02) return -2;   // no S_0^2 history terms in the refactorising march
    a.P = fs.P;
    a.levels = fs.levels;
    a.sub_P = fs.sub_P;
    a.sep_pos = fs.sep_pos;
    a.clen = fs.clen;
    a.fac = nullptr;
    a.sep = nullptr;
    a.pcr = nullptr;
    TdepArgs ta{a, V, vstride, h, kappa, sig_ik};
    switch (fs.L) {
        case 4: return launch_tdep_t<4>(ta, ngroups, s);
        case 8: return launch_tdep_t<8>(ta, ngroups, s);
        default: return -2;
    }
}

template <int L>
static int launch_march_t(MarchArgs a, int ngroups, cudaStream_t s, int mode) {
    const int slots = a.stage == 2 ? 2 * a.levels + 3 + 4 * L : (a.stage == 1 ? 2 * a.levels + 3 : 0);
    int smem = swr_march_smem_bytes(a.T, a.G, slots);
    void (*kern)(const MarchArgs) = a.kap ? k_march_static<L, 0, true> : k_march_static<L, 0>;
    if (!a.kap && !a.s02 && a.C == 1) kern = k_march_static<L, 0, false, true>;
    // a system spread over a cluster, or alone in its CTA: the two-level separator
    // solve (one cluster / CTA barrier per step) when its data was factored
    const bool one_system = (a.C > 1) || (a.G == 1 && !a.rag);
    if (one_system && mode == 0 && a.stage == 0 && a.fstride == 0 && a.tl_pcr &&
        (a.T & 31) == 0) {
        kern = a.kap ? k_march_tl<L, true> : k_march_tl<L, false>;
        smem = swr_march_tl_smem_bytes(a.T);
    }
    if constexpr (L <= 8) {   // record and gradient modes exist for L <= 8
        if (mode == 1) kern = k_march_static<L, 1>;
        if (mode == 2) kern = k_march_static<L, 2>;
        // ... and in the two-level form for a system spread over a cluster or alone in its
        // CTA with Robin or Neumann ends
        if ((mode == 1 || mode == 2) && one_system && a.stage == 0 && a.fstride == 0 &&
            a.tl_pcr && !a.s02 && !a.kap && (a.T & 31) == 0 && (mode == 1 || a.T <= 256)) {
            kern = (mode == 1) ? k_march_tl<L, false, 1> : k_march_tl<L, false, 2>;
            smem = swr_march_tl_smem_bytes(a.T);
        }
    }
    if (mode != 0 && a.kap) return -2;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
        return -1;
    if (a.C > 8 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return -1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ngroups * a.C);
    cfg.blockDim = dim3(a.T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = a.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    swr_count_launch(1);
    return cudaLaunchKernelEx(&cfg, kern, a) == cudaSuccess ? 0 : -1;
}

int swr_launch_march(const FactorSet& fs, MarchArgs a, int ngroups, cudaStream_t s, int mode) {
    if (fs.nsteps > 1) {
        // the launch's steps must lie inside the per-step factor sets
        const long long last = a.frev ? (long long)a.fstep0 - (a.nt - 1) : (long long)a.fstep0 + a.nt - 1;
        if (a.fstep0 < 0 || a.fstep0 >= fs.nsteps || last < 0 || last >= fs.nsteps) return -2;
    }
    a.fstride = fs.fstride;
    a.sstride = fs.sstride;
    a.pstride = fs.pstride;
    // streamed factors: stage them in shared memory when the slots fit (200 KB budget)
    a.stage = 0;
    if (fs.nsteps > 1) {
        const int npc = 2 * fs.levels + 3;
        const int budget = 200 * 1024;
        if (swr_march_smem_bytes(a.T, a.G, npc + 4 * fs.L) <= budget)
            a.stage = 2;
        else if (swr_march_smem_bytes(a.T, a.G, npc) <= budget)
            a.stage = 1;
    }
    a.P = fs.P;
    a.levels = fs.levels;
    a.sub_P = fs.sub_P;
    a.sep_pos = fs.sep_pos;
    a.clen = fs.clen;
    a.fac = fs.fac;
    a.sep = fs.sep;
    a.pcr = fs.pcr;
    if (fs.nsteps > 1) {   // start at step fstep0's factors; walk backwards when frev
        a.fac += (size_t)a.fstep0 * fs.fstride;
        a.sep += (size_t)a.fstep0 * fs.sstride;
        a.pcr += (size_t)a.fstep0 * fs.pstride;
        if (a.frev) {
            a.fstride = -a.fstride;
            a.sstride = -a.sstride;
            a.pstride = -a.pstride;
        }
    }
    // the constant-matrix two-level march reads the one-warp reduced system only
    a.tl_pcr = (fs.tl_ok && fs.tl_rs == 32) ? fs.tl_pcr : nullptr;
    a.tl_aux = fs.tl_aux;
    a.tl_red = fs.tl_red;
    a.tl_rs = fs.tl_rs;
    a.tl_rl = fs.tl_rl;
    if (!a.two_level) a.tl_pcr = nullptr;
    // adjoint modes: L <= 8, Robin or S_0^2 (not the per-end kernels)
    if (mode != 0 && (fs.L > 8 || a.kap)) return -2;
    switch (fs.L) {
        case 4: return launch_march_t<4>(a, ngroups, s, mode);
        case 8: return launch_march_t<8>(a, ngroups, s, mode);
        case 12: return launch_march_t<12>(a, ngroups, s, 0);
        case 16: return launch_march_t<16>(a, ngroups, s, 0);
        default: return -2;
    }
}
