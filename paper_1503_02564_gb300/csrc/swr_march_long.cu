// Long subdomains.  A system too long for one thread-block cluster (more than 16 CTAs
// of chunks) is marched by the whole grid: the chunk state u and the partial solves y
// live in global memory (element-major [system][L][P], coalesced over chunks), every
// thread takes chunks and separators in grid-stride order, and the phases of a time step
// — chunk right-hand sides and LU sweeps, separator right-hand sides, the PCR levels over
// the separators, the spike correction and CN update — are separated by grid-wide
// barriers (one cooperative launch, all CTAs resident; every wait bounded).  The
// arithmetic is that of k_march_static: the same factors (FactorSet), the same order of
// operations per node, the same transmission-condition terms at the ends (Robin, S_0^2
// and the per-end kernels of the higher-order conditions).
#include <algorithm>

#include <cuda/atomic>

#include "swr_internal.cuh"

namespace {
constexpr long long kBarrierPolls = 4000000;   // about 1-2 s with the back-off below
}

// Grid-wide barrier on bar[0] (arrivals) and bar[1] (generation).  Thread 0 of each CTA
// arrives; the last arrival resets the count and opens the next generation.  Returns
// false once any CTA has timed out (the abort flag), so that all CTAs leave together.
__device__ bool long_barrier(unsigned int* bar, unsigned int nblocks, int* abortf, int* status) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(bar[0]);
        cuda::atomic_ref<unsigned int, cuda::thread_scope_device> gen(bar[1]);
        cuda::atomic_ref<int, cuda::thread_scope_device> ab(*abortf);
        ok = 1;
        const unsigned int g = gen.load(cuda::memory_order_acquire);
        if (cnt.fetch_add(1u, cuda::memory_order_acq_rel) == nblocks - 1) {
            cnt.store(0u, cuda::memory_order_relaxed);
            gen.store(g + 1u, cuda::memory_order_release);
        } else {
            long long polls = 0;
            while (gen.load(cuda::memory_order_acquire) == g) {
                if (ab.load(cuda::memory_order_relaxed) != 0) { ok = 0; break; }
                if (++polls > kBarrierPolls) {
                    atomicOr(status, ST_TIMEOUT);
                    ab.store(1, cuda::memory_order_relaxed);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        if (ab.load(cuda::memory_order_relaxed) != 0) ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

struct LongScratch {
    double2* ust;       // chunk state u, [sys][L][P]
    double2* yst;       // chunk solves y, [sys][L][P]
    double2* usep;      // separator state u, [sys][P+1]
    double2* dA;        // separator right-hand sides / PCR ping-pong, [sys][P+1]
    double2* dB;
    double2* cend;      // chunk ends [sys][4][P]: u first, u last, y first, y last
    double2* hs;        // history sums [sys][2 ends][2] (own operator, flux operator)
    unsigned int* bar;  // barrier count and generation
    int* abortf;
};

template <int L>
__global__ void __launch_bounds__(256) k_march_long(const MarchArgs a, const LongScratch sc) {
    const int P = a.P, levels = a.levels, nt = a.nt, nsys = a.nsys;
    const size_t S1 = (size_t)P + 1;
    const long long gthreads = (long long)gridDim.x * blockDim.x;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned int nblocks = gridDim.x;
    const double2 zero = make_double2(0.0, 0.0);
    const bool gen = a.kap != nullptr;
    const long long nchunk = (long long)nsys * P, nsepa = (long long)nsys * (long long)S1;
    auto ST = [&](double2* base, int s, int i, int p) -> double2& {
        return base[((size_t)s * L + i) * P + p];
    };

    // ---- initial state and the ends' traces ----------------------------------------
    for (long long c = gtid; c < nchunk; c += gthreads) {
        const int s = (int)(c / P), p = (int)(c % P);
        const MarchSys sy = a.sys[s];
        const int j = sy.sub;
        const int Lp = a.clen[j * P + p];
        const int sp = a.sep_pos[(size_t)j * S1 + p];
        const int goff = a.sub_goff[j];
        const bool zu = (sy.flags & SYS_ZERO_U0) != 0;
        for (int i = 0; i < L; ++i)
            ST(sc.ust, s, i, p) = (i < Lp && !zu) ? a.u0[goff + sp + 1 + i] : zero;
    }
    for (long long q = gtid; q < nsepa; q += gthreads) {
        const int s = (int)(q / S1), p = (int)(q % S1);
        const MarchSys sy = a.sys[s];
        const int j = sy.sub, Pj = a.sub_P[j];
        const int sp = a.sep_pos[(size_t)j * S1 + p];
        const bool zu = (sy.flags & SYS_ZERO_U0) != 0;
        const double2 u0s = (p <= Pj && !zu) ? a.u0[a.sub_goff[j] + sp] : zero;
        sc.usep[q] = u0s;
        if (a.s02 && p <= Pj) {
            const int tcf = a.sub_tc[j];
            for (int side = 0; side < 2; ++side) {
                if (!((side == 0 && p == 0) || (side == 1 && p == Pj))) continue;
                if (!(tcf & (1 << side))) continue;
                double2 h0 = u0s;
                if (gen) h0 = cmul(a.rho[2 * j + side], h0);
                a.hist[((size_t)s * 2 + side) * (nt + 1)] = h0;
            }
        }
    }
    if (!long_barrier(sc.bar, nblocks, sc.abortf, a.status)) return;

    for (int t = 1; t <= nt; ++t) {
        // ---- phase A: chunk right-hand sides and LU sweeps; the ends' histories -------
        for (long long c = gtid; c < nchunk; c += gthreads) {
            const int s = (int)(c / P), p = (int)(c % P);
            const MarchSys sy = a.sys[s];
            const int j = sy.sub;
            const int Lp = a.clen[j * P + p];
            if (Lp == 0) continue;
            const double2* F = a.fac + (size_t)j * L * 4 * P + p;
            const double2 uL = sc.usep[(size_t)s * S1 + p], uR = sc.usep[(size_t)s * S1 + p + 1];
            double2 u[L], y[L];
#pragma unroll
            for (int i = 0; i < L; ++i) u[i] = (i < Lp) ? ST(sc.ust, s, i, p) : zero;
            double2 zprev = zero, cprev = zero, uf = zero, ul = zero;
#pragma unroll
            for (int i = 0; i < L; ++i) {
                y[i] = zero;
                if (i < Lp) {
                    const double2 left = (i == 0) ? uL : u[i - 1];
                    double2 right;
                    if (i + 1 < L)
                        right = (i == Lp - 1) ? uR : u[i + 1];
                    else
                        right = uR;
                    const double2 f = make_double2(fma(4.0, u[i].x, left.x + right.x),
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
                    double2 yi = cmul(F[(i * 4 + 0) * P], y[i]);
                    if (i != Lp - 1) yi = cfms(F[(i * 4 + 1) * P], ynext, yi);
                    else yl = yi;
                    y[i] = yi;
                    ynext = yi;
                }
            }
#pragma unroll
            for (int i = 0; i < L; ++i)
                if (i < Lp) ST(sc.yst, s, i, p) = y[i];
            double2* ce = sc.cend + (size_t)s * 4 * P;
            ce[0 * P + p] = uf;
            ce[1 * P + p] = ul;
            ce[2 * P + p] = y[0];
            ce[3 * P + p] = yl;
        }
        if (a.s02) {
            // one warp per end of every system: the history sums of step t
            const long long gw = gtid >> 5;
            const int lane = threadIdx.x & 31;
            for (long long e = gw; e < 2LL * nsys; e += gthreads >> 5) {
                const int s = (int)(e >> 1), side = (int)(e & 1);
                const int j = a.sys[s].sub;
                if (!(a.sub_tc[j] & (1 << side))) continue;
                const double2* hh = a.hist + ((size_t)s * 2 + side) * (nt + 1);
                double2 o1, o2;
                if (gen) {
                    const size_t ke = (size_t)(2 * j + side) * a.kstride;
                    conv_history2(a.kap + ke, a.kout + ke, hh, t, lane, o1, o2);
                } else {
                    o1 = s02_history(a.beta, hh, t, lane);
                    o2 = o1;
                }
                if (lane == 0) {
                    sc.hs[e * 2 + 0] = o1;
                    sc.hs[e * 2 + 1] = o2;
                }
            }
        }
        if (!long_barrier(sc.bar, nblocks, sc.abortf, a.status)) return;
        // ---- phase B: reduced right-hand sides at the separators -----------------------
        for (long long q = gtid; q < nsepa; q += gthreads) {
            const int s = (int)(q / S1), p = (int)(q % S1);
            const MarchSys sy = a.sys[s];
            const int j = sy.sub, Pj = a.sub_P[j], tcf = a.sub_tc[j];
            double2 d = zero;
            if (p <= Pj) {
                const double2* ce = sc.cend + (size_t)s * 4 * P;
                const double2 us = sc.usep[q];
                const bool le = (p == 0), re = (p == Pj);
                const double2 um = le ? zero : ce[1 * P + p - 1];
                const double2 up = re ? zero : ce[0 * P + p];
                double2 f;
                if (le)
                    f = make_double2(fma(2.0, us.x, up.x), fma(2.0, us.y, up.y));
                else if (re)
                    f = make_double2(fma(2.0, us.x, um.x), fma(2.0, us.y, um.y));
                else
                    f = make_double2(fma(4.0, us.x, um.x + up.x), fma(4.0, us.y, um.y + up.y));
                const double2 hmul = gen ? a.inv_ik : a.c2_ik;
                if (le && (tcf & 1)) {
                    double2 lin;
                    if (sy.flags & SYS_IMP_L)
                        lin = (t == 1) ? make_double2(1.0, 0.0) : zero;
                    else
                        lin = (sy.in_l >= 0 && a.gin) ? a.gin[(size_t)sy.in_l + t - 1] : zero;
                    f = cfms(lin, a.inv_ik, f);
                    if (a.s02) f = cfma(sc.hs[((size_t)s * 2 + 0) * 2 + 0], hmul, f);
                }
                if (re && (tcf & 2)) {
                    double2 rin;
                    if (sy.flags & SYS_IMP_R)
                        rin = (t == 1) ? make_double2(1.0, 0.0) : zero;
                    else
                        rin = (sy.in_r >= 0 && a.gin) ? a.gin[(size_t)sy.in_r + t - 1] : zero;
                    f = cfms(rin, a.inv_ik, f);
                    if (a.s02) f = cfma(sc.hs[((size_t)s * 2 + 1) * 2 + 0], hmul, f);
                }
                d = f;
                const double2 El = a.sep[(size_t)(j * 3 + 0) * S1 + p];
                const double2 Er = a.sep[(size_t)(j * 3 + 1) * S1 + p];
                if (!le) d = cfms(El, ce[3 * P + p - 1], d);
                if (!re) d = cfms(Er, ce[2 * P + p], d);
            }
            sc.dA[q] = d;
        }
        if (!long_barrier(sc.bar, nblocks, sc.abortf, a.status)) return;
        // ---- phase C: PCR over the separators (precomputed coefficients) ---------------
        double2* src = sc.dA;
        double2* dst = sc.dB;
        for (int k = 0; k < levels; ++k) {
            const int st = 1 << k;
            for (long long q = gtid; q < nsepa; q += gthreads) {
                const int s = (int)(q / S1), p = (int)(q % S1);
                const int j = a.sys[s].sub;
                const double2* pc = a.pcr + (size_t)j * levels * 2 * S1;
                const double2* row = src + (size_t)s * S1;
                double2 dd = row[p];
                if (p - st >= 0) dd = cfma(pc[(size_t)(k * 2 + 0) * S1 + p], row[p - st], dd);
                if (p + st <= P) dd = cfma(pc[(size_t)(k * 2 + 1) * S1 + p], row[p + st], dd);
                if (k == levels - 1) dd = cmul(dd, a.sep[(size_t)(j * 3 + 2) * S1 + p]);
                dst[q] = dd;
            }
            if (!long_barrier(sc.bar, nblocks, sc.abortf, a.status)) return;
            double2* tmp = src;
            src = dst;
            dst = tmp;
        }
        // ---- phase D: spike correction, CN update, fluxes --------------------------------
        for (long long c = gtid; c < nchunk; c += gthreads) {
            const int s = (int)(c / P), p = (int)(c % P);
            const MarchSys sy = a.sys[s];
            const int j = sy.sub;
            const int Lp = a.clen[j * P + p];
            if (Lp == 0) continue;
            const double2* F = a.fac + (size_t)j * L * 4 * P + p;
            const double2 vL = src[(size_t)s * S1 + p], vR = src[(size_t)s * S1 + p + 1];
            const bool rec = a.urec && (sy.flags & SYS_REC_U);
            const int sp = a.sep_pos[(size_t)j * S1 + p];
            double2* row = rec ? a.urec + sy.rec + (size_t)(t - 1) * a.sub_n[j] : nullptr;
#pragma unroll
            for (int i = 0; i < L; ++i) {
                if (i < Lp) {
                    double2 v = cfms(F[(i * 4 + 2) * P], vL, ST(sc.yst, s, i, p));
                    v = cfms(F[(i * 4 + 3) * P], vR, v);
                    const double2 uo = ST(sc.ust, s, i, p);
                    const double2 un = make_double2(fma(2.0, v.x, -uo.x), fma(2.0, v.y, -uo.y));
                    ST(sc.ust, s, i, p) = un;
                    if (rec) __stcs(row + sp + 1 + i, un);
                }
            }
        }
        for (long long q = gtid; q < nsepa; q += gthreads) {
            const int s = (int)(q / S1), p = (int)(q % S1);
            const MarchSys sy = a.sys[s];
            const int j = sy.sub, Pj = a.sub_P[j], tcf = a.sub_tc[j];
            if (p > Pj) continue;
            const double2 v = src[q];
            const double2 uo = sc.usep[q];
            const double2 un = make_double2(fma(2.0, v.x, -uo.x), fma(2.0, v.y, -uo.y));
            sc.usep[q] = un;
            if (a.urec && (sy.flags & SYS_REC_U))
                a.urec[sy.rec + (size_t)(t - 1) * a.sub_n[j] + a.sep_pos[(size_t)j * S1 + p]] = un;
            for (int side = 0; side < 2; ++side) {
                if (!((side == 0 && p == 0) || (side == 1 && p == Pj))) continue;
                if (!(tcf & (1 << side))) continue;
                if (a.s02) a.hist[((size_t)s * 2 + side) * (nt + 1) + t] = v;
                const int out = side ? sy.out_b : sy.out_a;
                if (out >= 0 && a.gout) {
                    double2 lr;
                    if (sy.flags & (side ? SYS_IMP_R : SYS_IMP_L))
                        lr = (t == 1) ? make_double2(1.0, 0.0) : zero;
                    else {
                        const int in = side ? sy.in_r : sy.in_l;
                        lr = (in >= 0 && a.gin) ? a.gin[(size_t)in + t - 1] : zero;
                    }
                    const double2 ts = gen ? a.kout[(size_t)(2 * j + side) * a.kstride] : a.two_sigma;
                    double2 o = csub(cmul(ts, v), lr);
                    if (gen) o = cadd(o, sc.hs[((size_t)s * 2 + side) * 2 + 1]);
                    else if (a.s02) o = cfma(a.two_c2, sc.hs[((size_t)s * 2 + side) * 2 + 0], o);
                    a.gout[(size_t)out + t - 1] = o;
                }
                if ((sy.flags & SYS_TRACE) && a.trace)
                    a.trace[((size_t)s * 2 + side) * nt + t - 1] = v;
            }
        }
        if (!long_barrier(sc.bar, nblocks, sc.abortf, a.status)) return;
    }
    // ---- final state ---------------------------------------------------------------------
    bool bad = false;
    for (long long c = gtid; c < nchunk; c += gthreads) {
        const int s = (int)(c / P), p = (int)(c % P);
        const MarchSys sy = a.sys[s];
        const int j = sy.sub;
        const int Lp = a.clen[j * P + p];
        const int sp = a.sep_pos[(size_t)j * S1 + p];
        const int goff = a.sub_goff[j];
        for (int i = 0; i < Lp; ++i) {
            const double2 u = ST(sc.ust, s, i, p);
            bad |= !cfinite(u);
            if ((sy.flags & SYS_WRITE_UT) && a.uT) a.uT[goff + sp + 1 + i] = u;
            if ((sy.flags & SYS_REC_LAST) && a.urec) a.urec[sy.rec + sp + 1 + i] = u;
        }
    }
    for (long long q = gtid; q < nsepa; q += gthreads) {
        const int s = (int)(q / S1), p = (int)(q % S1);
        const MarchSys sy = a.sys[s];
        const int j = sy.sub, Pj = a.sub_P[j], tcf = a.sub_tc[j];
        if (p > Pj) continue;
        const int sp = a.sep_pos[(size_t)j * S1 + p];
        const double2 us = sc.usep[q];
        bad |= !cfinite(us);
        if ((sy.flags & SYS_WRITE_UT) && a.uT && (sp > 0 || !(tcf & 1))) a.uT[a.sub_goff[j] + sp] = us;
        if ((sy.flags & SYS_REC_LAST) && a.urec) a.urec[sy.rec + sp] = us;
    }
    if (bad) atomicOr(a.status, ST_NONFINITE);
}

size_t swr_long_scratch_bytes(int nsys, int L, int P) {
    const size_t S1 = (size_t)P + 1;
    return sizeof(double2) * ((size_t)nsys * (2 * (size_t)L * P + 3 * S1 + 4 * (size_t)P + 4)) +
           sizeof(unsigned int) * 2 + sizeof(int) * 2;
}

// One cooperative launch over all systems of the list; fs must hold L = 16 factors.
int swr_launch_march_long(const FactorSet& fs, MarchArgs a, void* scratch, size_t scratch_bytes,
                          int nsm, cudaStream_t s) {
    if (fs.L != 16 || fs.nsteps != 1 || a.nsys <= 0) return -2;
    const int P = fs.P;
    if (swr_long_scratch_bytes(a.nsys, 16, P) > scratch_bytes) return -2;
    a.P = P;
    a.levels = fs.levels;
    a.sub_P = fs.sub_P;
    a.sep_pos = fs.sep_pos;
    a.clen = fs.clen;
    a.fac = fs.fac;
    a.sep = fs.sep;
    a.pcr = fs.pcr;
    const size_t S1 = (size_t)P + 1;
    LongScratch sc;
    double2* b = static_cast<double2*>(scratch);
    sc.ust = b;
    sc.yst = sc.ust + (size_t)a.nsys * 16 * P;
    sc.usep = sc.yst + (size_t)a.nsys * 16 * P;
    sc.dA = sc.usep + (size_t)a.nsys * S1;
    sc.dB = sc.dA + (size_t)a.nsys * S1;
    sc.cend = sc.dB + (size_t)a.nsys * S1;
    sc.hs = sc.cend + (size_t)a.nsys * 4 * P;
    sc.bar = reinterpret_cast<unsigned int*>(sc.hs + (size_t)a.nsys * 4);
    sc.abortf = reinterpret_cast<int*>(sc.bar + 2);
    if (cudaMemsetAsync(sc.bar, 0, sizeof(unsigned int) * 2 + sizeof(int) * 2, s) != cudaSuccess)
        return -1;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march_long<16>, 256, 0) !=
            cudaSuccess || per <= 0)
        return -1;
    const long long work = (long long)a.nsys * (P + 1);
    int nblk = per * nsm;
    if ((long long)nblk * 256 > work) nblk = (int)std::max(1LL, (work + 255) / 256);
    void* args[] = {(void*)&a, (void*)&sc};
    if (cudaLaunchCooperativeKernel((const void*)k_march_long<16>, dim3(nblk), dim3(256), args, 0,
                                    s) != cudaSuccess)
        return -1;
    swr_count_launch(1);
    return 0;
}
