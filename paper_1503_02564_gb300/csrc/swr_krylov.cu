// Interface algebra of the SWR method: the explicit interface operator of
// Algorithm 3 (blocks X^{j,p} are causal Toeplitz, Props. 3-4), the GMRES
// building blocks (Saad's restarted GMRES with classical Gram-Schmidt applied
// twice and Givens rotations), and the time-causal block forward substitution
// that inverts I - L (or I - L_0) block by block in time.
//
// Interface vector: 2N-2 blocks of nt values; block 2k = r_k, block 2k+1 = l_{k+1}
// (0-based subdomains).  First columns: slot 4j + (p-1) holds X^{j,p}, p = 1..4.
//   r_{j-1} = X^{j,1} l_j + X^{j,2} r_j,   l_{j+1} = X^{j,3} l_j + X^{j,4} r_j.
#include <cooperative_groups.h>

#include "swr_internal.cuh"

namespace cg = cooperative_groups;

// Sources of output block o: (column slot, input block) pairs, -1 if absent.
__device__ __forceinline__ void block_sources(int o, int N, int& c1, int& i1, int& c2, int& i2) {
    if ((o & 1) == 0) {          // r_k, produced by subdomain j = k+1
        const int j = o / 2 + 1;
        c1 = 4 * j + 0;
        i1 = 2 * j - 1;
        if (j <= N - 2) {
            c2 = 4 * j + 1;
            i2 = 2 * j;
        } else {
            c2 = -1;
            i2 = -1;
        }
    } else {                     // l_{k+1}, produced by subdomain j = k
        const int j = (o - 1) / 2;
        c1 = 4 * j + 3;
        i1 = 2 * j;
        if (j >= 1) {
            c2 = 4 * j + 2;
            i2 = 2 * j - 1;
        } else {
            c2 = -1;
            i2 = -1;
        }
    }
}

// ---------------------------------------------------------------------------
// y = x - L x (mode 0)  or  y = L x + add (mode 1, the fixed point of Alg. 3).
// One CTA per output block; the two first columns and the two input blocks
// are staged in shared memory (SMEM; read from L2 when they do not fit, nt >
// 3632); thread q computes the causal sums for times q and nt-1-q (equal work
// per thread).
// ---------------------------------------------------------------------------
template <bool SMEM>
__global__ void k_toeplitz(int N, int nt, const double2* __restrict__ cols,
                           const double2* __restrict__ x, const double2* __restrict__ add,
                           double2* __restrict__ y, int mode, const InstInfo* __restrict__ inst,
                           const int* __restrict__ blk_inst) {
    extern __shared__ double2 sh[];
    int o = blockIdx.x;
    if (inst) {   // batched plan: this block's instance
        const InstInfo I = inst[blk_inst[blockIdx.x]];
        N = I.N;
        nt = I.nt;
        o = blockIdx.x - I.blk0;
        cols += I.coff;
        x += I.foff;
        y += I.foff;
        if (add) add += I.foff;
    }
    int c1, i1, c2, i2;
    block_sources(o, N, c1, i1, c2, i2);
    const double2 zero = make_double2(0.0, 0.0);
    const bool two = (c2 >= 0);
    const double2 *C1, *X1, *C2, *X2;
    if constexpr (SMEM) {
        double2* c1s = sh;
        double2* x1s = sh + nt;
        double2* c2s = sh + 2 * nt;
        double2* x2s = sh + 3 * nt;
        for (int t = threadIdx.x; t < nt; t += blockDim.x) {
            c1s[t] = cols[(size_t)c1 * nt + t];
            x1s[t] = x[(size_t)i1 * nt + t];
            c2s[t] = two ? cols[(size_t)c2 * nt + t] : zero;
            x2s[t] = two ? x[(size_t)i2 * nt + t] : zero;
        }
        __syncthreads();
        C1 = c1s;
        X1 = x1s;
        C2 = c2s;
        X2 = x2s;
    } else {
        C1 = cols + (size_t)c1 * nt;
        X1 = x + (size_t)i1 * nt;
        C2 = two ? cols + (size_t)c2 * nt : C1;   // read only when two
        X2 = two ? x + (size_t)i2 * nt : X1;
    }
    for (int q = threadIdx.x; q < (nt + 1) / 2; q += blockDim.x) {
        for (int e = 0; e < 2; ++e) {
            const int n = (e == 0) ? q : nt - 1 - q;
            if (e == 1 && n == q) break;
            double2 acc0 = zero, acc1 = zero;
            int s = 0;
            for (; s + 1 <= n; s += 2) {
                acc0 = cfma(C1[n - s], X1[s], acc0);
                acc1 = cfma(C1[n - s - 1], X1[s + 1], acc1);
            }
            if (s <= n) acc0 = cfma(C1[n - s], X1[s], acc0);
            if (two) {
                s = 0;
                for (; s + 1 <= n; s += 2) {
                    acc0 = cfma(C2[n - s], X2[s], acc0);
                    acc1 = cfma(C2[n - s - 1], X2[s + 1], acc1);
                }
                if (s <= n) acc0 = cfma(C2[n - s], X2[s], acc0);
            }
            const double2 acc = cadd(acc0, acc1);
            const size_t idx = (size_t)o * nt + n;
            y[idx] = (mode == 0) ? csub(x[idx], acc) : cadd(acc, add[idx]);
        }
    }
}

int swr_launch_toeplitz(int N, int nt, const double2* cols, const double2* x, const double2* add,
                        double2* y, int mode, cudaStream_t s, const InstInfo* inst,
                        const int* blk_inst, int nblk_total, int ntmax) {
    const int nblk = inst ? nblk_total : 2 * N - 2;
    const long long smem = 4LL * (inst ? ntmax : nt) * (long long)sizeof(double2);
    if (smem > 227 * 1024) {
        k_toeplitz<false><<<nblk, 256, 0, s>>>(N, nt, cols, x, add, y, mode, inst, blk_inst);
    } else {
        if (cudaFuncSetAttribute(k_toeplitz<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return -1;
        k_toeplitz<true><<<nblk, 256, (int)smem, s>>>(N, nt, cols, x, add, y, mode, inst,
                                                      blk_inst);
    }
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// The same apply through the FFT.  An output block is c1 * x1 + c2 * x2 on
// steps 0..nt-1, each a causal convolution of two length-nt sequences; with a
// transform length M >= 2 nt - 1 (a power of two) the circular convolution of
// the zero-padded sequences equals it on 0..nt-1.  The spectra of the first
// columns are formed once per build (k_col_spectra); an apply transforms the two
// input blocks, multiplies by the spectra, sums and transforms back: 3 M log2 M
// radix-2 butterflies per block in place of nt^2 complex multiply-adds.
// The FFT is a radix-2 Stockham transform (self-sorting, out of place, ping-pong
// between two shared-memory buffers); stage s with m = 2^s: butterfly b = (j, k),
// j = b / m, k = b mod m, l = M / (2m):
//     y[k + 2jm] = x[k + jm] + x[k + jm + lm],
//     y[k + 2jm + m] = W^{jm} (x[k + jm] - x[k + jm + lm]),   W = exp(-2 pi i / M)
// (conj(W) for the inverse).  W^k, k < M/2, comes from a table built on the host.
// ---------------------------------------------------------------------------
__device__ double2* fft_stockham(double2* x, double2* y, int M, int logM,
                                 const double2* __restrict__ W, bool inverse) {
    const int half = M >> 1;
    for (int s = 0; s < logM; ++s) {
        const int m = 1 << s, l = half >> s;
        for (int b = threadIdx.x; b < half; b += blockDim.x) {
            const int j = b >> s, k = b & (m - 1);
            double2 w = __ldg(W + j * m);
            if (inverse) w.y = -w.y;
            const double2 c0 = x[k + j * m], c1 = x[k + j * m + l * m];
            y[k + 2 * j * m] = cadd(c0, c1);
            y[k + 2 * j * m + m] = cmul(w, csub(c0, c1));
        }
        __syncthreads();
        double2* t = x;
        x = y;
        y = t;
    }
    return x;
}

// Instance of a global subdomain (batched plans; inst sorted by sub0).
__device__ __forceinline__ int inst_of_sub(const InstInfo* inst, int ninst, int sub) {
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (inst[mid].sub0 <= sub) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Spectra of the first columns: slot 4 s + q of global subdomain s at spec[(4 s + q) M].
__global__ void k_col_spectra(int nt, const double2* __restrict__ cols, double2* __restrict__ spec,
                              int M, int logM, const double2* __restrict__ W,
                              const InstInfo* __restrict__ inst, int ninst) {
    extern __shared__ double2 sh[];
    const int slot = blockIdx.x;             // 4 s + q
    const double2* c = cols + (size_t)slot * nt;
    if (inst) {
        const InstInfo I = inst[inst_of_sub(inst, ninst, slot >> 2)];
        nt = I.nt;
        c = cols + I.coff + (size_t)(4 * ((slot >> 2) - I.sub0) + (slot & 3)) * I.nt;
    }
    const double2 zero = make_double2(0.0, 0.0);
    for (int t = threadIdx.x; t < M; t += blockDim.x) sh[t] = (t < nt) ? c[t] : zero;
    __syncthreads();
    const double2* r = fft_stockham(sh, sh + M, M, logM, W, false);
    for (int t = threadIdx.x; t < M; t += blockDim.x) spec[(size_t)slot * M + t] = r[t];
}

int swr_launch_col_spectra(int nsub_total, int nt, const double2* cols, double2* spec, int M,
                           const double2* W, cudaStream_t s, const InstInfo* inst, int ninst) {
    int logM = 0;
    while ((1 << logM) < M) ++logM;
    const int smem = 2 * M * (int)sizeof(double2);
    if (cudaFuncSetAttribute(k_col_spectra, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
        return -1;
    k_col_spectra<<<4 * nsub_total, 256, smem, s>>>(nt, cols, spec, M, logM, W, inst, ninst);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// y = x - L x (mode 0) or y = L x + add (mode 1), as k_toeplitz, from the spectra.
__global__ void __launch_bounds__(256) k_toeplitz_fft(
    int N, int nt, const double2* __restrict__ spec, const double2* __restrict__ x,
    const double2* __restrict__ add, double2* __restrict__ y, int mode, int M, int logM,
    const double2* __restrict__ W, const InstInfo* __restrict__ inst,
    const int* __restrict__ blk_inst) {
    extern __shared__ double2 sh[];
    int o = blockIdx.x;
    if (inst) {
        const InstInfo I = inst[blk_inst[blockIdx.x]];
        N = I.N;
        nt = I.nt;
        o = blockIdx.x - I.blk0;
        spec += (size_t)4 * I.sub0 * M;
        x += I.foff;
        y += I.foff;
        if (add) add += I.foff;
    }
    int c1, i1, c2, i2;
    block_sources(o, N, c1, i1, c2, i2);
    double2* A = sh;
    double2* B = sh + M;
    double2* acc = sh + 2 * M;
    const double2 zero = make_double2(0.0, 0.0);
    for (int e = 0; e < 2; ++e) {
        const int ci = e ? c2 : c1, ii = e ? i2 : i1;
        if (ci < 0) break;
        for (int t = threadIdx.x; t < M; t += blockDim.x)
            A[t] = (t < nt) ? x[(size_t)ii * nt + t] : zero;
        __syncthreads();
        const double2* r = fft_stockham(A, B, M, logM, W, false);
        const double2* sc = spec + (size_t)ci * M;
        for (int t = threadIdx.x; t < M; t += blockDim.x) {
            const double2 v = cmul(r[t], sc[t]);
            acc[t] = e ? cadd(acc[t], v) : v;
        }
        __syncthreads();
    }
    const double2* r = fft_stockham(acc, A, M, logM, W, true);
    const double inv = 1.0 / (double)M;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        const size_t idx = (size_t)o * nt + t;
        const double2 v = make_double2(r[t].x * inv, r[t].y * inv);
        y[idx] = (mode == 0) ? csub(x[idx], v) : cadd(v, add[idx]);
    }
}

int swr_launch_toeplitz_fft(int N, int nt, const double2* spec, const double2* x,
                            const double2* add, double2* y, int mode, int M, const double2* W,
                            cudaStream_t s, const InstInfo* inst, const int* blk_inst,
                            int nblk_total) {
    int logM = 0;
    while ((1 << logM) < M) ++logM;
    const int smem = 3 * M * (int)sizeof(double2);
    if (smem > 227 * 1024) return -2;
    if (cudaFuncSetAttribute(k_toeplitz_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
        return -1;
    k_toeplitz_fft<<<inst ? nblk_total : 2 * N - 2, 256, smem, s>>>(
        N, nt, spec, x, add, y, mode, M, logM, W, inst, blk_inst);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// Batched dot products out[i] = V_i^H w, i < nvec (V_i = V + i*ldv), in two
// deterministic passes (per-CTA partial sums, then a fixed-order reduction).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    return v;
}

__global__ void k_dots_partial(const double2* __restrict__ V, long long ldv, int nvec,
                               const double2* __restrict__ w, long long n,
                               double2* __restrict__ partial) {
    __shared__ double2 red[32];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int i = 0; i < nvec; ++i) {
        const double2* vi = V + (size_t)i * ldv;
        double2 acc = make_double2(0.0, 0.0);
        for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride)
            acc = cfma(make_double2(vi[k].x, -vi[k].y), w[k], acc);
        acc = warp_sum(acc);
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) red[wid] = acc;
        __syncthreads();
        if (wid == 0) {
            double2 v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : make_double2(0.0, 0.0);
            v = warp_sum(v);
            if (lane == 0) partial[(size_t)i * gridDim.x + blockIdx.x] = v;
        }
        __syncthreads();
    }
}

__global__ void k_dots_final(const double2* __restrict__ partial, int nblocks, int nvec,
                             double2* __restrict__ out) {
    const int i = blockIdx.x;
    if (i >= nvec) return;
    double2 acc = make_double2(0.0, 0.0);
    for (int b = threadIdx.x; b < nblocks; b += 32) acc = cadd(acc, partial[(size_t)i * nblocks + b]);
    acc = warp_sum(acc);
    if (threadIdx.x == 0) out[i] = acc;
}

int swr_launch_dots(const double2* V, long long ldv, int nvec, const double2* w, long long n,
                    double2* partial, int nblocks, double2* out, cudaStream_t s) {
    k_dots_partial<<<nblocks, 256, 0, s>>>(V, ldv, nvec, w, n, partial);
    k_dots_final<<<nvec, 32, 0, s>>>(partial, nblocks, nvec, out);
    swr_count_launch(2);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// w += sign * sum_i V_i h_i
__global__ void k_gemv(const double2* __restrict__ V, long long ldv, int nvec,
                       const double2* __restrict__ h, double2* __restrict__ w, long long n,
                       double sign) {
    __shared__ double2 hs[256];
    for (int i = threadIdx.x; i < nvec && i < 256; i += blockDim.x)
        hs[i] = make_double2(sign * h[i].x, sign * h[i].y);
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        double2 acc = w[k];
        for (int i = 0; i < nvec; ++i) acc = cfma(hs[i], V[(size_t)i * ldv + k], acc);
        w[k] = acc;
    }
}

int swr_launch_gemv_sub(const double2* V, long long ldv, int nvec, const double2* h, double2* w,
                        long long n, double sign, cudaStream_t s) {
    if (nvec > 256) return -2;
    k_gemv<<<152 * 4, 256, 0, s>>>(V, ldv, nvec, h, w, n, sign);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// y = a*y + b*x
__global__ void k_axpby(double2* __restrict__ y, const double2* __restrict__ x, long long n,
                        double2 a, double2 b) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const double2 yv = (a.x == 0.0 && a.y == 0.0) ? make_double2(0.0, 0.0) : cmul(a, y[k]);
        y[k] = (b.x == 0.0 && b.y == 0.0) ? yv : cfma(b, x[k], yv);
    }
}

int swr_launch_axpby(double2* y, const double2* x, long long n, double2 a, double2 b,
                     cudaStream_t s) {
    k_axpby<<<152 * 4, 256, 0, s>>>(y, x, n, a, b);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// v = w / hdiag[0].x  (hdiag points at the stored norm)
__global__ void k_scale_rnorm(double2* __restrict__ v, const double2* __restrict__ w, long long n,
                              const double2* __restrict__ hnorm) {
    const double nr = hnorm[0].x;
    const double s = (nr > 0.0) ? 1.0 / nr : 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride)
        v[k] = cscale(w[k], s);
}

int swr_launch_scale_by_rnorm(double2* v, const double2* w, long long n, const double2* hnorm,
                              cudaStream_t s) {
    k_scale_rnorm<<<152 * 4, 256, 0, s>>>(v, w, n, hnorm);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// Arnoldi column j finish + Givens rotations (one thread).
// H is column-major with leading dimension ldh = m+1.  On entry column j holds
// h1 (first Gram-Schmidt pass); sv[ldh..] scratch holds h2 (second pass) and the
// squared norm of the orthogonalised vector.  Layout of the scratch area
// work = sv + ldh:  work[0..j] = h2, work[j+1] = (|w|^2, 0).
// After: H(j+1, j) = |w| (stored unrotated in work[ldh], used for scaling),
// rotations applied, sv updated, *res_out = |sv[j+1]|.
// ---------------------------------------------------------------------------
__global__ void k_givens(double2* H, int ldh, double2* cs, double2* sn, double2* sv, int j,
                         double* res_out) {
    double2* col = H + (size_t)j * ldh;
    double2* work = sv + ldh;
    for (int i = 0; i <= j; ++i) col[i] = cadd(col[i], work[i]);
    const double hn = sqrt(fmax(work[j + 1].x, 0.0));
    col[j + 1] = make_double2(hn, 0.0);
    work[ldh] = make_double2(hn, 0.0);
    for (int i = 0; i < j; ++i) {
        const double2 a = col[i], b = col[i + 1];
        // [c s; -conj(s) c], c real
        col[i] = cfma(sn[i], b, cscale(a, cs[i].x));
        col[i + 1] = csub(cscale(b, cs[i].x), cconjmul(sn[i], a));
    }
    const double2 a = col[j], b = col[j + 1];
    const double aa = hypot(a.x, a.y), bb = hypot(b.x, b.y);
    const double den = hypot(aa, bb);
    double c;
    double2 s;
    if (den == 0.0) {
        c = 1.0;
        s = make_double2(0.0, 0.0);
    } else {
        const double2 ph = (aa > 0.0) ? make_double2(a.x / aa, a.y / aa) : make_double2(1.0, 0.0);
        c = aa / den;
        s = cscale(cmul(ph, make_double2(b.x, -b.y)), 1.0 / den);
    }
    cs[j] = make_double2(c, 0.0);
    sn[j] = s;
    col[j] = cfma(s, b, cscale(a, c));
    col[j + 1] = make_double2(0.0, 0.0);
    const double2 sj = sv[j];
    sv[j + 1] = cmul(make_double2(-s.x, s.y), sj);   // -conj(s) * s_j
    sv[j] = cscale(sj, c);
    *res_out = hypot(sv[j + 1].x, sv[j + 1].y);
}

int swr_launch_givens(double2* H, int ldh, double2* cs, double2* sn, double2* sv, int j,
                      double* res_out, cudaStream_t s) {
    k_givens<<<1, 1, 0, s>>>(H, ldh, cs, sn, sv, j, res_out);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Solve the k x k upper-triangular R y = sv (one thread).
__global__ void k_lsq(const double2* H, int ldh, const double2* sv, int k, double2* y) {
    for (int i = k - 1; i >= 0; --i) {
        double2 acc = sv[i];
        for (int c = i + 1; c < k; ++c) acc = cfms(H[(size_t)c * ldh + i], y[c], acc);
        y[i] = cmul(acc, crcp(H[(size_t)i * ldh + i]));
    }
}

int swr_launch_lsq(const double2* H, int ldh, const double2* sv, int k, double2* y,
                   cudaStream_t s) {
    k_lsq<<<1, 1, 0, s>>>(H, ldh, sv, k, y);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// Interface mismatch of the final march: max |v_j(b_j) - v_{j+1}(a_{j+1})|
// (trace buffer [sys][2][nt], systems 0..N-1 are the subdomains in order).
// ---------------------------------------------------------------------------
__global__ void k_jump(const double2* __restrict__ trace, int N, int nt,
                       unsigned long long* out, const InstInfo* __restrict__ inst,
                       const int* __restrict__ if_inst, int nif_total) {
    // trace rows have stride nt (the longest instance); interface k lies between
    // subdomains j and j+1 of its instance
    double m = 0.0;
    const long long tot = (long long)(inst ? nif_total : N - 1) * nt;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < tot;
         q += (long long)gridDim.x * blockDim.x) {
        int j = (int)(q / nt);
        const int n = (int)(q % nt);
        if (inst) {
            const InstInfo I = inst[if_inst[j]];
            if (n >= I.nt) continue;
            j = I.sub0 + (j - I.if0);
        }
        const double2 a = trace[((size_t)j * 2 + 1) * nt + n];
        const double2 b = trace[((size_t)(j + 1) * 2 + 0) * nt + n];
        m = fmax(m, hypot(a.x - b.x, a.y - b.y));
    }
    atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

int swr_launch_jump(const double2* trace, const MarchSys*, int N, int nt, double* out,
                    cudaStream_t s, const InstInfo* inst, const int* if_inst, int nif_total) {
    cudaMemsetAsync(out, 0, sizeof(double), s);
    k_jump<<<64, 256, 0, s>>>(trace, N, nt, reinterpret_cast<unsigned long long*>(out), inst,
                              if_inst, nif_total);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// The same mismatch without a final march.  With w = R(g) = L g + d, the fluxes
// of Eq. TransmisionCond give 2 S v_j(b_j) = w[l_{k+1}] + g[r_k] and 2 S v_{j+1}(a_{j+1}) =
// w[r_k] + g[l_{k+1}] (Robin, S the scalar p), so v_j(b_j) - v_{j+1}(a_{j+1}) =
// ((w - g)[l_{k+1}] - (w - g)[r_k]) / (2 S): the final residual's two blocks.
// ---------------------------------------------------------------------------
__global__ void k_jump_res(const double2* __restrict__ w, const double2* __restrict__ g, int N,
                           int nt, double scale, unsigned long long* out,
                           const InstInfo* __restrict__ inst, const int* __restrict__ if_inst,
                           int nif_total) {
    double m = 0.0;
    const long long tot = (long long)(inst ? nif_total : N - 1) * nt;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < tot;
         q += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(q / nt);
        const int n = (int)(q % nt);
        long long r, l;   // r_k and l_{k+1} at step n
        if (inst) {
            const InstInfo I = inst[if_inst[k]];
            if (n >= I.nt) continue;
            const int kk = k - I.if0;
            r = I.foff + (long long)(2 * kk) * I.nt + n;
            l = r + I.nt;
        } else {
            r = (long long)(2 * k) * nt + n;
            l = r + nt;
        }
        const double2 dl = csub(w[l], g[l]), dr = csub(w[r], g[r]);
        m = fmax(m, hypot(dl.x - dr.x, dl.y - dr.y));
    }
    atomicMax(out, (unsigned long long)__double_as_longlong(m * scale));
}

// The same for a convolution transmission operator (S_0^2 and the higher-order ones):
// the flux update's operator K = S-bar_j + S-bar_{j+1} acts on the mismatch trace dv
// (dv_0 = 0: both sides start from u0), K dv = (w - g)[l_{k+1}] - (w - g)[r_k], a lower-
// triangular Toeplitz system solved by forward substitution: one CTA per interface, dv
// in shared memory, the history sum of every step split over the threads (fixed-order
// reduction).  kout: the interface's kernel (the right end of subdomain j = k), or NULL
// with c2, beta for S_0^2 (K = 2 c2 beta).
__global__ void __launch_bounds__(256) k_jump_conv(
    const double2* __restrict__ w, const double2* __restrict__ g, int N, int nt,
    const double2* __restrict__ kout, int kstride, double2 c2, const double* __restrict__ beta,
    unsigned long long* out, const InstInfo* __restrict__ inst, const int* __restrict__ if_inst,
    int nif_total) {
    extern __shared__ double2 dv[];               // [nt + 1] trace, then kernel, right-hand side
    __shared__ double2 part[8];
    const int k = blockIdx.x;
    long long r0;
    int ntk = nt, sub;
    if (inst) {
        const InstInfo I = inst[if_inst[k]];
        const int kk = k - I.if0;
        ntk = I.nt;
        r0 = I.foff + (long long)(2 * kk) * I.nt;
        sub = I.sub0 + kk;
    } else {
        r0 = (long long)(2 * k) * nt;
        sub = k;
    }
    const long long l0 = r0 + ntk;
    const double2* K = kout ? kout + (size_t)(2 * sub + 1) * kstride : nullptr;
    auto kern = [&](int m) -> double2 {
        if (K) return K[m];
        return make_double2(2.0 * c2.x * beta[m], 2.0 * c2.y * beta[m]);
    };
    double2* kk = dv + (nt + 1);                  // the kernel and the right-hand sides, staged
    double2* rr = kk + (nt + 1);
    for (int q = threadIdx.x; q <= ntk; q += blockDim.x) {
        kk[q] = kern(q);
        if (q >= 1) {
            const double2 dl = csub(w[l0 + q - 1], g[l0 + q - 1]);
            const double2 dr = csub(w[r0 + q - 1], g[r0 + q - 1]);
            rr[q] = csub(dl, dr);
        }
    }
    const double2 k0 = kern(0);
    const double den = k0.x * k0.x + k0.y * k0.y;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    double m = 0.0;
    if (threadIdx.x == 0) dv[0] = make_double2(0.0, 0.0);
    __syncthreads();
    for (int n = 1; n <= ntk; ++n) {
        double2 acc = make_double2(0.0, 0.0);
        for (int s = 1 + threadIdx.x; s < n; s += blockDim.x) acc = cfma(kk[n - s], dv[s], acc);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
        }
        if (lane == 0) part[wi] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double2 tot = make_double2(0.0, 0.0);
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot = cadd(tot, part[q]);
            const double2 rhs = csub(rr[n], tot);
            const double2 v = make_double2((rhs.x * k0.x + rhs.y * k0.y) / den,
                                           (rhs.y * k0.x - rhs.x * k0.y) / den);
            dv[n] = v;
            m = fmax(m, hypot(v.x, v.y));
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

int swr_launch_jump_conv(const double2* w, const double2* g, int N, int nt, const double2* kout,
                         int kstride, double2 c2, const double* beta, double* out, cudaStream_t s,
                         const InstInfo* inst, const int* if_inst, int nif_total) {
    const int nif = inst ? nif_total : N - 1;
    cudaMemsetAsync(out, 0, sizeof(double), s);
    if (nif <= 0) return 0;
    const int smem = 3 * (nt + 1) * (int)sizeof(double2);
    if (smem > 200 * 1024) return -2;
    if (cudaFuncSetAttribute(k_jump_conv, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
        return -1;
    k_jump_conv<<<nif, 256, smem, s>>>(w, g, N, nt, kout, kstride, c2, beta,
                                       reinterpret_cast<unsigned long long*>(out), inst, if_inst,
                                       nif_total);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int swr_launch_jump_res(const double2* w, const double2* g, int N, int nt, double scale,
                        double* out, cudaStream_t s, const InstInfo* inst, const int* if_inst,
                        int nif_total) {
    cudaMemsetAsync(out, 0, sizeof(double), s);
    k_jump_res<<<64, 256, 0, s>>>(w, g, N, nt, scale, reinterpret_cast<unsigned long long*>(out),
                                  inst, if_inst, nif_total);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// u(T) by superposition (static V).  The subdomain march is linear and time
// invariant, so the response to a flux impulse at step n is the response to the
// impulse at step 1 delayed by n - 1 steps (the shift structure of Props. 3-4,
// here for the whole state, not only its end traces).  With Phi_l(k), Phi_r(k) the
// states after k steps of the build marches driven by l_{j,1} = 1 and r_{j,1} = 1,
// and U_d the final state of the march from u0 with zero fluxes,
//     u_j(T) = U_d + sum_{n=1}^{N} Phi_l(N - n + 1) l_j[n] + Phi_r(N - n + 1) r_j[n],
// a dense (n_j x N) complex matrix-vector product per subdomain and flux side.
// One thread per node, reading one row of states per step (coalesced); the
// fluxes of a tile of steps are staged in shared memory, in the order of k.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_superpose(
    const double2* __restrict__ urec, const long long* __restrict__ rec_base,
    const MarchSys* __restrict__ sys, const int* __restrict__ sub_n,
    const int* __restrict__ sub_goff, const int* __restrict__ sub_tc,
    const double2* __restrict__ g, double2* __restrict__ uT) {
    constexpr int KT = 256;
    __shared__ double2 fl[KT], fr[KT];
    const int j = blockIdx.y;
    const int n = sub_n[j];
    if (blockIdx.x * blockDim.x >= n) return;   // the whole CTA lies past this subdomain
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = li < n;
    const MarchSys sy = sys[j];
    const int nt = sy.nt;
    const double2* Pl = urec + rec_base[j] + li;
    const double2* Pr = Pl + (size_t)nt * n;
    const double2 zero = make_double2(0.0, 0.0);
    double2 a0 = in ? Pl[(size_t)2 * nt * n] : zero, a1 = zero, a2 = zero, a3 = zero;
    const bool hl = sy.in_l >= 0, hr = sy.in_r >= 0;
    for (int k0 = 0; k0 < nt; k0 += KT) {
        const int kc = min(KT, nt - k0);
        __syncthreads();
        for (int q = threadIdx.x; q < kc; q += blockDim.x) {
            const int gi = nt - 1 - (k0 + q);   // Phi(k) multiplies the flux of step nt - k + 1
            fl[q] = hl ? g[(size_t)sy.in_l + gi] : zero;
            fr[q] = hr ? g[(size_t)sy.in_r + gi] : zero;
        }
        __syncthreads();
        if (!in) continue;
        const double2* pl = Pl + (size_t)k0 * n;
        const double2* pr = Pr + (size_t)k0 * n;
        int q = 0;
        if (hl && hr) {
            for (; q + 1 < kc; q += 2) {   // each state is read once: streaming loads
                a0 = cfma(__ldcs(pl + (size_t)q * n), fl[q], a0);
                a1 = cfma(__ldcs(pr + (size_t)q * n), fr[q], a1);
                a2 = cfma(__ldcs(pl + (size_t)(q + 1) * n), fl[q + 1], a2);
                a3 = cfma(__ldcs(pr + (size_t)(q + 1) * n), fr[q + 1], a3);
            }
            for (; q < kc; ++q) {
                a0 = cfma(__ldcs(pl + (size_t)q * n), fl[q], a0);
                a1 = cfma(__ldcs(pr + (size_t)q * n), fr[q], a1);
            }
        } else if (hl || hr) {
            const double2* pp = hl ? pl : pr;
            const double2* ff = hl ? fl : fr;
            for (; q + 1 < kc; q += 2) {
                a0 = cfma(__ldcs(pp + (size_t)q * n), ff[q], a0);
                a2 = cfma(__ldcs(pp + (size_t)(q + 1) * n), ff[q + 1], a2);
            }
            if (q < kc) a0 = cfma(__ldcs(pp + (size_t)q * n), ff[q], a0);
        }
    }
    // the interface node belongs to the left subdomain
    if (in && !(li == 0 && (sub_tc[j] & 1)))
        uT[sub_goff[j] + li] = cadd(cadd(a0, a1), cadd(a2, a3));
}

int swr_launch_superpose(const double2* urec, const long long* rec_base, const MarchSys* sys,
                         int N, const int* sub_n, const int* sub_goff, const int* sub_tc,
                         int nmax, const double2* g, double2* uT, cudaStream_t s) {
    dim3 grid((nmax + 255) / 256, N);
    k_superpose<<<grid, 256, 0, s>>>(urec, rec_base, sys, sub_n, sub_goff, sub_tc, g, uT);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// Time-causal block forward substitution for (I - L) x = y.
// Every block of L is lower-triangular Toeplitz in time (Props. 3-4), so with
// x_n the values of all blocks at time n:
//     x_n - L[0] x_n = y_n + sum_{s<n} L[n-s] x_s.
// The lag-0 matrix L[0] couples the two fluxes of one interface (r_k, l_{k+1})
// strongly (2x2 block D_k, solved exactly) and neighbouring interfaces only
// through the corner entries of the subdomain inverse (X^{j,2}[0], X^{j,3}[0]),
// which are resolved by `sweeps` block-Jacobi sweeps (0: dropped).  The
// substitution runs as a wavefront over the interfaces (k_causal_wave below);
// k_lag0_setup forms the inverses of the 2x2 lag-0 blocks D_k once per build.
// ---------------------------------------------------------------------------
__global__ void k_lag0_setup(int N, int nt, const double2* __restrict__ cols,
                             double2* __restrict__ lag0, const InstInfo* __restrict__ inst,
                             const int* __restrict__ if_inst, int nif_total) {
    const int kg = blockIdx.x * blockDim.x + threadIdx.x;
    if (kg >= (inst ? nif_total : N - 1)) return;
    int k = kg;
    if (inst) {
        const InstInfo I = inst[if_inst[kg]];
        nt = I.nt;
        k = kg - I.if0;
        cols += I.coff;
    }
    const double2 a = cols[(size_t)(4 * (k + 1) + 0) * nt];   // X^{k+1,1}[0]: r_k <- l_{k+1}
    const double2 b = cols[(size_t)(4 * k + 3) * nt];         // X^{k,4}[0]:   l_{k+1} <- r_k
    // D = [[1, -a], [-b, 1]],  D^{-1} = [[1, a], [b, 1]] / (1 - a b)
    const double2 det = csub(make_double2(1.0, 0.0), cmul(a, b));
    const double2 r = crcp(det);
    lag0[kg * 4 + 0] = r;
    lag0[kg * 4 + 1] = cmul(a, r);
    lag0[kg * 4 + 2] = cmul(b, r);
    lag0[kg * 4 + 3] = r;
}

int swr_launch_lag0_setup(int N, int nt, const double2* cols, double2* lag0, cudaStream_t s,
                          const InstInfo* inst, const int* if_inst, int nif_total) {
    const int nif = inst ? nif_total : N - 1;
    k_lag0_setup<<<(nif + 127) / 128, 128, 0, s>>>(N, nt, cols, lag0, inst, if_inst, nif_total);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Wavefront form of the substitution: one CTA per interface k, all CTAs
// resident at once (cooperative launch).  At time step n, CTA k needs the
// values of its own two blocks and of the neighbouring blocks 2k-1 (interface
// k-1) and 2k+2 (interface k+1) at steps < n, so it waits only for its two
// neighbours' progress counters.  Progress is counted in sub-steps: step n,
// sweep sw is complete when progress >= n (S+1) + sw + 1, S = sweeps.
// Every wait is bounded; on timeout the CTA raises ST_TIMEOUT and a global abort
// flag, and all CTAs leave their loops.
#include <cuda/atomic>

namespace {
constexpr long long kWaitPolls = 4000000;    // about 1-2 s with the back-off below
}

// Test hook of the bounded waits (swr_test_wait_hook; defaults: the poll limit above,
// no interface withheld).  With d_wait_withhold = k >= 0, interface k's CTA never
// publishes its progress, so its neighbours' waits run out after d_wait_poll_limit
// polls and every CTA leaves through the abort flag with ST_TIMEOUT raised.
__device__ long long d_wait_poll_limit = kWaitPolls;
__device__ int d_wait_withhold = -1;

__device__ __forceinline__ int load_acquire(const int* p) {
    cuda::atomic_ref<const int, cuda::thread_scope_device> r(*p);
    return r.load(cuda::memory_order_acquire);
}
__device__ __forceinline__ void store_release(int* p, int v) {
    cuda::atomic_ref<int, cuda::thread_scope_device> r(*p);
    r.store(v, cuda::memory_order_release);
}

// Wait until the neighbours of interface k (global index; hl, hr: they exist in
// its instance) have reached `target`; returns false (after raising the abort
// flag) on timeout or when another CTA aborted.
// The polls: the first kSpinPolls re-read the counter at once (a hand-off usually
// lands within a few L2 round trips), later ones back off; the abort flag, a second
// L2 round trip, is looked at only every 32nd poll.
constexpr int kSpinPolls = 32;

__device__ __forceinline__ int load_relaxed(const int* p) {
    cuda::atomic_ref<const int, cuda::thread_scope_device> r(*p);
    return r.load(cuda::memory_order_relaxed);
}

// Relaxed polls (no cache maintenance per poll), one acquire once the value is there.
__device__ __forceinline__ bool poll_until(const int* cnt, int target, int* abortf, int* status,
                                           long long lim) {
    long long polls = 0;
    while (load_relaxed(cnt) < target) {
        ++polls;
        if ((polls & 31) == 0 && load_acquire(abortf) != 0) return false;
        if (polls > lim) {
            atomicOr(status, ST_TIMEOUT);
            store_release(abortf, 1);
            return false;
        }
        if (polls > kSpinPolls) __nanosleep(64);
    }
    (void)load_acquire(cnt);   // orders the reads that follow after the publisher's writes
    return true;
}

__device__ bool wait_neighbours(int k, bool hl, bool hr, int target, const int* progress,
                                int* abortf, int* status, long long lim) {
    if (hl && !poll_until(progress + (size_t)(k - 1) * kProgStride, target, abortf, status, lim))
        return false;
    if (hr && !poll_until(progress + (size_t)(k + 1) * kProgStride, target, abortf, status, lim))
        return false;
    return true;
}

// Wait until interface nb has reached `target` (one lane per interface waited on).
__device__ bool wait_one(int nb, int target, const int* progress, int* abortf, int* status,
                         long long lim) {
    return poll_until(progress + (size_t)nb * kProgStride, target, abortf, status, lim);
}

// Rows of the inverse of the lag-0 system.  With z_k = (r_k, l_{k+1}) the values
// of interface k at one time step, the same-step part of (I - L) is block
// tridiagonal, A0 = D + U + Lw:
//     D_k = [[1, -a_k], [-b_k, 1]],  a_k = X^{k+1,1}[0],  b_k = X^{k,4}[0],
//     U_k z_{k+1} = -cB_k r_{k+1} e_1,   cB_k = X^{k+1,2}[0],
//     Lw_k z_{k-1} = -cD_k l_k e_2,      cD_k = X^{k,3}[0].
// A0 = (I - F) D with F = -(U + Lw) D^{-1}, so row k of A0^{-1} is
// D_k^{-1} sum_m psi^(m), psi^(0) = e_k, psi^(m+1)_j = psi^(m)_{j-1} F_{j-1,j} +
// psi^(m)_{j+1} F_{j+1,j} = [cB_{j-1} psi_{j-1}[:,0] | cD_{j+1} psi_{j+1}[:,1]] D_j^{-1}.
// The couplings cB, cD are the corner entries of the subdomain inverses (small:
// psi^(m) decays like (|c| |D^{-1}|)^m); m runs to H + 4 over a window of H + 4
// interfaces each side, and the blocks |j - k| <= H are kept:
//     Gw[(k (2H+1) + j - k + H) 4 + {00, 01, 10, 11}] = (A0^{-1})_{k,j}.
// One warp per interface (below).
constexpr int kWinMaxH = 8;

// One warp per interface k, lane q for block j = k + q - W of the window (2W + 1 <= 25
// lanes): psi^(m) and the running sum live in the lanes' registers, the neighbours'
// blocks come by shuffles.
__global__ void __launch_bounds__(128) k_lag0_window(int N, int nt,
                                                     const double2* __restrict__ cols,
                                                     const double2* __restrict__ lag0,
                                                     double2* __restrict__ Gw, int H,
                                                     const InstInfo* __restrict__ inst,
                                                     const int* __restrict__ if_inst,
                                                     int nif_total) {
    const int kg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, q = threadIdx.x & 31;
    if (kg >= (inst ? nif_total : N - 1)) return;   // whole warps leave together
    int k = kg;
    if (inst) {
        const InstInfo I = inst[if_inst[kg]];
        N = I.N;
        nt = I.nt;
        k = kg - I.if0;
        cols += I.coff;
    }
    const int nI = N - 1, W = H + 4;
    const double2 zero = make_double2(0.0, 0.0);
    const int j = k + q - W;
    const bool in = (q <= 2 * W) && j >= 0 && j < nI;
    // this lane's constants: D_j^{-1}, cB_{j-1} (from the left block), cD_{j+1} (right)
    double2 Di0 = zero, Di1 = zero, Di2 = zero, Di3 = zero, cBl = zero, cDr = zero;
    if (in) {
        const double2* Di = lag0 + (size_t)(kg + q - W) * 4;
        Di0 = Di[0];
        Di1 = Di[1];
        Di2 = Di[2];
        Di3 = Di[3];
        if (q > 0 && j - 1 >= 0 && j <= N - 2) cBl = cols[(size_t)(4 * j + 1) * nt];
        if (q < 2 * W && j + 1 < nI && j + 1 >= 1) cDr = cols[(size_t)(4 * (j + 1) + 2) * nt];
    }
    double2 p0 = zero, p1 = zero, p2 = zero, p3 = zero;
    if (q == W) p0 = p3 = make_double2(1.0, 0.0);
    double2 s0 = p0, s1 = p1, s2 = p2, s3 = p3;
    auto shfl2 = [&](double2 v, int delta, bool up) {
        double2 r;
        r.x = up ? __shfl_up_sync(0xffffffffu, v.x, delta)
                 : __shfl_down_sync(0xffffffffu, v.x, delta);
        r.y = up ? __shfl_up_sync(0xffffffffu, v.y, delta)
                 : __shfl_down_sync(0xffffffffu, v.y, delta);
        return r;
    };
    for (int m = 1; m <= W; ++m) {
        // T = [cB_{j-1} psi_{j-1}[:,0] | cD_{j+1} psi_{j+1}[:,1]]
        const double2 l0 = shfl2(p0, 1, true), l2 = shfl2(p2, 1, true);
        const double2 r1 = shfl2(p1, 1, false), r3 = shfl2(p3, 1, false);
        const double2 t00 = cmul(cBl, l0), t10 = cmul(cBl, l2);
        const double2 t01 = cmul(cDr, r1), t11 = cmul(cDr, r3);
        double2 n0 = cfma(t00, Di0, cmul(t01, Di2));
        double2 n1 = cfma(t00, Di1, cmul(t01, Di3));
        double2 n2 = cfma(t10, Di0, cmul(t11, Di2));
        double2 n3 = cfma(t10, Di1, cmul(t11, Di3));
        if (!in) n0 = n1 = n2 = n3 = zero;
        p0 = n0;
        p1 = n1;
        p2 = n2;
        p3 = n3;
        s0 = cadd(s0, n0);
        s1 = cadd(s1, n1);
        s2 = cadd(s2, n2);
        s3 = cadd(s3, n3);
    }
    // row k of A0^{-1}: D_k^{-1} times the summed blocks, for |d| <= H
    const int d = q - W;
    auto from_w = [&](double2 v) {   // lane W's value: D_k^{-1}
        return make_double2(__shfl_sync(0xffffffffu, v.x, W), __shfl_sync(0xffffffffu, v.y, W));
    };
    const double2 K0 = from_w(Di0), K1 = from_w(Di1), K2 = from_w(Di2), K3 = from_w(Di3);
    if (d >= -H && d <= H) {
        double2* g = Gw + ((size_t)kg * (2 * H + 1) + d + H) * 4;
        g[0] = cfma(K0, s0, cmul(K1, s2));
        g[1] = cfma(K0, s1, cmul(K1, s3));
        g[2] = cfma(K2, s0, cmul(K3, s2));
        g[3] = cfma(K2, s1, cmul(K3, s3));
    }
}

int swr_launch_lag0_window(int N, int nt, const double2* cols, const double2* lag0, double2* Gw,
                           int H, cudaStream_t s, const InstInfo* inst, const int* if_inst,
                           int nif_total) {
    if (H < 1 || H > kWinMaxH) return -2;
    const int nif = inst ? nif_total : N - 1;
    k_lag0_window<<<(nif + 3) / 4, 128, 0, s>>>(N, nt, cols, lag0, Gw, H, inst, if_inst,
                                                nif_total);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Both forms below share the history sums.  Warp 0 solves and hands on; warps 1-4
// (one per source block) form the history sums of the lags beyond what warp 0 adds
// itself, a few steps ahead of warp 0 and without a per-step barrier: each runs as soon
// as its source's values are there and hands its sum over in a ring with one ready flag
// per warp (s_hdone), refilling a slot only after warp 0 has consumed it (s_hused).
//
// k_causal_flag: the values are the hand-off.  Every value that another CTA reads
// (x_n of an interface's two blocks and, in the window form, its partial right-hand
// side P_n) is written once, into an array preset to an "unset" bit pattern (all ones:
// a NaN that is never stored, a computed value with that pattern being stored as the
// canonical quiet NaN).  Readers poll the value itself with relaxed gpu-scope loads
// until it is set, so no flag, fence or acquire lies between one interface's step and
// its neighbours' next.  Each 8-byte word is single-copy atomic: a word that reads as
// set holds its final value.
// The same-step coupling of neighbouring interfaces is resolved exactly (to
// (|c| |D^{-1}|)^{H+1}) by the window form, x_n(k) = sum_d G_{k,k+d} R_n(k+d), with
// the rows of the lag-0 inverse (k_lag0_window) and R_n(i) the right-hand side of
// interface i at step n: P_n(i), i.e. y_n(i) and the lags >= 2, plus the lag-1 terms.
// H = 0 drops the coupling (G_{k,k} = D_k^{-1}, the lag-0 inverses themselves) and
// keeps P_n(k) in a register.
// k_causal_sweeps: the coupling resolved by `sweeps` >= 1 block-Jacobi sweeps, with
// progress counters (release / acquire) around the values exchanged per sweep.
namespace {
constexpr long long kLocalPolls = 1LL << 24;   // bound of a wait between warps of one CTA
constexpr long long kUnsetBits = -1LL;          // bit pattern of a value not yet written
constexpr int kLA = 3;                          // k_causal_flag: warp 0 adds lags 2..kLA
constexpr int kHB = 8;                          // history loads per lane in flight together
// inputs of one step of the window form: 4H + 4 blocks and 2(2H + 1) partial right-hand
// sides, at most kMaxInLane per lane (eight slots)
constexpr int kMaxIn = 4 * kWinMaxH + 4 + 2 * (2 * kWinMaxH + 1);
constexpr int kMaxInLane = (kMaxIn + 7) / 8;
constexpr int kCausalThreads = 192;             // warp 0, four history warps, one idle
}

// Flags between the warps of one CTA (shared memory, CTA-scope release/acquire).
__device__ __forceinline__ int cta_load_acquire(const int* p) {
    cuda::atomic_ref<const int, cuda::thread_scope_block> r(*p);
    return r.load(cuda::memory_order_acquire);
}
__device__ __forceinline__ void cta_store_release(int* p, int v) {
    cuda::atomic_ref<int, cuda::thread_scope_block> r(*p);
    r.store(v, cuda::memory_order_release);
}
// Wait until *flag >= target, or until *stop is set; false on stop or when the bound
// runs out.
__device__ __forceinline__ bool cta_wait_ge(const int* flag, int target, const int* stop) {
    long long polls = 0;
    while (cta_load_acquire(flag) < target) {
        if (cta_load_acquire(stop)) return false;
        if (++polls > kLocalPolls) return false;
        __nanosleep(32);
    }
    return true;
}

// Relaxed gpu-scope 16-byte load / store (two single-copy-atomic 8-byte words).
__device__ __forceinline__ double2 ld_relaxed2(const double2* p) {
    double a, b;
    asm volatile("ld.relaxed.gpu.global.v2.f64 {%0, %1}, [%2];" : "=d"(a), "=d"(b) : "l"(p));
    return make_double2(a, b);
}
__device__ __forceinline__ bool is_set(double2 v) {
    return __double_as_longlong(v.x) != kUnsetBits && __double_as_longlong(v.y) != kUnsetBits;
}
__device__ __forceinline__ double never_unset(double v) {
    return __double_as_longlong(v) == kUnsetBits ? __longlong_as_double(0x7ff8000000000000LL) : v;
}
__device__ __forceinline__ void st_relaxed2(double2* p, double2 v) {
    asm volatile("st.relaxed.gpu.global.v2.f64 [%0], {%1, %2};" ::"l"(p), "d"(never_unset(v.x)),
                 "d"(never_unset(v.y))
                 : "memory");
}
__device__ __forceinline__ void st_relaxed1(double* p, double v) {
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(never_unset(v)) : "memory");
}
// One more round of a bounded poll: false (after raising the abort flag on timeout)
// when the bound has run out or another CTA aborted.
__device__ __forceinline__ bool poll_tick(long long& polls, int* abortf, int* status,
                                          long long lim) {
    ++polls;
    if ((polls & 31) == 0 && load_relaxed(abortf) != 0) return false;
    if (polls > lim) {
        atomicOr(status, ST_TIMEOUT);
        store_release(abortf, 1);
        return false;
    }
    if (polls > kSpinPolls) __nanosleep(64);
    return true;
}

// Source e of interface i (N, nt, cols and x of its instance):
//  e=0: r_i     <- X^{i+1,1} l_{i+1} (block 2i+1)   e=1: r_i <- X^{i+1,2} r_{i+1} (block 2i+2)
//  e=2: l_{i+1} <- X^{i,4}   r_i     (block 2i)     e=3: l_{i+1} <- X^{i,3} l_i (block 2i-1)
// has: the source exists; cc: its Toeplitz column; xin: its block of x.
__device__ __forceinline__ void causal_source(int N, int nt, const double2* cols, double2* x,
                                              int i, int e, bool& has, const double2*& cc,
                                              double2*& xin) {
    int cslot = 0, inb = 0;
    has = true;
    if (e == 0) { cslot = 4 * (i + 1) + 0; inb = 2 * i + 1; }
    if (e == 1) { has = (i + 1 <= N - 2); cslot = 4 * (i + 1) + 1; inb = 2 * i + 2; }
    if (e == 2) { cslot = 4 * i + 3; inb = 2 * i; }
    if (e == 3) { has = (i >= 1); cslot = 4 * i + 2; inb = 2 * i - 1; }
    cc = has ? cols + (size_t)cslot * nt : nullptr;
    xin = has ? x + (size_t)inb * nt : nullptr;
}

// 64-point transform by one warp (radix-2 Stockham as fft_stockham, one butterfly per
// lane and stage), a and b 64-entry shared buffers; returns the buffer holding the result.
// W: W^k = exp(-2 pi i k / 64), k < 32 (conjugated for the inverse; unscaled).
__device__ __forceinline__ double2* warp_fft64(double2* a, double2* b, const double2* W,
                                               bool inverse, int lane) {
#pragma unroll
    for (int st = 0; st < 6; ++st) {
        const int m = 1 << st, l = 32 >> st;
        const int j = lane >> st, kk = lane & (m - 1);
        double2 w = W[j * m];
        if (inverse) w.y = -w.y;
        const double2 c0 = a[kk + j * m], c1 = a[kk + j * m + l * m];
        b[kk + 2 * j * m] = cadd(c0, c1);
        b[kk + 2 * j * m + m] = cmul(w, csub(c0, c1));
        __syncwarp();
        double2* tt = a;
        a = b;
        b = tt;
    }
    return a;
}

// One CTA of kCausalThreads per interface: warp 0 solves, warps 1, 2, 3 and 5 form the
// history sums of sources 0..3 (warp 4, which would share warp 0's sub-partition, leaves at
// once).  cols_smem: the dynamic shared memory holds the four Toeplitz columns (4 nt).
template <bool FLAG>
__global__ void __launch_bounds__(kCausalThreads, 4) k_causal_wave(
    int N, int nt, int sweeps, const double2* __restrict__ cols, const double2* __restrict__ lag0,
    const double2* __restrict__ y, double2* x, double2* xsw, double2* P, int* progress,
    int* abortf, int* status, const InstInfo* __restrict__ inst, const int* __restrict__ if_inst,
    int k0, int nif_all, const double2* __restrict__ Gw, int H, int cols_smem,
    const double2* __restrict__ hspec, double2* xspec, int nbt) {
    // lookahead: warp 0 adds the lags 2..LA itself, the history warps the lags > LA
    constexpr int LA = FLAG ? kLA : 2;
    extern __shared__ double2 s_cols[];  // [4][nt] when cols_smem
    __shared__ double2 hp[LA + 1][4];   // lags > LA of step t (slot t % (LA + 1)), per source
    __shared__ int s_xown;              // x_0 .. x_{s_xown - 1} of this interface are written
    __shared__ int s_hused;             // warp 0 has consumed the history sums of steps <= s_hused
    __shared__ int s_hdone[4];          // history warp e has filled the slots of steps <= s_hdone[e]
    __shared__ int s_stop;              // warp 0 left its loop (done, timeout or abort)
    // warp 0 of the value-polling form: its inputs (type, offset, per-lane weights) and
    // the step's recent values
    __shared__ int s_itype[FLAG ? kMaxIn : 1];
    __shared__ long long s_ioff[FLAG ? kMaxIn : 1];
    __shared__ double2 s_wq[FLAG ? kMaxIn : 1][4];
    __shared__ double2 s_xo[2], s_P[2], s_nb[2], s_l3[4], s_c23[2][4];
    __shared__ int s_nbin[2];
    // FFT form of the history: per history warp two blocks of source values and the
    // transform's ping-pong buffers; the 32 twiddles of the 64-point transform
    __shared__ double2 s_hx[FLAG ? 4 : 1][64];
    __shared__ double2 s_hf[FLAG ? 4 : 1][128];
    __shared__ double2 s_w64[32];
    // global interface kg (sweep values, progress, lag-0 blocks); local k within its
    // instance (blocks, columns)
    const int kg = k0 + blockIdx.x;
    const long long lim = d_wait_poll_limit;
    const bool publish = (kg != d_wait_withhold);     // false only under the test hook
    int k = kg;
    if (inst) {
        const InstInfo I = inst[if_inst[kg]];
        N = I.N;
        nt = I.nt;
        k = kg - I.if0;
        cols += I.coff;
        y += I.foff;
        x += I.foff;
        if (P) P += I.foff;
    }
    const bool has_l = (k >= 1), has_r = (k + 1 <= N - 2);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double2 zero = make_double2(0.0, 0.0);
    if (threadIdx.x < 4 * (LA + 1)) hp[threadIdx.x >> 2][threadIdx.x & 3] = zero;
    if (FLAG && hspec && threadIdx.x < 32) {   // W^k = exp(-2 pi i k / 64)
        double sn, cs;
        sincospi(-(double)threadIdx.x / 32.0, &sn, &cs);
        s_w64[threadIdx.x] = make_double2(cs, sn);
    }
    if (threadIdx.x < 4) s_hdone[threadIdx.x] = LA;   // steps 0..LA have no lag > LA
    if (threadIdx.x == 0) {
        s_xown = 0;
        s_hused = 0;
        s_stop = 0;
    }
    __syncthreads();

    // ---- history warps: the lags > LA of step m + LA from the values s <= m - 1 -------
    // Sources 0 and 2 are this interface's own blocks (written by warp 0: wait on
    // s_xown); sources 1 and 3 are the neighbours'.  A slot is refilled only after warp 0
    // has consumed the step it held (m - 1).
    if (w == 4) return;
    if (w >= 1) {
        const int e = (w == 5) ? 3 : w - 1;
        bool has = false;
        const double2* cc = nullptr;
        double2* xin = nullptr;
        causal_source(N, nt, cols, x, k, e, has, cc, xin);
        if (cols_smem && has) {   // this source's column into shared memory
            for (int j = lane; j < nt; j += 32) s_cols[(size_t)e * nt + j] = __ldg(cc + j);
            __syncwarp();
            cc = s_cols + (size_t)e * nt;
        }
        const bool own = (e == 0 || e == 2);
        const int nb = (e == 1) ? kg + 1 : kg - 1;
        if constexpr (FLAG) {
            if (hspec) {
                // ---- FFT form of the history (single instance, nt >= 64) --------------
                // Lags > LA of step t, t in output block K = t / 32 (tau = t mod 32), split
                // at the blocks of 32 input steps:
                //   near: input blocks K-1 and K, accumulated as each value x_s arrives
                //         (lane tau adds c[t - s] x_s for its step t of block J = s / 32 and
                //         of block J + 1; two accumulators, one per block parity);
                //   far:  input blocks J <= K-2, sum_J IFFT(C_{K-J} . X_J)[32 + tau] with
                //         X_J the 64-point transform of block J zero-padded and C_d that of
                //         the column's segment c[(d-1) 32 .. (d+1) 32) (precomputed, / 64);
                //         formed while block K-1 arrives: the transform of block K-2 at its
                //         first value, one product term per value, the inverse at the 28th.
                // The source's values are read once, as they arrive (kept per block in
                // shared memory for the transform).
                double2* sx = s_hx[e];                  // [2][32]: blocks of parity 0, 1
                double2* fa = s_hf[e];                  // [2][64]: transform ping-pong
                double2* xs = xspec + (size_t)(4 * kg + e) * nbt * 64;
                const double2* cs = hspec + (size_t)(4 * kg + e) * nbt * 64;
                // accumulators and far parts of the output blocks of parity 0 and 1
                double2 A0 = zero, A1 = zero, F0 = zero, F1 = zero, Fa0 = zero, Fa1 = zero;
                for (int m = 1; m + LA < nt; ++m) {
                    bool ok = __all_sync(0xffffffffu, cta_wait_ge(&s_hused, m - 1, &s_stop));
                    if (!ok) break;
                    const int s = m - 1, J = s >> 5, sg = s & 31, t = m + LA;
                    double2 v = zero;
                    if (has) {
                        if (own) {
                            ok = __all_sync(0xffffffffu, cta_wait_ge(&s_xown, m, &s_stop));
                            if (ok) v = __ldcg(xin + s);
                        } else {
                            long long polls = 0;
                            bool o = true;
                            if (lane == 0)
                                while (!is_set(v = ld_relaxed2(xin + s)))
                                    if (!poll_tick(polls, abortf, status, lim)) {
                                        o = false;
                                        break;
                                    }
                            ok = __shfl_sync(0xffffffffu, o, 0);
                            v.x = __shfl_sync(0xffffffffu, v.x, 0);
                            v.y = __shfl_sync(0xffffffffu, v.y, 0);
                        }
                        if (!ok) break;
                    }
                    if (lane == 0) sx[(J & 1) * 32 + sg] = v;
                    if (sg == 0) {
                        if (J & 1) A0 = zero;
                        else A1 = zero;
                    }
                    // near: this value's terms for the steps of blocks J and J + 1
                    if (has) {
                        const int lc = lane - sg, ln = 32 + lane - sg;
                        const double2 tc = (lc > LA) ? cc[lc] : zero;
                        const double2 tn = (ln > LA) ? cc[ln] : zero;
                        // block J's accumulator gets tc, block J + 1's gets tn
                        const bool odd = J & 1;
                        A0 = cfma(odd ? tn : tc, v, A0);
                        A1 = cfma(odd ? tc : tn, v, A1);
                    }
                    // far part of block Kf = J + 1, formed during block J
                    const int Kf = J + 1;
                    if (has && Kf >= 2 && 32 * Kf < nt) {
                        if (sg == 0) {
                            __syncwarp();
                            fa[lane] = sx[((J - 1) & 1) * 32 + lane];
                            fa[32 + lane] = zero;
                            __syncwarp();
                            const double2* r = warp_fft64(fa, fa + 64, s_w64, false, lane);
                            const double2 x0 = r[lane], x1 = r[32 + lane];
                            xs[(size_t)(J - 1) * 64 + lane] = x0;
                            xs[(size_t)(J - 1) * 64 + 32 + lane] = x1;
                            Fa0 = Fa1 = zero;
                            __syncwarp();
                        }
                        // terms q = 0 .. J-1 (X_q with C_{Kf-q}), spread over sg = 1 .. 26
                        if (sg >= 1 && sg <= 26) {
                            const int per = (J + 25) / 26;
                            const int q0 = (sg - 1) * per, q1 = min(J, sg * per);
                            for (int q = q0; q < q1; ++q) {
                                const double2* xq = xs + (size_t)q * 64;
                                const double2* cq = cs + (size_t)(Kf - q) * 64;
                                Fa0 = cfma(__ldg(cq + lane), xq[lane], Fa0);
                                Fa1 = cfma(__ldg(cq + 32 + lane), xq[32 + lane], Fa1);
                            }
                        }
                        if (sg == 27) {
                            fa[lane] = Fa0;
                            fa[32 + lane] = Fa1;
                            __syncwarp();
                            const double2* r = warp_fft64(fa, fa + 64, s_w64, true, lane);
                            if (Kf & 1) F1 = r[32 + lane];
                            else F0 = r[32 + lane];
                            __syncwarp();
                        }
                    } else if (sg == 27) {
                        if (Kf & 1) F1 = zero;
                        else F0 = zero;
                    }
                    // this step's sum: lane t mod 32
                    if (lane == (t & 31)) {
                        const int K = t >> 5;
                        hp[t % (LA + 1)][e] = (K & 1) ? cadd(A1, F1) : cadd(A0, F0);
                        cta_store_release(&s_hdone[e], t);
                    }
                }
                return;
            }
        }
        for (int m = 1; m + LA < nt; ++m) {
            bool ok = __all_sync(0xffffffffu, cta_wait_ge(&s_hused, m - 1, &s_stop));
            if (!ok) break;
            double2 a0 = zero, a1 = zero;
            if (has) {
                if (own) {
                    ok = __all_sync(0xffffffffu, cta_wait_ge(&s_xown, m, &s_stop));
                } else if (!FLAG) {
                    // x_{<= m-1} of the neighbour: progress >= m (sweeps + 1)
                    bool o = true;
                    if (lane == 0) o = wait_one(nb, m * (sweeps + 1), progress, abortf, status, lim);
                    ok = __shfl_sync(0xffffffffu, o, 0);
                } else {
                    // the neighbour's newest value first (its values are read as written)
                    long long polls = 0;
                    bool o = true;
                    if (lane == 0)
                        while (!is_set(ld_relaxed2(xin + m - 1)))
                            if (!poll_tick(polls, abortf, status, lim)) {
                                o = false;
                                break;
                            }
                    ok = __shfl_sync(0xffffffffu, o, 0);
                }
                if (!ok) break;
                if (own || !FLAG) {
                    for (int base = 0; base < m; base += 32 * kHB) {
                        double2 u[kHB];
#pragma unroll
                        for (int b = 0; b < kHB; ++b) {
                            const int s = base + 32 * b + lane;
                            u[b] = (s < m) ? __ldcg(xin + s) : zero;
                        }
#pragma unroll
                        for (int b = 0; b < kHB; ++b) {
                            const int s = base + 32 * b + lane;
                            if (s < m) {
                                if (b & 1) a1 = cfma(cc[m + LA - s], u[b], a1);
                                else a0 = cfma(cc[m + LA - s], u[b], a0);
                            }
                        }
                    }
                } else {
                    // the whole sum with every value checked, repeated until all were set;
                    // kHB loads per lane issued together (one L2 round trip per 32 kHB values)
                    long long polls = 0;
                    while (true) {
                        bool all = true;
                        a0 = a1 = zero;
                        for (int base = 0; base < m; base += 32 * kHB) {
                            double2 u[kHB];
#pragma unroll
                            for (int b = 0; b < kHB; ++b) {
                                const int s = base + 32 * b + lane;
                                u[b] = (s < m) ? ld_relaxed2(xin + s) : zero;
                            }
#pragma unroll
                            for (int b = 0; b < kHB; ++b) {
                                const int s = base + 32 * b + lane;
                                if (s < m) {
                                    all = all && is_set(u[b]);
                                    if (b & 1) a1 = cfma(cc[m + LA - s], u[b], a1);
                                    else a0 = cfma(cc[m + LA - s], u[b], a0);
                                }
                            }
                        }
                        if (__all_sync(0xffffffffu, all)) break;
                        bool o = true;
                        if (lane == 0) o = poll_tick(polls, abortf, status, lim);
                        if (!__shfl_sync(0xffffffffu, o, 0)) {
                            ok = false;
                            break;
                        }
                    }
                    if (!ok) break;
                }
            }
            const double2 acc = warp_sum(cadd(a0, a1));
            if (lane == 0) {
                hp[(m + LA) % (LA + 1)][e] = acc;
                cta_store_release(&s_hdone[e], m + LA);
            }
        }
        return;
    }

    // ---- warp 0 ----------------------------------------------------------------------
    // Lane 0 forms the history of step t for this interface: the warps' lags > LA plus
    // the lags lo..LA, s_cl[j - 2][e] x_{t-j} of source e, with x_{t-j} = s_xl[j - lo][e]
    // (the caller keeps s_xl[0] = x_{n-2} at the top of step n).  Both tables in shared
    // memory, filled by lane 0.
    __shared__ double2 s_cl[LA - 1][4];
    __shared__ double2 s_xl[LA - 1][4];
    double2* xsrc[4] = {nullptr, nullptr, nullptr, nullptr};
    if (lane == 0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            bool has;
            const double2* cc;
            causal_source(N, nt, cols, x, k, e, has, cc, xsrc[e]);
            for (int j = 2; j <= LA; ++j)
                s_cl[j - 2][e] = (has && nt > j) ? cc[j] : zero;
            for (int j = 0; j < LA - 1; ++j) s_xl[j][e] = zero;
        }
    }
    __syncwarp();
    auto hist = [&](int t, int lo, double2 (&h)[4]) -> bool {
        bool ok = true;
#pragma unroll
        for (int e = 0; e < 4; ++e) ok = ok && cta_wait_ge(&s_hdone[e], t, &s_stop);
        if (!ok) return false;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            h[e] = hp[t % (LA + 1)][e];
#pragma unroll
            for (int j = 2; j <= LA; ++j)
                if (j >= lo && t >= j) h[e] = cfma(s_cl[j - 2][e], s_xl[j - lo][e], h[e]);
        }
        cta_store_release(&s_hused, t);
        return true;
    };
    // lane 0: a new x_{n-1} of the sources enters the recent values
    auto push_recent = [&](const double2 (&v)[4]) {
#pragma unroll
        for (int j = LA - 2; j >= 1; --j)
#pragma unroll
            for (int e = 0; e < 4; ++e) s_xl[j][e] = s_xl[j - 1][e];
#pragma unroll
        for (int e = 0; e < 4; ++e) s_xl[0][e] = v[e];
    };
    auto fail_local = [&]() {   // a wait between this CTA's warps ran out: leave everywhere
        atomicOr(status, ST_TIMEOUT);
        store_release(abortf, 1);
    };

    if constexpr (FLAG) {
        // ---- the values are the hand-off (window H >= 0) --------------------------------
        // x_n(k), two blocks (outputs o = 0: block 2k, o = 1: block 2k+1), is linear in the
        // inputs of step n: x_{n-1} of the window's blocks b = 2(k-H)-1 .. 2(k+H)+2 and
        // the partial right-hand sides P_n(k+d)[row], |d| <= H:
        //   x_n(k)[o] = sum_inputs w_o u,   w_o = G_{k,k+d}[o][row] for P_n(k+d)[row], and
        //   for a block b the sum of G_{k,i}[o][row] c1 over the sources (i, row, e) that
        //   read b, c1 their lag-1 coefficient.
        // On this part every FP64 warp instruction costs the same whatever the number of
        // active lanes, so the arithmetic is spread over the lanes: q = lane >> 3 picks a
        // real output (o = q >> 1, real or imaginary part q & 1), s = lane & 7 a slot that
        // takes the inputs s, s + 8, ...; a three-level butterfly over the slots sums.
        // P_{n+1}(k) (y_{n+1}, the history warps' lags > LA, lags 2..3) is formed the same
        // way, row = q >> 1, one term per slot.
        const int q = lane >> 3, sl = lane & 7, o = q >> 1, part = q & 1;
        const int ilo = max(k - H, 0), ihi = min(k + H, N - 2);
        const int blo = max(2 * (k - H) - 1, 0), bhi = min(2 * (k + H) + 2, 2 * N - 3);
        const int nxin = bhi - blo + 1, nin = nxin + 2 * (ihi - ilo + 1);
        auto G = [&](int i, int oo, int row) {   // (A0^{-1})_{k,i}[oo][row]
            return Gw[((size_t)kg * (2 * H + 1) + (i - k) + H) * 4 + oo * 2 + row];
        };
        auto c1of = [&](int i, int e) {          // lag-1 coefficient of source e of i
            bool has;
            const double2* cc;
            double2* xi;
            causal_source(N, nt, cols, x, i, e, has, cc, xi);
            return (has && nt > 1) ? cc[1] : zero;
        };
        for (int j = lane; j < nin; j += 32) {
            double2 w0 = zero, w1 = zero;
            int type;
            long long off;
            if (j < nxin) {
                const int b = blo + j;
                type = (b == 2 * k) ? 2 : (b == 2 * k + 1) ? 3 : 0;
                off = (long long)b * nt;
                // readers of block b: (i, row, e) = (b/2, 1, 2), (b/2 - 1, 0, 1) for even b;
                // ((b-1)/2, 0, 0), ((b-1)/2 + 1, 1, 3) for odd b
                const int i1 = (b & 1) ? (b - 1) / 2 : b / 2;
                const int i2 = (b & 1) ? i1 + 1 : i1 - 1;
                const int r1 = (b & 1) ? 0 : 1, r2 = 1 - r1;
                const int e1 = (b & 1) ? 0 : 2, e2 = (b & 1) ? 3 : 1;
                if (i1 >= ilo && i1 <= ihi) {
                    const double2 c = c1of(i1, e1);
                    w0 = cfma(G(i1, 0, r1), c, w0);
                    w1 = cfma(G(i1, 1, r1), c, w1);
                }
                if (i2 >= ilo && i2 <= ihi) {
                    const double2 c = c1of(i2, e2);
                    w0 = cfma(G(i2, 0, r2), c, w0);
                    w1 = cfma(G(i2, 1, r2), c, w1);
                }
            } else {
                const int i = ilo + (j - nxin) / 2, row = (j - nxin) & 1;
                type = (i == k) ? 4 + row : 1;
                off = (long long)(2 * i + row) * nt;
                w0 = G(i, 0, row);
                w1 = G(i, 1, row);
            }
            s_itype[j] = type;
            s_ioff[j] = off;
            // lane q's share: a1 b1 + a2 b2 with (b1, b2) = (re, im) of the input for a
            // real part, (im, re) for an imaginary part
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const double2 ww = (qq >> 1) ? w1 : w0;
                s_wq[j][qq] = make_double2(ww.x, (qq & 1) ? ww.y : -ww.y);
            }
        }
        if (lane < 4) {
            bool has;
            const double2* cc;
            double2* xi;
            causal_source(N, nt, cols, x, k, lane, has, cc, xi);
            s_c23[0][lane] = (has && nt > 2) ? cc[2] : zero;
            s_c23[1][lane] = (has && nt > 3) ? cc[3] : zero;
            s_l3[lane] = zero;
        }
        if (lane < 2) {
            s_xo[lane] = zero;
            s_nb[lane] = zero;
            const double2 y0 = y[(size_t)(2 * k + lane) * nt];   // P_0(k) = y_0(k)
            s_P[lane] = y0;
            if (H > 0 && publish) st_relaxed2(P + (size_t)(2 * k + lane) * nt, y0);
        }
        if (lane == 0) {
            // inputs that are the neighbours' source blocks (lag 2 of P_{n+1})
            s_nbin[0] = has_r ? 2 * k + 2 - blo : -1;
            s_nbin[1] = has_l ? 2 * k - 1 - blo : -1;
        }
        __syncwarp();
        // lanes sl == 0: y_{n+1}(k)[row] of their P_{n+1} part, one step ahead
        double yv = 0.0;
        if (sl == 0 && nt > 1) {
            const double2 yy = y[(size_t)(2 * k + o) * nt + 1];
            yv = part ? yy.y : yy.x;
        }
        for (int n = 0; n < nt; ++n) {
            // ---- this lane's inputs: shared ones now, global ones polled until set
            double2 u[kMaxInLane];
            unsigned need = 0;
#pragma unroll
            for (int t = 0; t < kMaxInLane; ++t) {
                const int j = sl + 8 * t;
                u[t] = zero;
                if (j < nin) {
                    const int ty = s_itype[j];
                    if (ty == 0) {
                        if (n >= 1) need |= 1u << t;
                    } else if (ty == 1) {
                        need |= 1u << t;
                    } else if (ty <= 3) {
                        u[t] = s_xo[ty - 2];      // x_{n-1} of this interface (0 at n = 0)
                    } else {
                        u[t] = s_P[ty - 4];
                    }
                }
            }
            bool ok = true;
            long long polls = 0;
            while (need) {
#pragma unroll
                for (int t = 0; t < kMaxInLane; ++t) {
                    if (need & (1u << t)) {
                        const int j = sl + 8 * t;
                        const double2* p = (s_itype[j] == 0) ? x + s_ioff[j] + n - 1
                                                              : P + s_ioff[j] + n;
                        u[t] = ld_relaxed2(p);
                        if (is_set(u[t])) need &= ~(1u << t);
                    }
                }
                if (need && !poll_tick(polls, abortf, status, lim)) {
                    ok = false;
                    break;
                }
            }
            if (!__all_sync(0xffffffffu, ok)) break;
            // ---- x_n(k)
            double acc = 0.0;
#pragma unroll
            for (int t = 0; t < kMaxInLane; ++t) {
                const int j = sl + 8 * t;
                if (j < nin) {
                    const double2 a = s_wq[j][q];
                    acc = fma(a.x, part ? u[t].y : u[t].x, fma(a.y, part ? u[t].x : u[t].y, acc));
                }
            }
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            acc += __shfl_xor_sync(0xffffffffu, acc, 4);
            if (sl == 0 && publish)
                st_relaxed1(reinterpret_cast<double*>(x + (size_t)(2 * k + o) * nt + n) + part,
                            acc);
            // x_{n-1} of the neighbours' source blocks, for the lag-2 terms
            if (q == 0 && n >= 1) {
#pragma unroll
                for (int t = 0; t < kMaxInLane; ++t) {
                    const int j = sl + 8 * t;
                    if (j == s_nbin[0]) s_nb[0] = u[t];
                    if (j == s_nbin[1]) s_nb[1] = u[t];
                }
            }
            __syncwarp();
            // ---- P_{n+1}(k): row o (sources ea, eb), one term per slot
            double accp = 0.0;
            if (n + 1 < nt) {
                const int ea = o ? 2 : 0, eb = o ? 3 : 1;
                if (sl == 0) {
                    accp = yv;
                } else if (sl <= 2) {
                    const int e = (sl == 1) ? ea : eb;
                    if (cta_wait_ge(&s_hdone[e], n + 1, &s_stop)) {
                        const double2 h = hp[(n + 1) % (LA + 1)][e];
                        accp = part ? h.y : h.x;
                    } else {
                        ok = false;
                    }
                } else if (sl <= 6) {
                    const int e = (sl & 1) ? ea : eb;       // sl 3, 5: ea; 4, 6: eb
                    const int lag = (sl <= 4) ? 0 : 1;      // lag 2 or lag 3
                    const double2 c = s_c23[lag][e];
                    // x_{n-1} (lag 2) or x_{n-2} (lag 3) of source e
                    const double2 v = lag ? s_l3[e]
                                          : (e == 0) ? s_xo[1] : (e == 2) ? s_xo[0]
                                          : (e == 1) ? s_nb[0] : s_nb[1];
                    accp = fma(c.x, part ? v.y : v.x, (part ? c.y : -c.y) * (part ? v.x : v.y));
                }
                accp += __shfl_xor_sync(0xffffffffu, accp, 1);
                accp += __shfl_xor_sync(0xffffffffu, accp, 2);
                accp += __shfl_xor_sync(0xffffffffu, accp, 4);
                if (sl == 0 && H > 0 && publish)
                    st_relaxed1(reinterpret_cast<double*>(P + (size_t)(2 * k + o) * nt + n + 1) +
                                    part,
                                accp);
            }
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) fail_local();
                break;
            }
            // ---- hand the step over: recent values, own x_n and P_{n+1}, the CTA flags
            if (lane == 0 && n >= 1) {
                s_l3[0] = s_xo[1];
                s_l3[2] = s_xo[0];
                s_l3[1] = s_nb[0];
                s_l3[3] = s_nb[1];
            }
            __syncwarp();
            if (sl == 0) {
                double* xo = reinterpret_cast<double*>(&s_xo[o]);
                double* po = reinterpret_cast<double*>(&s_P[o]);
                xo[part] = acc;
                po[part] = accp;
                if (n + 2 < nt) {
                    const double2 yy = y[(size_t)(2 * k + o) * nt + n + 2];
                    yv = part ? yy.y : yy.x;
                }
            }
            __syncwarp();
            if (lane == 0) {
                cta_store_release(&s_hused, n + 1);
                cta_store_release(&s_xown, n + 1);
            }
        }
    } else {
        // ---- sweep form (sweeps >= 1) ----------------------------------------------
        // Progress is counted in sub-steps: step n, sweep sw is complete when
        // progress >= n (S+1) + sw + 1, S = sweeps; the step's values x_n are ordered
        // by progress = (n+1)(S+1).
        const int S1 = sweeps + 1;
        double2 D00 = zero, D01 = zero, D10 = zero, D11 = zero, cB0 = zero, cD0 = zero;
        double2 c1[4] = {zero, zero, zero, zero};
        bool hs[4] = {false, false, false, false};
        const bool solver = (lane == 0);
        if (solver) {
            D00 = lag0[kg * 4 + 0];
            D01 = lag0[kg * 4 + 1];
            D10 = lag0[kg * 4 + 2];
            D11 = lag0[kg * 4 + 3];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const double2* cc;
                causal_source(N, nt, cols, x, k, e, hs[e], cc, xsrc[e]);
                if (hs[e] && nt > 1) c1[e] = cc[1];
                if (hs[e] && e == 1) cB0 = cc[0];
                if (hs[e] && e == 3) cD0 = cc[0];
            }
        }
        for (int n = 0; n < nt; ++n) {
            // lanes 0 and 1 wait for the left and right neighbours' values < n
            bool ok = true;
            if (lane < 2 && (lane == 0 ? has_l : has_r))
                ok = wait_one(kg + (lane == 0 ? -1 : 1), n * S1, progress, abortf, status, lim);
            ok = __all_sync(0xffffffffu, ok);                  // values < n visible
            if (!ok) break;
            int go = 1;
            if (solver) {
                // x_{n-1} of the sources (the lag-1 terms; lag 2 at the next step)
                double2 x1[4] = {zero, zero, zero, zero};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (n >= 1 && hs[e]) x1[e] = __ldcg(xsrc[e] + n - 1);
                double2 h[4];
                if (!hist(n, 2, h)) {
                    go = 0;
                    fail_local();
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) h[e] = cfma(c1[e], x1[e], h[e]);
                    push_recent(x1);
                    const double2 r1 = cadd(y[(size_t)(2 * k) * nt + n], cadd(h[0], h[1]));
                    const double2 r2 = cadd(y[(size_t)(2 * k + 1) * nt + n], cadd(h[2], h[3]));
                    double2 z1 = cfma(D01, r2, cmul(D00, r1));
                    double2 z2 = cfma(D11, r2, cmul(D10, r1));
                    for (int sw = 1; sw <= sweeps; ++sw) {
                        // publish sweep sw-1 of this step, then use the neighbours' sweep sw-1
                        double2* out = xsw + (size_t)((sw - 1) & 1) * 2 * nif_all;
                        out[2 * kg] = z1;
                        out[2 * kg + 1] = z2;
                        if (publish) store_release(progress + (size_t)kg * kProgStride, n * S1 + sw);
                        if (!wait_neighbours(kg, has_l, has_r, n * S1 + sw, progress, abortf,
                                             status, lim)) {
                            go = 0;
                            break;
                        }
                        const double2 xr = has_r ? out[2 * (kg + 1)] : zero;       // r_{k+1}
                        const double2 xlk = has_l ? out[2 * (kg - 1) + 1] : zero;  // l_k
                        const double2 e1 = cfma(cB0, xr, r1), e2 = cfma(cD0, xlk, r2);
                        z1 = cfma(D01, e2, cmul(D00, e1));
                        z2 = cfma(D11, e2, cmul(D10, e1));
                    }
                    if (go) {
                        x[(size_t)(2 * k) * nt + n] = z1;
                        x[(size_t)(2 * k + 1) * nt + n] = z2;
                        cta_store_release(&s_xown, n + 1);
                        if (publish) store_release(progress + (size_t)kg * kProgStride, (n + 1) * S1);   // orders x
                    }
                }
            }
            go = __shfl_sync(0xffffffffu, go, 0);
            if (!go) break;
        }
    }
    if (lane == 0) cta_store_release(&s_stop, 1);   // releases history warps still waiting
}

// Spectra of the column segments for the FFT form of the history sums: for interface k,
// source e (pair 4k + e) and d = 2 .. nbt-1, the 64-point transform of
// c[(d-1) 32 .. (d+1) 32) (zero beyond nt), scaled by 1/64, at
// hspec[((4k + e) nbt + d) 64 ..].  One CTA of 32 threads per pair.
__global__ void __launch_bounds__(32) k_hist_spectra(int N, int nt, int nbt,
                                                     const double2* __restrict__ cols,
                                                     double2* __restrict__ hspec) {
    __shared__ double2 a[128];
    __shared__ double2 w64[32];
    const int pair = blockIdx.x, kg = pair >> 2, e = pair & 3, lane = threadIdx.x;
    double sn, cs;
    sincospi(-(double)lane / 32.0, &sn, &cs);
    w64[lane] = make_double2(cs, sn);
    bool has;
    const double2* cc;
    double2* xin;
    causal_source(N, nt, cols, nullptr, kg, e, has, cc, xin);
    const double2 zero = make_double2(0.0, 0.0);
    double2* out = hspec + (size_t)pair * nbt * 64;
    for (int d = 0; d < nbt; ++d) {
        if (d < 2 || !has) {
            out[(size_t)d * 64 + lane] = zero;
            out[(size_t)d * 64 + 32 + lane] = zero;
            continue;
        }
        const int i0 = (d - 1) * 32 + lane, i1 = i0 + 32;
        __syncwarp();
        a[lane] = (i0 < nt) ? cc[i0] : zero;
        a[32 + lane] = (i1 < nt) ? cc[i1] : zero;
        __syncwarp();
        const double2* r = warp_fft64(a, a + 64, w64, false, lane);
        const double sc = 1.0 / 64.0;
        out[(size_t)d * 64 + lane] = make_double2(r[lane].x * sc, r[lane].y * sc);
        out[(size_t)d * 64 + 32 + lane] = make_double2(r[32 + lane].x * sc, r[32 + lane].y * sc);
    }
}

int swr_hist_blocks(int nt) { return (nt + 31) / 32; }

int swr_launch_hist_spectra(int N, int nt, const double2* cols, double2* hspec, cudaStream_t s) {
    if (nt < kHistFftMinNt || N < 2) return -2;
    k_hist_spectra<<<4 * (N - 1), 32, 0, s>>>(N, nt, swr_hist_blocks(nt), cols, hspec);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int swr_set_wait_hook(long long max_polls, int withhold) {
    const long long lim = max_polls > 0 ? max_polls : kWaitPolls;
    const int wh = withhold >= 0 ? withhold : -1;
    if (cudaMemcpyToSymbol(d_wait_poll_limit, &lim, sizeof(lim)) != cudaSuccess ||
        cudaMemcpyToSymbol(d_wait_withhold, &wh, sizeof(wh)) != cudaSuccess)
        return -1;
    return 0;
}

size_t swr_causal_scratch_bytes(int N) {
    // xsw: 2 x 2(N-1) complex sweep values, then N-1 progress counters and the abort
    // flag, kProgStride ints apart (a batched plan passes N = its total interface count + 1)
    return sizeof(double2) * (size_t)4 * (N - 1) + sizeof(int) * (size_t)N * kProgStride;
}

// Interfaces one cooperative launch can hold (all CTAs resident at once).
int swr_causal_capacity(int) {
    int dev = 0, nsm = 0, per = 0, perf = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_causal_wave<false>,
                                                      kCausalThreads, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perf, k_causal_wave<true>,
                                                      kCausalThreads, 0) != cudaSuccess)
        return 0;
    return nsm * std::min(per, perf);
}

namespace {
// Dynamic shared memory for a launch of ncta CTAs of kernel fn: as much as lets no more
// than ceil(ncta / SMs) CTAs share an SM (the history sums of CTAs on one SM share its
// FP64 pipes, so the CTAs are spread as far as the count allows), and the use made of
// it: the four Toeplitz columns (4 nt complex) when they fit.  0 when nothing is gained.
size_t causal_dyn_smem(const void* fn, int ncta, int nt, int* cols_smem) {
    *cols_smem = 0;
    int dev = 0, nsm = 0, smem_sm = 0, smem_optin = 0, reserved = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
            cudaSuccess ||
        cudaFuncGetAttributes(&fa, fn) != cudaSuccess || nsm <= 0)
        return 0;
    const int per_sm = (ncta + nsm - 1) / nsm;
    long long dyn = (long long)smem_sm / per_sm - reserved - (long long)fa.sharedSizeBytes;
    dyn = std::min<long long>(dyn, (long long)smem_optin - (long long)fa.sharedSizeBytes);
    dyn = (dyn / 1024) * 1024;
    const long long need_cols = 4LL * nt * (long long)sizeof(double2);
    if (dyn < 1024) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int fit = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, kCausalThreads, (size_t)dyn) !=
            cudaSuccess ||
        (long long)fit * nsm < ncta) {
        cudaGetLastError();
        return 0;
    }
    *cols_smem = (need_cols <= dyn) ? 1 : 0;
    return (size_t)dyn;
}
}  // namespace

// Single instance (inst == NULL): interfaces 0..N-2; x (and P) are preset here.
// Batched plan: interfaces k0 .. k0+nif_group-1 of the nif_total, whole instances only
// (a wave never waits on an interface outside its instance); the caller presets the
// whole of x (and P) to the unset pattern (0xff bytes) before the first group when
// sweeps == 0 or H >= 1.
int swr_launch_causal(int N, int nt, const double2* cols, const double2* lag0, const double2* y,
                      double2* x, int sweeps, void* scratch, int* status, cudaStream_t s,
                      const InstInfo* inst, const int* if_inst, int k0, int nif_group,
                      int nif_total, const double2* Gw, int H, double2* P,
                      const double2* hspec, double2* xspec) {
    if (H < 0 || H > kWinMaxH || (H > 0 && (!Gw || !P)) || (H > 0 && sweeps > 0)) return -2;
    // the FFT form of the history: single instance, value-polling form, nt >= 64
    if (inst || sweeps > 0 || nt < kHistFftMinNt || !xspec) hspec = nullptr;
    const int nbt = swr_hist_blocks(nt);
    const int nif = inst ? nif_total : N - 1;
    const int ncta = inst ? nif_group : N - 1;
    if (!inst) k0 = 0;
    if (ncta <= 0) return 0;
    double2* xsw = static_cast<double2*>(scratch);
    int* progress = reinterpret_cast<int*>(xsw + (size_t)4 * nif);
    int* abortf = progress + (size_t)nif * kProgStride;
    const int cap = swr_causal_capacity(nt);
    if (cap <= 0) return -1;
    if (ncta > cap) return -2;           // all CTAs must be resident at once
    const bool flag = (sweeps == 0);
    if (flag && H == 0) Gw = lag0;       // G_{k,k} = D_k^{-1}: the same [nif][1][4] layout
    if (cudaMemsetAsync(abortf, 0, sizeof(int), s) != cudaSuccess) return -1;
    if (flag) {
        if (!inst) {
            const size_t bytes = sizeof(double2) * (size_t)(2 * N - 2) * nt;
            if (cudaMemsetAsync(x, 0xff, bytes, s) != cudaSuccess ||
                (H > 0 && cudaMemsetAsync(P, 0xff, bytes, s) != cudaSuccess))
                return -1;
        }
    } else if (cudaMemsetAsync(progress + (size_t)k0 * kProgStride, 0,
                               sizeof(int) * (size_t)ncta * kProgStride, s) != cudaSuccess) {
        return -1;   // this launch's progress counters start at zero
    }
    const void* fn = flag ? (const void*)k_causal_wave<true> : (const void*)k_causal_wave<false>;
    // batched instances have their own nt: the columns go to shared memory only for one
    // instance
    int cols_smem = 0;
    const size_t dyn = causal_dyn_smem(fn, ncta, nt, &cols_smem);
    if (inst) cols_smem = 0;
    void* args[] = {(void*)&N, (void*)&nt, (void*)&sweeps, (void*)&cols, (void*)&lag0,
                    (void*)&y, (void*)&x, (void*)&xsw, (void*)&P, (void*)&progress,
                    (void*)&abortf, (void*)&status, (void*)&inst, (void*)&if_inst, (void*)&k0,
                    (void*)&nif, (void*)&Gw, (void*)&H, (void*)&cols_smem, (void*)&hspec,
                    (void*)&xspec, (void*)&nbt};
    if (cudaLaunchCooperativeKernel(fn, dim3(ncta), dim3(kCausalThreads), args, dyn, s) !=
        cudaSuccess)
        return -1;
    swr_count_launch(1);
    return 0;
}

// ---------------------------------------------------------------------------
// Final-time misfit and adjoint helpers.
// J = (u - u_target)^H M (u - u_target), M the P1 mass matrix on the whole grid
// (h/6 tridiag(1, 4, 1), h/3 on the two end rows); ubar = 2 (u - u_target), the
// M-weighted cotangent: dJ = Re(ubar^H M du).  Partial sums per block are added
// in a fixed order by one block: the result is reproducible.
// ---------------------------------------------------------------------------
__global__ void k_misfit_partial(const double2* __restrict__ u, const double2* __restrict__ tgt,
                                 long long n, double h, double2* __restrict__ ubar,
                                 double* __restrict__ part) {
    __shared__ double red[256];
    double acc = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const double2 e = csub(u[k], tgt[k]);
        double2 me = cscale(e, (k == 0 || k == n - 1) ? h / 3.0 : 2.0 * h / 3.0);
        if (k > 0) me = cadd(me, cscale(csub(u[k - 1], tgt[k - 1]), h / 6.0));
        if (k < n - 1) me = cadd(me, cscale(csub(u[k + 1], tgt[k + 1]), h / 6.0));
        acc += e.x * me.x + e.y * me.y;                 // Re(conj(e) (M e))
        if (ubar) ubar[k] = cscale(e, 2.0);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(const double* __restrict__ part, int nb, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double acc = 0.0;
        for (int b = 0; b < nb; ++b) acc += part[b];
        *out = acc;
    }
}

int swr_launch_misfit(const double2* u, const double2* tgt, long long n, double h, double2* ubar,
                      double* part, double* out, cudaStream_t s) {
    const int nbk = 128;   // part holds nbk + 1 doubles
    k_misfit_partial<<<nbk, 256, 0, s>>>(u, tgt, n, h, ubar, part);
    k_sum_partials<<<1, 32, 0, s>>>(part, nbk, out);
    swr_count_launch(2);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Initial state of the adjoint march: y_0 = (dt / 2i) conj(ubar).
__global__ void k_adj_seed(const double2* __restrict__ ubar, double half_dt, long long n,
                           double2* __restrict__ y) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double2 b = ubar[k];
    y[k] = make_double2(-half_dt * b.y, -half_dt * b.x);   // -i (dt/2) (b.x - i b.y)
}

// dJ/dV_k = -2 (interior + left-element + right-element parts of the potential form).
__global__ void k_grad_combine(const double* __restrict__ gint, const double* __restrict__ gl,
                               const double* __restrict__ gr, long long n, double* __restrict__ out) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    out[k] = -2.0 * (gint[k] + gl[k] + gr[k]);
}

__global__ void k_grad_step_tdep(double* __restrict__ gint, double* __restrict__ gl,
                                 double* __restrict__ gr, long long nx, int n,
                                 double* __restrict__ out) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nx) return;
    const double half = -(gint[k] + gl[k] + gr[k]);   // (1/2) dJ/dW_n
    out[(size_t)n * nx + k] += half;
    out[(size_t)(n - 1) * nx + k] += half;
    gint[k] = 0.0;
    gl[k] = 0.0;
    gr[k] = 0.0;
}

int swr_launch_grad_step_tdep(double* gint, double* gl, double* gr, long long nx, int n,
                              double* out, cudaStream_t s) {
    if (n < 1) return -2;
    k_grad_step_tdep<<<(unsigned)((nx + 255) / 256), 256, 0, s>>>(gint, gl, gr, nx, n, out);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int swr_launch_adj_seed(const double2* ubar, double half_dt, long long n, double2* y,
                        cudaStream_t s) {
    k_adj_seed<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ubar, half_dt, n, y);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int swr_launch_grad_combine(const double* gint, const double* gl, const double* gr, long long n,
                            double* out, cudaStream_t s) {
    k_grad_combine<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(gint, gl, gr, n, out);
    swr_count_launch(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
