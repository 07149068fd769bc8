// C ABI of libswr (declared in include/swr.h): plans, interface build, solvers.
//
// Algorithms (Besse & Xing): Algorithm 3 (V = V(x)): build d = R 0 and the first
// columns of the Toeplitz blocks X^{j,p} with three marches per interior
// subdomain, solve (I - L) g = d, final march.  Algorithm 2 / Section 5
// (V = V(t,x)): GMRES on g - R g + d, right-preconditioned by P = I - L_0.
// Algorithm 1: g <- R g with full marches.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>   // header-only; the ranges cost nothing without a tool attached

#include "swr_internal.cuh"

static std::atomic<long long> g_launches{0};
void swr_count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

struct Workspace {
    long long n = 0;
    int m = 0;
    double2* V = nullptr;       // (m+1) x n Krylov basis
    double2* Z = nullptr;       // m x n preconditioned basis vectors P^{-1} v_j (preconditioned runs)
    double2* w = nullptr;       // n
    double2* z = nullptr;       // n
    double2* r = nullptr;       // n
    double2* H = nullptr;       // (m+1) x m column-major, ldh = m+1
    double2* cs = nullptr;      // m
    double2* sn = nullptr;      // m
    double2* sv = nullptr;      // 2(m+1)+1: rotated rhs, then scratch (h2, |w|^2, |w|)
    double2* y = nullptr;       // m
    double2* h = nullptr;       // m+1 scratch for gemv coefficients
    double2* partial = nullptr; // (m+1) x nblocks
    double* res = nullptr;      // residual estimate
    double2* bcg = nullptr;     // 7 x n BiCGStab vectors (first BiCGStab solve)
};

}  // namespace

struct swr_plan_s {
    swr_desc d{};
    cudaStream_t s = nullptr;
    // N, nx, nblk: totals over the plan's instances; nt: the longest instance
    int N = 0, nx = 0, nt = 0, nblk = 0, nmax = 0, ntot = 0, nsm = 152;
    // instances (a single problem, or a batch of independent problems with equal h
    // and dt): interface vectors and Toeplitz columns concatenated
    int ninst = 1;
    bool batched = false;          // more than one instance: kernels take the tables
    std::vector<InstInfo> inst;
    std::vector<int> inst_nx, inst_xoff;
    long long nb = 0, ncols = 0;   // interface vector length, first-column length
    int nif = 0;                   // interfaces
    std::vector<std::pair<int, int>> causal_groups;   // (first interface, count) per launch
    InstInfo* d_inst = nullptr;
    int *d_blk_inst = nullptr, *d_if_inst = nullptr;
    double h = 0.0;
    double2 inv_ik{}, sigma0{}, two_sigma{};
    double2 c2{}, c2_ik{};         // S_0^2: c2 and c2 / (i kappa)
    double* d_beta = nullptr;      // S_0^2: beta_0..beta_nt
    double2* d_s02hist = nullptr;  // S_0^2: end traces of every system of a launch
    double2* d_gconv = nullptr;    // interface vector of the last successful swr_solve
    bool solved = false;
    // adjoint work, allocated by the first swr_adjoint (checkpoint interval adj_K)
    int adj_K = 0;
    // nonlinear plans: d_slab holds v_n of every step of the last solve's final march
    // (adj_K == nt), so swr_adjoint need not re-march the forward scheme
    bool nl_rec = false;
    double2 *d_ckpt = nullptr, *d_slab = nullptr, *d_ya = nullptr, *d_yb = nullptr;
    double2 *d_dy = nullptr, *d_gy = nullptr;
    double *d_gint = nullptr, *d_gl = nullptr, *d_gr = nullptr, *d_part = nullptr;
    MarchSys* d_sys_seg = nullptr;
    // nonlinear adjoint: the whole grid as one system with Neumann ends
    int* d_mono = nullptr;                          // {n, goff, loff, tc} of that system
    double2 *d_mdg = nullptr, *d_mod = nullptr;     // its A - B for V0
    FactorSet fsM;
    MarchSys* d_sys_mono = nullptr;
    std::vector<int> off, n, goff, loff, tc;
    int *d_n = nullptr, *d_goff = nullptr, *d_loff = nullptr, *d_tc = nullptr;
    double2 *d_dg = nullptr, *d_od = nullptr;       // A - B for V (static) or V0
    double2 *d_dg0 = nullptr, *d_od0 = nullptr;     // A - B for V = 0
    FactorSet fsL[5], fs0L[5];     // chunked factorisations for L = 4, 8, 16, 12, 2 (V and V = 0)
    swr_tuning tune{};             // execution choices (swr_plan_ex; zero: defaults)
    int forceL = 0;                // tune.chunk_L (0: chosen per launch)
    bool autotune = true;          // tune.autotune >= 0: measured launch shapes
    // V(t,x): factor every step's matrix once per build and stream the factors
    // (tune.tdep_precomp < 0, or too little free memory: refactorise inside the march)
    int tdep_pre = -1;             // -1: not decided yet
    // launch shapes chosen by the autotuner: {kind, nsys, L, C, G, T, ngroups, ragged}
    std::vector<std::array<int, 8>> tuned;
    // host copies of the uploaded system lists (device pointer, systems), and the
    // ragged packings built for them: key (list, count, L, T) -> device tables
    std::vector<std::pair<const MarchSys*, std::vector<MarchSys>>> host_sys;
    struct Packing {
        const MarchSys* sys;
        int nsys, L, T, nctas, gmax;
        int* d_start;
        int2* d_rag;
    };
    std::vector<Packing> packings;
    // The build after the first is captured into a CUDA graph (assembly,
    // factorisations, marches, lag-0 setup) and later builds replay it
    // (tune.graph < 0 disables).  Launches inside the graph are timed by their own
    // events, read back after the replay.
    bool use_graph = true, capturing = false, graph_pending = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    long long graph_kernels = 0;
    static const int NGPROF = 64;
    int gcount = 0;
    int gkind[NGPROF] = {};
    long long gwork[NGPROF] = {};
    cudaEvent_t gev[2 * NGPROF] = {};
    double2* d_u0 = nullptr;
    double* d_V = nullptr;
    double* d_Vbar = nullptr;      // potential of the preconditioner operator (MEAN_POTENTIAL)
    double2* d_iface = nullptr;    // d (nblk blocks) followed by cols (4N blocks)
    double2* d_iface0 = nullptr;   // L_0: zero d (nblk blocks) followed by cols (4N blocks)
    double2* d_lag0 = nullptr;     // (N-1) x 4, for L
    double2* d_lag0_0 = nullptr;   // for L_0
    double2* d_hist = nullptr;     // scratch of the causal substitution
    double2* d_gtmp = nullptr;     // nblk x nt scratch
    double2* d_gtmp2 = nullptr;
    double2* d_trace = nullptr;    // N x 2 x nt
    MarchSys *d_sys_build = nullptr, *d_sys_R = nullptr, *d_sys_final = nullptr;
    int nsys_build = 0;
    long long work_build = 0, work_build_imp = 0, work_R = 0;   // point-steps per launch
    int* d_status = nullptr;
    // subdomains too long for one cluster of the constant-matrix march: every march of
    // the plan runs on the whole grid (k_march_long), its state in d_long
    bool long_march = false;
    void* d_long = nullptr;
    size_t long_bytes = 0;
    // Toeplitz applies through the FFT (tune.toeplitz_fft < 0: direct causal sums):
    // transform length fftM (0: direct), twiddles, spectra of the two column sets
    int fftM = 0;
    double2* d_W = nullptr;
    double2 *d_spec = nullptr, *d_spec0 = nullptr;
    // static V, Robin: u(T) by superposition of the build marches' recorded states
    // instead of a final march (tune.superpose < 0, or too little free memory: final march)
    bool superpose = false;
    double2* d_urec = nullptr;
    std::vector<long long> rec_base;   // per subdomain: Phi_l (nt x n_j), Phi_r, U_d (n_j)
    long long* d_rec_base = nullptr;
    unsigned long long* d_pit = nullptr;   // nonlinear marches: nodes x inner iterations
    double* d_scal = nullptr;      // [0] jump
    Workspace ws;
    int causal_sweeps = 0;
    bool auto_sweeps = false;      // pc_sweeps < 0: chosen from the lag-0 corners at the first build
    int causal_H = 0;              // >= 1: window form of the substitution (exact lag-0 solve)
    double2* d_Gw = nullptr;       // rows of the lag-0 inverse, [nif][2H+1][4]
    double2* d_Pwin = nullptr;     // window form: partial right-hand sides P_n, layout of y
    // FFT form of the substitution's history sums (single instance, nt >= 64): the
    // column-segment spectra (per build) and the launch's block spectra
    double2* d_hspec = nullptr;
    double2* d_hspec0 = nullptr;   // the same for L_0 (zero / mean-potential preconditioner)
    double2* d_xspec = nullptr;
    // S_0^3, S_0^4, S_1^2, S_1^4: per-end kernels (own, flux update) and s = 0 factors
    double2 *d_kap = nullptr, *d_kout = nullptr, *d_rho = nullptr;
    bool built = false;
    bool have_L0 = false;
    int two_level = 1;             // two-level separator solve for cluster-spread systems
    double2* d_hseg = nullptr;     // S_0^2 adjoint: segment marches' end traces [2][N][2][nt+1]
    // the interface problem the matrix-free operator (V(t,x), Algorithm 2) applies:
    // the forward one (the plan's u0 and d, factors in time order) unless the adjoint
    // of a time-dependent plan has switched to its time-reversed problem
    const double2* cur_u0 = nullptr;
    const double2* cur_d = nullptr;
    int cur_rev = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    double t_build_ms = 0.0;
    // per-launch timing ring: kind 0 = march, 1 = Toeplitz apply, 2 = P^{-1}
    static const int NPROF = 128;
    cudaEvent_t pev[2 * NPROF] = {};
    int pkind[NPROF] = {};
    long long pwork[NPROF] = {};
    int pcount = 0;
    swr_stats stats{};
};

namespace {

// Failing CUDA calls are reported on stderr while a call into a plan created with
// swr_tuning.debug >= 1 runs on this thread (set at the entry points).
thread_local int t_debug = 0;
bool debug_on() { return t_debug >= 1; }

// Named host range around each phase of the method (build, interface solve, final
// state, adjoint) for timeline tools (Nsight Systems and the like).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
swr_status cuda_fail(cudaError_t e, const char* what, int line) {
    if (debug_on()) fprintf(stderr, "libswr: %s failed at line %d: %s\n", what, line, cudaGetErrorString(e));
    return SWR_ERR_CUDA;
}
swr_status launch_fail(const char* what, int line) {
    cudaError_t e = cudaGetLastError();
    if (debug_on())
        fprintf(stderr, "libswr: launch of %s failed at line %d: %s\n", what, line, cudaGetErrorString(e));
    return SWR_ERR_CUDA;
}

#define CK(x)                                               \
    do {                                                    \
        cudaError_t ck_e_ = (x);                            \
        if (ck_e_ != cudaSuccess) return cuda_fail(ck_e_, #x, __LINE__); \
    } while (0)
#define LK(x)                                               \
    do {                                                    \
        if ((x) != 0) return launch_fail(#x, __LINE__);     \
    } while (0)

template <typename T>
swr_status dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return SWR_ERR_NOMEM;
    }
    return SWR_OK;
}

// Resolve the pending launch timings (call only after the stream is synchronised).
void prof_add(swr_plan_t p, int kind, long long work, float ms) {
    if (kind == 0 || kind == 3) {   // 3: a nonlinear march, also counted on its own
        p->stats.march_launches += 1;
        p->stats.march_point_steps += work;
        p->stats.march_ms += ms;
        if (kind == 3) {
            p->stats.nl_march_launches += 1;
            p->stats.nl_march_ms += ms;
        }
    } else if (kind == 1) {
        p->stats.toeplitz_launches += 1;
        p->stats.toeplitz_ms += ms;
    } else {
        p->stats.precond_calls += 1;
        p->stats.precond_ms += ms;
    }
}

void prof_flush(swr_plan_t p) {
    for (int i = 0; i < p->pcount; ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p->pev[2 * i], p->pev[2 * i + 1]);
        prof_add(p, p->pkind[i], p->pwork[i], ms);
    }
    p->pcount = 0;
    if (p->graph_pending) {   // launches of the last graph replay
        for (int i = 0; i < p->gcount; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, p->gev[2 * i], p->gev[2 * i + 1]);
            prof_add(p, p->gkind[i], p->gwork[i], ms);
        }
        p->graph_pending = false;
    }
}

// Bracket a launch with events; when the ring is full, synchronise and resolve.
int prof_begin(swr_plan_t p, int kind, long long work) {
    if (p->capturing) {   // a launch inside the build graph: its own events
        if (p->gcount == swr_plan_s::NGPROF) return -1;
        const int i = p->gcount++;
        p->gkind[i] = kind;
        p->gwork[i] = work;
        cudaEventRecord(p->gev[2 * i], p->s);
        return 1000000 + i;
    }
    if (p->pcount == swr_plan_s::NPROF) {
        cudaStreamSynchronize(p->s);
        prof_flush(p);
    }
    const int i = p->pcount++;
    p->pkind[i] = kind;
    p->pwork[i] = work;
    cudaEventRecord(p->pev[2 * i], p->s);
    return i;
}
void prof_end(swr_plan_t p, int i) {
    if (i < 0) return;
    if (i >= 1000000)
        cudaEventRecord(p->gev[2 * (i - 1000000) + 1], p->s);
    else
        cudaEventRecord(p->pev[2 * i + 1], p->s);
}

swr_status read_status(swr_plan_t p) {
    int st = 0;
    CK(cudaMemcpyAsync(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, p->s));
    CK(cudaStreamSynchronize(p->s));
    prof_flush(p);
    if (st & ST_SINGULAR) return SWR_ERR_SINGULAR;
    if (st & ST_NONFINITE) return SWR_ERR_NONFINITE;
    if (st & ST_TIMEOUT) return SWR_ERR_TIMEOUT;
    if (st & ST_NL_NOCONV) return SWR_ERR_NOT_CONVERGED;
    return SWR_OK;
}

// Launch geometry of a march over nsys systems.  Every system has P+1 threads
// (P chunks of <= L interior nodes, one separator each).  The chunk length L is
// the largest of 16, 8, 4 that still gives about four full warps per SM (the
// FP64 pipe saturates with one warp per SM sub-partition); systems are packed G
// to a CTA so that the CTAs fit in one wave, and a system too long for one CTA
// (or too few systems for the SMs) is spread over a thread-block cluster.
struct MarchCfg {
    int L = 8, C = 1, G = 1, T = 32, ngroups = 1;
    int ragged = 0;   // C == 1 only: systems packed by size (G, ngroups from the packing)
};

inline int chunks_for(int nmax, int L) { return (nmax - 1 + L) / (L + 1); }

// march kernel kinds: constant matrix; V(t,x) refactorised per step inside the
// march; nonlinear; V(t,x) with per-step factorisations streamed from HBM
enum { MK_STATIC = 0, MK_TDEP = 1, MK_NL = 2, MK_TSTAT = 3, MK_ADJ = 4 };

// Threads per CTA and CTA groups for a shape whose L, C, G are set; tps = P + 1.
inline MarchCfg shape_of(MarchCfg c, int tps, int nsys) {
    if (c.C == 1) {
        c.T = ((c.G * tps + 31) / 32) * 32;
        c.ngroups = (nsys + c.G - 1) / c.G;
    } else {
        c.T = (((tps + c.C - 1) / c.C + 31) / 32) * 32;
        c.ngroups = nsys;
    }
    return c;
}

// Largest CTA the march kernel of this kind and chunk length is compiled for.
inline int march_tmax(int kind, int L) {
    return (L == 16 || kind == MK_TDEP || kind == MK_NL || kind == MK_ADJ) ? 256 : 384;
}

// Extra arguments of the segment marches of the adjoint gradient (MK_ADJ).
struct SegArgs {
    int mode = 0;             // 0 march, 1 record v, 2 accumulate the potential form
    int t0 = 0;               // first step of the segment within the flux blocks
    long long gstride = 0;    // flux block stride (0: the launch's own step count)
    double2* hist = nullptr;  // S_0^2: end traces over the whole time axis [N][2][nt+1]
    int ht0 = 0;              // absolute step before the segment's first step
    int fstep0 = 0;           // V(t,x): per-step factor set of the segment's first step
    int frev = 0;             // walk the factor sets backwards (time-reversed march)
    double2* vrec = nullptr;
    const double2* vfwd = nullptr;
    double *gint = nullptr, *gl = nullptr, *gr = nullptr;
};

// fixL > 0: the modelled shape for that chunk length (no tuned entry)
MarchCfg march_config(const swr_plan_t p, int nsys, int kind = MK_STATIC, int fixL = 0) {
    MarchCfg c;
    if (p->long_march && kind == MK_STATIC) {   // the grid-wide march, 16-node chunks
        c.L = 16;
        c.T = 256;
        return c;
    }
    for (const auto& t : p->tuned)
        if (fixL == 0 && t[0] == kind && t[1] == nsys) {
            c.L = t[2];
            c.C = t[3];
            c.G = t[4];
            c.T = t[5];
            c.ngroups = t[6];
            c.ragged = t[7];
            return c;
        }
    const int nsm = p->nsm;
    const long long want = (long long)nsm * 4 * 32;
    const int cand[3] = {16, 8, 4};
    int L = 4;
    if (fixL > 0) {
        L = fixL;
    } else if (kind == MK_TDEP) {
        L = 4;   // per-step refactorisation keeps LU, spikes and state in registers
    } else if (kind == MK_NL && (p->forceL == 2 || p->forceL == 4 || p->forceL == 8)) {
        L = p->forceL;
    } else if (kind == MK_NL || kind == MK_ADJ) {
        // state, right-hand side, iterate and solve (or the adjoint sums) per node
        // in registers: L <= 8
        L = ((long long)(chunks_for(p->nmax, 8) + 1) * nsys >= want) ? 8 : 4;
    } else if (p->forceL && p->forceL != 2) {
        L = p->forceL;
    } else {
        for (int k = 0; k < 3; ++k) {
            const long long tps = chunks_for(p->nmax, cand[k]) + 1;
            if (tps * nsys >= want || cand[k] == 4) {
                L = cand[k];
                break;
            }
        }
    }
    c.L = L;
    const int P = chunks_for(p->nmax, L);
    const int tps = P + 1;
    const int TMAX = march_tmax(kind, L);
    if (tps <= TMAX) {
        c.C = 1;
        c.G = std::max(1, std::min(TMAX / tps, (nsys + nsm - 1) / nsm));
        const int nctas = (nsys + c.G - 1) / c.G;
        if (c.G == 1 && nctas * 2 <= nsm) {
            // few systems: spread each over a cluster, keeping >= 64 threads per CTA
            int C = std::min(16, nsm / std::max(nsys, 1));
            C = std::min(C, tps / 64);
            if (C >= 2) c.C = C;
        }
    } else {
        c.C = (tps + TMAX - 1) / TMAX;
        c.G = 1;
        if (nsys * c.C * 2 <= nsm) {
            int C = std::min(16, nsm / std::max(nsys, 1));
            C = std::min(C, tps / 64);
            c.C = std::max(c.C, C);
        }
    }
    c = shape_of(c, tps, nsys);
    if (p->batched && kind == MK_STATIC && c.C == 1) {
        // uneven subdomains of several instances: pack by size instead of padding
        c.ragged = 1;
        c.T = std::min(TMAX, std::max(128, ((tps + 31) / 32) * 32));
    }
    return c;
}

inline int lidx(int L) { return L == 4 ? 0 : (L == 8 ? 1 : (L == 16 ? 2 : (L == 2 ? 4 : 3))); }

inline double2 cmul_h(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Ragged packing of a system list for chunk length L and T threads per CTA:
// systems sorted by step count, then by thread count P_j + 1 (largest first),
// fill CTAs in order, a new CTA starting when the next system does not fit.  A
// CTA then holds systems of (nearly) equal length, and the longest CTAs come
// first in the grid, which the hardware schedules first.  Returns the cached
// packing, or nullptr when a system needs more than T threads or the list is
// not known on the host.
const swr_plan_s::Packing* ragged_packing(swr_plan_t p, const MarchSys* d_sys, int nsys, int L,
                                          int T) {
    for (const auto& k : p->packings)
        if (k.sys == d_sys && k.nsys == nsys && k.L == L && k.T == T) return &k;
    const MarchSys* hs = nullptr;
    for (const auto& e : p->host_sys) {
        const MarchSys* b = e.first;
        if (d_sys >= b && d_sys + nsys <= b + e.second.size()) {
            hs = e.second.data() + (d_sys - b);
            break;
        }
    }
    if (!hs) return nullptr;
    std::vector<int> need(nsys), order(nsys);
    for (int q = 0; q < nsys; ++q) {
        need[q] = chunks_for(p->n[hs[q].sub], L) + 1;
        if (need[q] > T) return nullptr;
        order[q] = q;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (hs[a].nt != hs[b].nt) return hs[a].nt > hs[b].nt;
        return need[a] > need[b];
    });
    std::vector<int> start{0};
    std::vector<int2> rag;
    int used = 0, gmax = 0, cnt = 0;
    for (int q : order) {
        if (used + need[q] > T) {
            start.push_back((int)rag.size());
            gmax = std::max(gmax, cnt);
            used = cnt = 0;
        }
        rag.push_back(make_int2(q, used));
        used += need[q];
        ++cnt;
    }
    gmax = std::max(gmax, cnt);
    start.push_back((int)rag.size());
    swr_plan_s::Packing k{d_sys, nsys, L, T, (int)start.size() - 1, gmax, nullptr, nullptr};
    if (dalloc(&k.d_start, start.size()) || dalloc(&k.d_rag, rag.size())) {
        cudaFree(k.d_start);
        return nullptr;
    }
    if (cudaMemcpy(k.d_start, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice) ||
        cudaMemcpy(k.d_rag, rag.data(), sizeof(int2) * rag.size(), cudaMemcpyHostToDevice)) {
        cudaFree(k.d_start);
        cudaFree(k.d_rag);
        return nullptr;
    }
    p->packings.push_back(k);
    return &p->packings.back();
}

// Launch one march with an explicit shape; nt_run < nt runs only the first steps
// (the autotuner's probes).  Returns 0 or a launcher error code.
int launch_cfg(swr_plan_t p, const MarchCfg& cfg, int kind, bool zero_potential,
               const MarchSys* d_sys, int nsys, const double2* gin, double2* gout, double2* uT,
               double2* trace, const double2* u0, int nt_run, const SegArgs& seg = SegArgs()) {
    if (cfg.C > 16) return -2;
    const FactorSet& fs = zero_potential ? p->fs0L[lidx(cfg.L)] : p->fsL[lidx(cfg.L)];
    if (fs.L != cfg.L) return -3;
    MarchArgs a{};
    a.nt = nt_run;
    a.C = cfg.C;
    a.G = cfg.G;
    a.T = cfg.T;
    int ngroups = cfg.ngroups;
    if (cfg.ragged) {
        if (cfg.C != 1 || kind != MK_STATIC || fs.nsteps > 1) return -2;
        const swr_plan_s::Packing* pk = ragged_packing(p, d_sys, nsys, cfg.L, cfg.T);
        if (!pk) return -2;
        a.rag_start = pk->d_start;
        a.rag = pk->d_rag;
        a.G = pk->gmax;
        ngroups = pk->nctas;
    }
    a.nsys = nsys;
    a.sys = d_sys;
    a.sub_n = p->d_n;
    a.sub_goff = p->d_goff;
    a.sub_tc = p->d_tc;
    a.u0 = u0;
    a.gin = gin;
    a.gout = gout;
    a.uT = uT;
    a.trace = trace;
    a.urec = (!zero_potential && p->superpose) ? p->d_urec : nullptr;
    a.two_sigma = p->two_sigma;
    a.inv_ik = p->inv_ik;
    a.status = p->d_status;
    a.two_level = p->two_level;
    a.fstep0 = seg.fstep0;
    a.frev = seg.frev;
    a.t0 = seg.t0;
    a.gstride = seg.gstride > 0 ? seg.gstride : nt_run;
    a.nxrec = p->nx;
    a.vrec = seg.vrec;
    a.vfwd = seg.vfwd;
    a.gint = seg.gint;
    a.gl = seg.gl;
    a.gr = seg.gr;
    a.h12 = p->h / 12.0;
    if (p->d.tc >= SWR_TC_S03 && !zero_potential) {
        a.kap = p->d_kap;
        a.kout = p->d_kout;
        a.rho = p->d_rho;
        a.kstride = p->nt + 1;
    }
    if (p->d.tc >= SWR_TC_S02) {
        a.s02 = 1;
        a.beta = p->d_beta;
        a.hist = p->d_s02hist;
        a.c2_ik = p->c2_ik;
        a.two_c2 = make_double2(2.0 * p->c2.x, 2.0 * p->c2.y);
        if (seg.hist) {   // a segment of the adjoint's marches: traces over the whole axis
            a.hist = seg.hist;
            a.hstride = p->nt + 1;
            a.ht0 = seg.ht0;
        }
    }
    const double kappa = 2.0 / p->d.dt * (p->h / 6.0);
    if (p->long_march && kind == MK_STATIC) {
        if (seg.mode != 0 || cfg.L != 16) return -2;
        return swr_launch_march_long(fs, a, p->d_long, p->long_bytes, p->nsm, p->s);
    }
    if (kind == MK_TDEP)
        return swr_launch_march_tdep(fs, a, p->d_V, p->nx, p->h, kappa,
                                     cmul_h(p->sigma0, p->inv_ik), cfg.ngroups, p->s);
    if (kind == MK_NL)   // mode 0, or 1 recording v_n into seg.vrec
        return swr_launch_march_nl(fs, a, (p->h / 12.0) / kappa, p->d.nl_coef, p->d.nl_tol,
                                   p->d.nl_maxit, nullptr, cfg.ngroups, p->s, seg.mode,
                                   p->d_pit);
    const int rc = swr_launch_march(fs, a, ngroups, p->s, seg.mode);
    if (rc == 0 && (cfg.C > 1 || (cfg.G == 1 && !cfg.ragged)) && seg.mode == 0 &&
        fs.nsteps == 1 && fs.tl_ok && p->two_level)
        p->stats.two_level_launches += 1;
    return rc;
}

inline int march_kind(swr_plan_t p, bool zero_potential) {
    if (zero_potential) return MK_STATIC;
    if (p->d.vkind == SWR_V_TIME) return p->tdep_pre > 0 ? MK_TSTAT : MK_TDEP;
    if (p->d.vkind == SWR_V_NONLINEAR) return MK_NL;
    return MK_STATIC;
}

// vrec (nonlinear marches only): also record v_n of every step, rows of nx values
swr_status run_march(swr_plan_t p, bool zero_potential, const MarchSys* d_sys, int nsys,
                     const double2* gin, double2* gout, double2* uT, double2* trace,
                     const double2* u0, long long work, double2* vrec = nullptr) {
    const int kind = march_kind(p, zero_potential);
    const MarchCfg cfg = march_config(p, nsys, kind);
    const int pi = prof_begin(p, kind == MK_NL ? 3 : 0, work);
    SegArgs sa;
    if (vrec) {
        if (kind != MK_NL) return SWR_ERR_UNSUPPORTED;
        sa.mode = 1;
        sa.vrec = vrec;
    }
    if (p->cur_rev && !zero_potential) {   // time-reversed problem: last step's factors first
        sa.fstep0 = p->nt - 1;
        sa.frev = 1;
    }
    const int rc = launch_cfg(p, cfg, kind, zero_potential, d_sys, nsys, gin, gout, uT, trace, u0,
                              p->nt, sa);
    prof_end(p, pi);
    if (rc == -2) return SWR_ERR_UNSUPPORTED;
    if (rc == -3) return SWR_ERR_STATE;
    if (rc != 0) return launch_fail(kind == MK_TDEP ? "march (time-dependent)" : (kind == MK_NL ? "march (nonlinear)" : "march"), __LINE__);
    return SWR_OK;
}

// Assemble A - B for V (NULL: V = 0) and factor it for chunk length L.
swr_status factor_for(swr_plan_t p, FactorSet& fs, int L, const double* V, double2* dg,
                      double2* od) {
    if (fs.L != L || fs.nsteps != 1) {
        if (swr_factor_alloc(fs, p->N, L, chunks_for(p->nmax, L), p->s) != 0) return SWR_ERR_NOMEM;
    }
    if (swr_launch_factor(fs, p->N, p->d_n, p->d_loff, dg, od, p->d_status, p->s) != 0) {
        cudaGetLastError();
        return SWR_ERR_CUDA;
    }
    if (swr_launch_factor_tl(fs, p->N, p->d_loff, dg, od, p->d_status, p->s) == -1) {
        cudaGetLastError();
        return SWR_ERR_CUDA;
    }
    return SWR_OK;
}

// Measured launch-shape choice.  The first build of a plan times short probe
// marches (the first few steps of the real launch, into the real output buffer
// with stride nt_probe) over candidate chunk lengths L, cluster sizes C and
// packings G, and caches the fastest shape per (kernel kind, system count) in
// p->tuned; march_config returns it from then on.  Candidates the device cannot
// launch (cluster too large for the SMs' resources) are skipped.  The model
// behind the default shape (four full warps per SM, one wave of CTAs) is only a
// first guess: wave quantisation, cluster scheduling and the PCR depth move the
// optimum by up to 2x, so the probes decide.
swr_status factor_steps_for(swr_plan_t p, FactorSet& fs, int L, int nsteps);

swr_status tune_march(swr_plan_t p, int kind, bool zero_potential, const MarchSys* d_sys,
                      int nsys, double2* gout, const double* V, double2* dg, double2* od) {
    if (!p->autotune || nsys <= 0 || (p->long_march && kind == MK_STATIC)) return SWR_OK;
    for (const auto& t : p->tuned)
        if (t[0] == kind && t[1] == nsys) return SWR_OK;
    const MarchCfg guess = march_config(p, nsys, kind);
    std::vector<int> Ls;
    if (kind == MK_TDEP) Ls = {4};
    else if (kind == MK_NL && (p->forceL == 2 || p->forceL == 4 || p->forceL == 8))
        Ls = {p->forceL};
    else if (kind == MK_NL) Ls = {8, 4, 2};   // 2: two warps per sub-partition for short systems
    else if (kind == MK_ADJ) Ls = {8, 4};
    else if (p->forceL && p->forceL != 2) Ls = {p->forceL};
    else Ls = {16, 12, 8, 4};   // 12: six systems of ~780 nodes in one 384-thread CTA
    std::vector<MarchCfg> cands;
    cands.push_back(guess);
    for (int L : Ls) {
        const int tps = chunks_for(p->nmax, L) + 1;
        const int TMAX = march_tmax(kind, L);
        MarchCfg c;
        c.L = L;
        if (tps <= TMAX) {
            const int Gmax = std::max(1, std::min(TMAX / tps, nsys));
            std::vector<int> Gs;
            for (int G = 1; G <= Gmax; G *= 2) Gs.push_back(G);
            Gs.push_back(Gmax);
            Gs.push_back(std::min(Gmax, (nsys + p->nsm - 1) / p->nsm));
            Gs.push_back(std::min(Gmax, (nsys + 2 * p->nsm - 1) / (2 * p->nsm)));
            for (int G : Gs) {
                c.C = 1;
                c.G = G;
                cands.push_back(shape_of(c, tps, nsys));
            }
        }
        // batched plans of uneven subdomains: ragged packings by size, for the CTA
        // sizes that hold the largest system
        if (p->batched && kind == MK_STATIC && tps <= TMAX) {
            const int Ts[8] = {64, 96, 128, 160, 192, 256, 320, 384};
            for (int T : Ts) {
                if (T < tps || T > TMAX) continue;
                MarchCfg r;
                r.L = L;
                r.C = 1;
                r.T = T;
                r.ragged = 1;
                cands.push_back(r);
            }
        }
        // clusters: each CTA keeps at least one full warp of separators and
        // none is left without separators
        const int Cmin = std::max(2, (tps + TMAX - 1) / TMAX);
        for (int C = Cmin; C <= 16; C = (C < 4 ? C + 1 : C * 2)) {
            if (C > Cmin && (tps + C - 1) / C < 32) break;
            c.C = C;
            c.G = 1;
            const MarchCfg sc = shape_of(c, tps, nsys);
            if ((C - 1) * sc.T < tps) cands.push_back(sc);
        }
    }
    // factors for every candidate chunk length (per-step kinds: the probed steps)
    // streamed per-step factors: probe enough steps that their factors overflow
    // L2 (129 MB), as in the real march, instead of probing an L2-resident set
    int ntp = std::min(p->nt, 48);
    if (kind == MK_TSTAT) {
        const size_t step = swr_factor_step_bytes(p->N, 4, chunks_for(p->nmax, 4));
        const size_t want = ((size_t)256 << 20) / std::max<size_t>(step, 1) + 1;
        ntp = (int)std::min<size_t>((size_t)p->nt, std::max<size_t>(16, std::min<size_t>(want, 256)));
    }
    for (int L : Ls) {
        FactorSet& fs = zero_potential ? p->fs0L[lidx(L)] : p->fsL[lidx(L)];
        swr_status st = (kind == MK_TSTAT) ? factor_steps_for(p, fs, L, ntp)
                                           : factor_for(p, fs, L, V, dg, od);
        if (st) return st;
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    MarchCfg best = guess;
    float best_ms = -1.f;
    for (size_t k = 0; k < cands.size(); ++k) {
        const MarchCfg& c = cands[k];
        bool dup = false;
        for (size_t q = 0; q < k && !dup; ++q)
            dup = cands[q].L == c.L && cands[q].C == c.C && cands[q].G == c.G &&
                  cands[q].ragged == c.ragged && (!c.ragged || cands[q].T == c.T);
        if (dup) continue;
        if (launch_cfg(p, c, kind, zero_potential, d_sys, nsys, nullptr, gout, nullptr, nullptr,
                       p->d_u0, ntp) != 0) {
            cudaGetLastError();
            continue;
        }
        // fastest of three timed probes (after the warm one above)
        float ms = -1.f;
        int rc = 0;
        for (int r = 0; r < 3 && rc == 0; ++r) {
            cudaEventRecord(e0, p->s);
            rc = launch_cfg(p, c, kind, zero_potential, d_sys, nsys, nullptr, gout, nullptr,
                            nullptr, p->d_u0, ntp);
            cudaEventRecord(e1, p->s);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return cuda_fail(cudaGetLastError(), "autotune probe", __LINE__);
            }
            float m = 0.f;
            cudaEventElapsedTime(&m, e0, e1);
            if (rc == 0 && (ms < 0.f || m < ms)) ms = m;
        }
        if (rc != 0) {
            cudaGetLastError();
            continue;
        }
        if (p->tune.debug >= 2)
                fprintf(stderr, "swr autotune probe kind %d nsys %d: L %d C %d G %d T %d%s %.3f ms\n",
                        kind, nsys, c.L, c.C, c.G, c.T, c.ragged ? " ragged" : "", ms);
        if (best_ms < 0.f || ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (p->tune.debug >= 1)
        fprintf(stderr, "swr autotune kind %d nsys %d: L %d C %d G %d T %d%s (%.3f ms / %d steps)\n",
                kind, nsys, best.L, best.C, best.G, best.T, best.ragged ? " ragged" : "", best_ms,
                ntp);
    p->tuned.push_back({kind, nsys, best.L, best.C, best.G, best.T, best.ngroups, best.ragged});
    if (kind == MK_TSTAT)   // probe-sized per-step sets of the losing chunk lengths
        for (int L : Ls)
            if (L != best.L) swr_factor_free(p->fsL[lidx(L)]);
    // probes may have flagged the status word with partial data; start clean
    CK(cudaMemsetAsync(p->d_status, 0, sizeof(int), p->s));
    return SWR_OK;
}

// Per-step factorisations of steps 1..nsteps of the tabulated V(t,x) in d_V.
swr_status factor_steps_for(swr_plan_t p, FactorSet& fs, int L, int nsteps) {
    if (fs.L != L || fs.nsteps != nsteps) {
        if (swr_factor_alloc(fs, p->N, L, chunks_for(p->nmax, L), p->s, nsteps, p->ntot) != 0)
            return SWR_ERR_NOMEM;
    }
    if (swr_launch_factor_steps(fs, p->N, p->d_n, p->d_goff, p->d_loff, p->d_tc, p->nmax, p->d_V,
                                p->nx, p->h, p->d.dt, p->sigma0, p->inv_ik, p->d_status,
                                p->s) != 0) {
        cudaGetLastError();
        return SWR_ERR_CUDA;
    }
    return SWR_OK;
}

swr_status assemble(swr_plan_t p, const double* V, double2* dg, double2* od) {
    // the higher-order conditions: the ends' kernels from this V first (their lag-0
    // entries are the boundary matrix entries)
    const bool gen = p->d_kap && dg == p->d_dg;
    if (gen)
        LK(swr_launch_tc_kernels(p->d.tc, V, p->N, p->d_n, p->d_goff, p->d_tc, p->nt + 1, p->h,
                                 p->d.dt, p->d_beta, p->c2, p->d_kap, p->d_kout, p->d_rho,
                                 p->s));
    swr_launch_assemble_static(V, p->N, p->d_n, p->d_goff, p->d_loff, p->d_tc, p->nmax, p->h,
                               p->d.dt, p->sigma0, p->inv_ik, dg, od, p->s,
                               gen ? p->d_kap : nullptr, p->nt + 1);
    CK(cudaGetLastError());
    return SWR_OK;
}

// March systems of every instance.  Flux offsets are absolute (complex entries):
// an instance's interface blocks (2N-2 of nt) start at its foff, block 2k = r_k,
// 2k+1 = l_{k+1}; its first columns start at nb + coff in the build buffer
// (d followed by the columns), slot 4j + p - 1 = X^{j,p}.
std::vector<MarchSys> build_systems(const swr_plan_s* p, bool with_d) {
    std::vector<MarchSys> v;
    const long long nb = p->nb;
    // superposed u(T): every impulse march records its states, the d march its final state
    const bool rec = p->superpose;
    auto slot = [&](int sub, int which, int nt) -> long long {   // 0: Phi_l, 1: Phi_r, 2: U_d
        return rec ? p->rec_base[sub] + (long long)which * nt * p->n[sub] : 0;
    };
    if (with_d) {   // d = R 0: one march per subdomain, all instances first
        for (const InstInfo& I : p->inst)
            for (int j = 0; j < I.N; ++j) {
                MarchSys s{I.sub0 + j, rec ? SYS_REC_LAST : 0, I.nt, -1, -1, -1, -1,
                           slot(I.sub0 + j, 2, I.nt)};
                if (j > 0) s.out_a = (int)(I.foff + (long long)(2 * (j - 1)) * I.nt);      // r_{j-1}
                if (j < I.N - 1) s.out_b = (int)(I.foff + (long long)(2 * (j + 1) - 1) * I.nt);  // l_{j+1}
                v.push_back(s);
            }
    }
    for (const InstInfo& I : p->inst) {   // l impulse: X^{j,1} (r_{j-1}), X^{j,3} (l_{j+1})
        const long long c = nb + I.coff;
        for (int j = 1; j < I.N; ++j) {
            MarchSys s{I.sub0 + j, SYS_ZERO_U0 | SYS_IMP_L | (rec ? SYS_REC_U : 0), I.nt, -1, -1,
                       (int)(c + (long long)(4 * j + 0) * I.nt), -1, slot(I.sub0 + j, 0, I.nt)};
            if (j < I.N - 1) s.out_b = (int)(c + (long long)(4 * j + 2) * I.nt);
            v.push_back(s);
        }
    }
    for (const InstInfo& I : p->inst) {   // r impulse: X^{j,2} (r_{j-1}), X^{j,4} (l_{j+1})
        const long long c = nb + I.coff;
        for (int j = 0; j < I.N - 1; ++j) {
            MarchSys s{I.sub0 + j, SYS_ZERO_U0 | SYS_IMP_R | (rec ? SYS_REC_U : 0), I.nt, -1, -1,
                       -1, (int)(c + (long long)(4 * j + 3) * I.nt), slot(I.sub0 + j, 1, I.nt)};
            if (j > 0) s.out_a = (int)(c + (long long)(4 * j + 1) * I.nt);
            v.push_back(s);
        }
    }
    return v;
}

// One system per subdomain (global order) reading and writing interface vectors.
std::vector<MarchSys> apply_systems(const swr_plan_s* p, int extra_flags) {
    std::vector<MarchSys> v;
    for (const InstInfo& I : p->inst)
        for (int j = 0; j < I.N; ++j) {
            MarchSys s{I.sub0 + j, extra_flags, I.nt, -1, -1, -1, -1};
            if (j > 0) {
                s.in_l = (int)(I.foff + (long long)(2 * j - 1) * I.nt);
                s.out_a = (int)(I.foff + (long long)(2 * (j - 1)) * I.nt);
            }
            if (j < I.N - 1) {
                s.in_r = (int)(I.foff + (long long)(2 * j) * I.nt);
                s.out_b = (int)(I.foff + (long long)(2 * (j + 1) - 1) * I.nt);
            }
            v.push_back(s);
        }
    return v;
}

swr_status upload_systems(MarchSys** dst, const std::vector<MarchSys>& v,
                          swr_plan_s* p = nullptr) {
    cudaFree(*dst);
    *dst = nullptr;
    swr_status st = dalloc(dst, v.size());
    if (st) return st;
    CK(cudaMemcpy(*dst, v.data(), sizeof(MarchSys) * v.size(), cudaMemcpyHostToDevice));
    if (p) p->host_sys.push_back({*dst, v});
    return SWR_OK;
}

swr_status ensure_workspace(swr_plan_t p) {
    Workspace& w = p->ws;
    const long long n = p->nb;
    const int m = p->d.restart;
    if (w.V && w.m == m && w.n == n) return SWR_OK;
    cudaFree(w.V); cudaFree(w.w); cudaFree(w.z); cudaFree(w.r); cudaFree(w.H); cudaFree(w.cs);
    cudaFree(w.sn); cudaFree(w.sv); cudaFree(w.y); cudaFree(w.h); cudaFree(w.partial);
    cudaFree(w.res); cudaFree(w.Z); cudaFree(w.bcg);
    w = Workspace();
    w.n = n;
    w.m = m;
    swr_status st = SWR_OK;
    if ((st = dalloc(&w.V, (size_t)(m + 1) * n))) return st;
    if ((st = dalloc(&w.w, n))) return st;
    if ((st = dalloc(&w.z, n))) return st;
    if ((st = dalloc(&w.r, n))) return st;
    if ((st = dalloc(&w.H, (size_t)(m + 1) * m))) return st;
    if ((st = dalloc(&w.cs, m))) return st;
    if ((st = dalloc(&w.sn, m))) return st;
    if ((st = dalloc(&w.sv, 3 * (m + 1) + 2))) return st;
    if ((st = dalloc(&w.y, m))) return st;
    if ((st = dalloc(&w.h, m + 1))) return st;
    if ((st = dalloc(&w.partial, (size_t)(m + 2) * 512))) return st;
    if ((st = dalloc(&w.res, 1))) return st;
    return SWR_OK;
}

// ||v||_2 (device -> host)
// Interface algebra over all instances of the plan (tables only for a batch).
int p_toeplitz(swr_plan_t p, const double2* cols, const double2* x, const double2* add,
               double2* y, int mode) {
    if (p->fftM) {
        const double2* spec = (cols == p->d_iface + p->nb) ? p->d_spec
                            : (cols == p->d_iface0 + p->nb) ? p->d_spec0 : nullptr;
        if (spec)
            return swr_launch_toeplitz_fft(p->N, p->nt, spec, x, add, y, mode, p->fftM, p->d_W,
                                           p->s, p->batched ? p->d_inst : nullptr,
                                           p->d_blk_inst, p->nblk);
    }
    return swr_launch_toeplitz(p->N, p->nt, cols, x, add, y, mode, p->s,
                               p->batched ? p->d_inst : nullptr, p->d_blk_inst, p->nblk, p->nt);
}
int p_lag0(swr_plan_t p, const double2* cols, double2* lag0) {
    return swr_launch_lag0_setup(p->N, p->nt, cols, lag0, p->s,
                                 p->batched ? p->d_inst : nullptr, p->d_if_inst, p->nif);
}
int p_jump(swr_plan_t p) {
    return swr_launch_jump(p->d_trace, p->d_sys_final, p->N, p->nt, p->d_scal, p->s,
                           p->batched ? p->d_inst : nullptr, p->d_if_inst, p->nif);
}
int p_causal(swr_plan_t p, const double2* cols, const double2* lag0, const double2* y,
             double2* x) {
    // the window form applies to the plan's own operator (the rows of its lag-0 inverse)
    const bool own = cols == p->d_iface + p->nb;   // the plan's own operator
    const bool win = p->causal_H > 0 && own;
    const double2* Gw = win ? p->d_Gw : nullptr;
    const int H = win ? p->causal_H : 0;
    const int sweeps = win ? 0 : p->causal_sweeps;
    if (!p->batched)
        return swr_launch_causal(p->N, p->nt, cols, lag0, y, x, sweeps, p->d_hist, p->d_status,
                                 p->s, nullptr, nullptr, 0, 0, 0, Gw, H, p->d_Pwin,
                                 own ? p->d_hspec
                                 : (p->d_iface0 && cols == p->d_iface0 + p->nb) ? p->d_hspec0
                                                                                  : nullptr,
                                 p->d_xspec);
    // the values are the hand-off (sweeps == 0): x and the window's partial right-hand
    // sides start unset, once for all groups
    if (sweeps == 0) {
        const size_t bytes = sizeof(double2) * (size_t)p->nb;
        if (cudaMemsetAsync(x, 0xff, bytes, p->s) != cudaSuccess ||
            (H > 0 && cudaMemsetAsync(p->d_Pwin, 0xff, bytes, p->s) != cudaSuccess))
            return -1;
    }
    // whole instances per cooperative launch, as many as fit at once
    for (const auto& g : p->causal_groups) {
        const int rc = swr_launch_causal(p->N, p->nt, cols, lag0, y, x, sweeps, p->d_hist,
                                         p->d_status, p->s, p->d_inst, p->d_if_inst, g.first,
                                         g.second, p->nif, Gw, H, p->d_Pwin);
        if (rc) return rc;
    }
    return 0;
}

swr_status norm2(swr_plan_t p, const double2* v, long long n, double* out) {
    Workspace& w = p->ws;
    LK(swr_launch_dots(v, 0, 1, v, n, w.partial, 512, w.h, p->s));
    double2 r;
    CK(cudaMemcpyAsync(&r, w.h, sizeof(double2), cudaMemcpyDeviceToHost, p->s));
    CK(cudaStreamSynchronize(p->s));
    prof_flush(p);
    *out = std::sqrt(std::max(r.x, 0.0));
    return SWR_OK;
}

// y = A x for the interface system (I - L) g = d.
swr_status apply_A(swr_plan_t p, const double2* x, double2* y) {
    const long long n = p->nb;
    if (p->d.vkind == SWR_V_STATIC) {
        const int pi = prof_begin(p, 1, 0);
        const int rc = p_toeplitz(p, p->d_iface + p->nb, x, nullptr, y, 0);
        prof_end(p, pi);
        return rc ? SWR_ERR_UNSUPPORTED : SWR_OK;
    }
    // matrix-free: y = x - R x + d   (Algorithm 2)
    const double2* u0 = p->cur_u0 ? p->cur_u0 : p->d_u0;
    const double2* d = p->cur_d ? p->cur_d : p->d_iface;
    swr_status st = run_march(p, false, p->d_sys_R, p->N, x, y, nullptr, nullptr, u0, p->work_R);
    if (st) return st;
    LK(swr_launch_axpby(y, x, n, make_double2(-1.0, 0.0), make_double2(1.0, 0.0), p->s));
    LK(swr_launch_axpby(y, d, n, make_double2(1.0, 0.0), make_double2(1.0, 0.0), p->s));
    return SWR_OK;
}

bool has_precond(swr_plan_t p) {
    return (p->d.precond == SWR_PC_CAUSAL && p->d.vkind == SWR_V_STATIC) ||
           ((p->d.precond == SWR_PC_ZERO_POTENTIAL || p->d.precond == SWR_PC_MEAN_POTENTIAL) &&
            p->have_L0);
}

// x = P^{-1} y
swr_status apply_M(swr_plan_t p, const double2* y, double2* x) {
    const double2* cols;
    const double2* lag0;
    if (p->d.precond == SWR_PC_CAUSAL && p->d.vkind == SWR_V_STATIC) {
        cols = p->d_iface + (size_t)p->nb;
        lag0 = p->d_lag0;
    } else if ((p->d.precond == SWR_PC_ZERO_POTENTIAL || p->d.precond == SWR_PC_MEAN_POTENTIAL) &&
               p->have_L0) {
        cols = p->d_iface0 + (size_t)p->nb;
        lag0 = p->d_lag0_0;
    } else {
        return SWR_ERR_STATE;
    }
    const int pi = prof_begin(p, 2, 0);
    int rc = p_causal(p, cols, lag0, y, x);
    prof_end(p, pi);
    if (rc == -2) return SWR_ERR_UNSUPPORTED;
    if (rc) return launch_fail("causal substitution", __LINE__);
    return SWR_OK;
}

// Restarted right-preconditioned GMRES(m) on A g = d (Saad, Alg. 6.9 with
// classical Gram-Schmidt applied twice).  Stops on the true residual.
// GMRES(m) on (I - L) g = b (b = d for the forward problem), stopping on the
// true residual ||b - (I - L) g||_2 < tol.
swr_status gmres(swr_plan_t p, const double2* b, double tol, double2* g, bool g_init,
                 swr_info* info) {
    NvtxRange nvtx_range("swr: GMRES interface solve");
    swr_status st = ensure_workspace(p);
    if (st) return st;
    Workspace& w = p->ws;
    const long long n = w.n;
    const int m = w.m, ldh = m + 1;
    const bool pc = has_precond(p);
    // the preconditioned basis is kept, so the update g += P^{-1} V y = Z y costs no
    // further substitution
    if (pc && !w.Z && (st = dalloc(&w.Z, (size_t)m * n))) return st;
    if (!g_init) CK(cudaMemsetAsync(g, 0, sizeof(double2) * n, p->s));
    // r = b - A g
    if (g_init) {
        if ((st = apply_A(p, g, w.r))) return st;
        LK(swr_launch_axpby(w.r, b, n, make_double2(-1.0, 0.0), make_double2(1.0, 0.0), p->s));
    } else {
        CK(cudaMemcpyAsync(w.r, b, sizeof(double2) * n, cudaMemcpyDeviceToDevice, p->s));
    }
    double beta;
    if ((st = norm2(p, w.r, n, &beta))) return st;
    if (info) info->residual0 = beta;
    int it = 0, restarts = 0;
    while (beta >= tol && it < p->d.maxit) {
        if (!std::isfinite(beta)) return SWR_ERR_NONFINITE;
        // v_0 = r / beta, sv = (beta, 0, ...)
        CK(cudaMemsetAsync(w.sv, 0, sizeof(double2) * (3 * (m + 1) + 2), p->s));
        double2 b0 = make_double2(beta, 0.0);
        CK(cudaMemcpyAsync(w.sv, &b0, sizeof(double2), cudaMemcpyHostToDevice, p->s));
        CK(cudaMemcpyAsync(w.sv + ldh + ldh, &b0, sizeof(double2), cudaMemcpyHostToDevice, p->s));
        LK(swr_launch_scale_by_rnorm(w.V, w.r, n, w.sv + 2 * ldh, p->s));
        CK(cudaMemsetAsync(w.H, 0, sizeof(double2) * ldh * m, p->s));
        int k = 0;
        double est = beta;
        for (int j = 0; j < m && it < p->d.maxit; ++j) {
            double2* vj = w.V + (size_t)j * n;
            const double2* av = vj;
            if (pc) {
                double2* zj = w.Z + (size_t)j * n;
                if ((st = apply_M(p, vj, zj))) return st;
                av = zj;
            }
            if ((st = apply_A(p, av, w.w))) return st;
            double2* Hc = w.H + (size_t)j * ldh;
            double2* work = w.sv + ldh;
            // first Gram-Schmidt pass -> H column
            LK(swr_launch_dots(w.V, n, j + 1, w.w, n, w.partial, 512, Hc, p->s));
            LK(swr_launch_gemv_sub(w.V, n, j + 1, Hc, w.w, n, -1.0, p->s));
            // second pass -> work[0..j]
            LK(swr_launch_dots(w.V, n, j + 1, w.w, n, w.partial, 512, work, p->s));
            LK(swr_launch_gemv_sub(w.V, n, j + 1, work, w.w, n, -1.0, p->s));
            // |w|^2 -> work[j+1]
            LK(swr_launch_dots(w.w, 0, 1, w.w, n, w.partial, 512, work + j + 1, p->s));
            LK(swr_launch_givens(w.H, ldh, w.cs, w.sn, w.sv, j, w.res, p->s));
            // v_{j+1} = w / |w|  (norm stored at work[ldh])
            LK(swr_launch_scale_by_rnorm(w.V + (size_t)(j + 1) * n, w.w, n, work + ldh, p->s));
            CK(cudaMemcpyAsync(&est, w.res, sizeof(double), cudaMemcpyDeviceToHost, p->s));
            CK(cudaStreamSynchronize(p->s));
            prof_flush(p);
            ++it;
            k = j + 1;
            if (!std::isfinite(est)) return SWR_ERR_NONFINITE;
            if (est < tol) break;
        }
        // g += P^{-1} V_k y = Z_k y
        LK(swr_launch_lsq(w.H, ldh, w.sv, k, w.y, p->s));
        LK(swr_launch_gemv_sub(pc ? w.Z : w.V, n, k, w.y, g, n, 1.0, p->s));
        // true residual
        if ((st = apply_A(p, g, w.r))) return st;
        LK(swr_launch_axpby(w.r, b, n, make_double2(-1.0, 0.0), make_double2(1.0, 0.0), p->s));
        if ((st = norm2(p, w.r, n, &beta))) return st;
        ++restarts;
    }
    if (info) {
        info->iterations = it;
        info->restarts = restarts;
        info->residual = beta;
    }
    if (!std::isfinite(beta)) return SWR_ERR_NONFINITE;
    return beta < tol ? SWR_OK : SWR_ERR_NOT_CONVERGED;
}

// Right-preconditioned BiCGStab (van der Vorst 1992) on (I - L) g = b, the
// alternative Krylov method of Section 6 (Tables 6-7), with the plan's
// preconditioner as for GMRES; complex inner products <x, y> = x^H y, shadow residual
// r^ = r_0.  Each iteration: two operator applications and two preconditioner
// applications; stops on the true residual ||b - (I - L) g||_2 < tol, recomputed
// when the recurrence's residual passes the test.
swr_status bicgstab(swr_plan_t p, const double2* b, double tol, double2* g, bool g_init,
                    swr_info* info) {
    NvtxRange nvtx_range("swr: BiCGStab interface solve");
    swr_status st = ensure_workspace(p);
    if (st) return st;
    Workspace& w = p->ws;
    const long long n = w.n;
    const bool pc = has_precond(p);
    if (!w.bcg && (st = dalloc(&w.bcg, (size_t)7 * n))) return st;
    double2 *r = w.bcg, *rh = r + n, *pv = rh + n, *v = pv + n, *ph = v + n, *sv = ph + n,
            *t = sv + n;
    double2* sh = w.z;                                 // P^{-1} s
    auto dot = [&](const double2* x, const double2* y, double2* out) -> swr_status {
        LK(swr_launch_dots(x, 0, 1, y, n, w.partial, 512, w.h, p->s));
        CK(cudaMemcpyAsync(out, w.h, sizeof(double2), cudaMemcpyDeviceToHost, p->s));
        CK(cudaStreamSynchronize(p->s));
        return SWR_OK;
    };
    auto cdiv = [](double2 a, double2 c) {
        const double den = c.x * c.x + c.y * c.y;
        return make_double2((a.x * c.x + a.y * c.y) / den, (a.y * c.x - a.x * c.y) / den);
    };
    auto precond = [&](const double2* x, double2* y) -> swr_status {
        if (pc) return apply_M(p, x, y);
        CK(cudaMemcpyAsync(y, x, sizeof(double2) * n, cudaMemcpyDeviceToDevice, p->s));
        return SWR_OK;
    };
    auto true_residual = [&](double* out) -> swr_status {   // r = b - A g
        if ((st = apply_A(p, g, r))) return st;
        LK(swr_launch_axpby(r, b, n, make_double2(-1.0, 0.0), make_double2(1.0, 0.0), p->s));
        return norm2(p, r, n, out);
    };
    double res = 0.0;
    if (g_init) {
        if ((st = true_residual(&res))) return st;
    } else {
        CK(cudaMemsetAsync(g, 0, sizeof(double2) * n, p->s));
        CK(cudaMemcpyAsync(r, b, sizeof(double2) * n, cudaMemcpyDeviceToDevice, p->s));
        if ((st = norm2(p, r, n, &res))) return st;
    }
    if (info) info->residual0 = res;
    CK(cudaMemcpyAsync(rh, r, sizeof(double2) * n, cudaMemcpyDeviceToDevice, p->s));
    CK(cudaMemsetAsync(pv, 0, sizeof(double2) * n, p->s));
    CK(cudaMemsetAsync(v, 0, sizeof(double2) * n, p->s));
    double2 rho_prev = make_double2(1.0, 0.0), alpha = rho_prev, omega = rho_prev;
    int it = 0;
    const double2 one = make_double2(1.0, 0.0);
    while (res >= tol && it < p->d.maxit) {
        if (!std::isfinite(res)) return SWR_ERR_NONFINITE;
        double2 rho;
        if ((st = dot(rh, r, &rho))) return st;
        if (rho.x == 0.0 && rho.y == 0.0) break;          // breakdown: restart below
        const double2 beta = cmul_h(cdiv(rho, rho_prev), cdiv(alpha, omega));
        // p = r + beta (p - omega v)
        LK(swr_launch_axpby(pv, v, n, one, make_double2(-omega.x, -omega.y), p->s));
        LK(swr_launch_axpby(pv, r, n, beta, one, p->s));
        if ((st = precond(pv, ph))) return st;
        if ((st = apply_A(p, ph, v))) return st;
        double2 rv;
        if ((st = dot(rh, v, &rv))) return st;
        alpha = cdiv(rho, rv);
        // s = r - alpha v
        CK(cudaMemcpyAsync(sv, r, sizeof(double2) * n, cudaMemcpyDeviceToDevice, p->s));
        LK(swr_launch_axpby(sv, v, n, one, make_double2(-alpha.x, -alpha.y), p->s));
        double sn = 0.0;
        if ((st = norm2(p, sv, n, &sn))) return st;
        ++it;
        if (sn < tol) {
            LK(swr_launch_axpby(g, ph, n, one, alpha, p->s));
            if ((st = true_residual(&res))) return st;
            if (res < tol) break;
            CK(cudaMemcpyAsync(rh, r, sizeof(double2) * n, cudaMemcpyDeviceToDevice, p->s));
            rho_prev = alpha = omega = one;
            CK(cudaMemsetAsync(pv, 0, sizeof(double2) * n, p->s));
            CK(cudaMemsetAsync(v, 0, sizeof(double2) * n, p->s));
            continue;
        }
        if ((st = precond(sv, sh))) return st;
        if ((st = apply_A(p, sh, t))) return st;
        double2 ts, tt;
        if ((st = dot(t, sv, &ts)) || (st = dot(t, t, &tt))) return st;
        omega = cdiv(ts, tt);
        // g += alpha p^ + omega s^,  r = s - omega t
        LK(swr_launch_axpby(g, ph, n, one, alpha, p->s));
        LK(swr_launch_axpby(g, sh, n, one, omega, p->s));
        CK(cudaMemcpyAsync(r, sv, sizeof(double2) * n, cudaMemcpyDeviceToDevice, p->s));
        LK(swr_launch_axpby(r, t, n, one, make_double2(-omega.x, -omega.y), p->s));
        if ((st = norm2(p, r, n, &res))) return st;
        rho_prev = rho;
        if (res < tol && (st = true_residual(&res))) return st;
    }
    if (info) {
        info->iterations = it;
        info->residual = res;
    }
    if (!std::isfinite(res)) return SWR_ERR_NONFINITE;
    return res < tol ? SWR_OK : SWR_ERR_NOT_CONVERGED;
}

// Fixed point g <- L g + d (Algorithm 3 with the fixed point) or g <- R g
// (Algorithm 1), until ||g^{k+1} - g^k||_2 < tol.
swr_status fixed_point(swr_plan_t p, double2* g, bool g_init, bool classical, swr_info* info) {
    NvtxRange nvtx_range("swr: fixed-point interface iteration");
    swr_status st = ensure_workspace(p);
    if (st) return st;
    Workspace& w = p->ws;
    const long long n = w.n;
    if (!g_init) CK(cudaMemsetAsync(g, 0, sizeof(double2) * n, p->s));
    double diff = INFINITY;
    int it = 0;
    while (it < p->d.maxit) {
        if (classical) {
            if ((st = run_march(p, false, p->d_sys_R, p->N, g, w.z, nullptr, nullptr, p->d_u0,
                                p->work_R)))
                return st;
        } else {
            if (p_toeplitz(p, p->d_iface + p->nb, g, p->d_iface, w.z, 1))
                return SWR_ERR_UNSUPPORTED;
        }
        CK(cudaMemcpyAsync(w.r, w.z, sizeof(double2) * n, cudaMemcpyDeviceToDevice, p->s));
        LK(swr_launch_axpby(w.r, g, n, make_double2(1.0, 0.0), make_double2(-1.0, 0.0), p->s));
        CK(cudaMemcpyAsync(g, w.z, sizeof(double2) * n, cudaMemcpyDeviceToDevice, p->s));
        if ((st = norm2(p, w.r, n, &diff))) return st;
        ++it;
        if (!std::isfinite(diff)) return SWR_ERR_NONFINITE;
        if (diff < p->d.tol_abs) break;
    }
    if (info) {
        info->iterations = it;
        info->residual = diff;
    }
    return diff < p->d.tol_abs ? SWR_OK : SWR_ERR_NOT_CONVERGED;
}

// Direct time-causal solve of (I - L) g = d (static V): block forward substitution
// in time, g = P^{-1} d, refined by g += P^{-1} r, r = d - (I - L) g, while the
// true residual ||r||_2 >= tol (at most maxit substitutions).
swr_status causal_direct(swr_plan_t p, double2* g, bool g_init, swr_info* info) {
    NvtxRange nvtx_range("swr: causal interface solve");
    swr_status st = ensure_workspace(p);
    if (st) return st;
    Workspace& w = p->ws;
    const long long n = w.n;
    const double2* cols = p->d_iface + (size_t)p->nb;
    auto residual = [&](double* out) -> swr_status {   // w.r = d - (I - L) g
        if (p_toeplitz(p, cols, g, nullptr, w.z, 0)) return SWR_ERR_UNSUPPORTED;
        CK(cudaMemcpyAsync(w.r, p->d_iface, sizeof(double2) * n, cudaMemcpyDeviceToDevice, p->s));
        LK(swr_launch_axpby(w.r, w.z, n, make_double2(1.0, 0.0), make_double2(-1.0, 0.0), p->s));
        return norm2(p, w.r, n, out);
    };
    double res = INFINITY;
    if (g_init) {
        if ((st = residual(&res))) return st;
    } else {
        CK(cudaMemsetAsync(g, 0, sizeof(double2) * n, p->s));
        CK(cudaMemcpyAsync(w.r, p->d_iface, sizeof(double2) * n, cudaMemcpyDeviceToDevice, p->s));
        if ((st = norm2(p, w.r, n, &res))) return st;
    }
    const double res0 = res;
    int it = 0;
    while (res >= p->d.tol_abs && it < p->d.maxit) {
        const int pi = prof_begin(p, 2, 0);
        const int rc = p_causal(p, cols, p->d_lag0, w.r, w.w);
        prof_end(p, pi);
        if (rc == -2) return SWR_ERR_UNSUPPORTED;
        if (rc) return launch_fail("causal substitution", __LINE__);
        LK(swr_launch_axpby(g, w.w, n, make_double2(1.0, 0.0), make_double2(1.0, 0.0), p->s));
        ++it;
        if ((st = residual(&res))) return st;
        if (!std::isfinite(res)) return SWR_ERR_NONFINITE;
    }
    if (info) {
        info->iterations = it;
        info->residual = res;
        info->residual0 = res0;
    }
    return res < p->d.tol_abs ? SWR_OK : SWR_ERR_NOT_CONVERGED;
}

// Nonlinear potential (Section 5): g^{k+1} = g^k - P^{-1}(g^k - R_nl g^k) with the
// plan's preconditioner (reading of Eq. chp2_algopd_NL), or g^{k+1} = R_nl g^k
// without one (Algorithm 1); stop when ||g^{k+1} - g^k||_2 < tol.
swr_status nl_fixed_point(swr_plan_t p, double2* g, bool g_init, swr_info* info) {
    swr_status st = ensure_workspace(p);
    if (st) return st;
    Workspace& w = p->ws;
    const long long n = w.n;
    const bool pc = has_precond(p) && p->d.solver != SWR_SOLVER_CLASSICAL;
    if (!g_init) CK(cudaMemsetAsync(g, 0, sizeof(double2) * n, p->s));
    double diff = INFINITY;
    int it = 0;
    while (it < p->d.maxit) {
        if ((st = run_march(p, false, p->d_sys_R, p->N, g, w.z, nullptr, nullptr, p->d_u0,
                            p->work_R)))
            return st;
        // r = g - R_nl g
        CK(cudaMemcpyAsync(w.r, g, sizeof(double2) * n, cudaMemcpyDeviceToDevice, p->s));
        LK(swr_launch_axpby(w.r, w.z, n, make_double2(1.0, 0.0), make_double2(-1.0, 0.0), p->s));
        const double2* dx = w.r;
        if (pc) {
            if ((st = apply_M(p, w.r, w.w))) return st;
            dx = w.w;
        }
        LK(swr_launch_axpby(g, dx, n, make_double2(1.0, 0.0), make_double2(-1.0, 0.0), p->s));
        if ((st = norm2(p, dx, n, &diff))) return st;
        ++it;
        if (!std::isfinite(diff)) return SWR_ERR_NONFINITE;
        if (diff < p->d.tol_abs) break;
    }
    if (info) {
        info->iterations = it;
        info->residual = diff;
    }
    return diff < p->d.tol_abs ? SWR_OK : SWR_ERR_NOT_CONVERGED;
}

}  // namespace

// ===========================================================================
// Entry points
// ===========================================================================
// ---------------------------------------------------------------------------
// Nonlinear adjoint (Eq. CNS_NL / AvMNL with f(v) = c|v|^2, static V0).  Every
// step of the forward scheme solves F(v_n) = A0 v_n + M_{c|v_n|^2} v_n -
// B u_{n-1} = 0, u_n = 2 v_n - u_{n-1} (A0 = (2i/dt) M - S + M_V0, B = (2i/dt)
// M).  With dJ = Re(lambda_N^H du_N), lambda_N = M ubar, the adjoint of one step
// solves T_n^* mu_n = 2 lambda_n, lambda_{n-1} = B^H mu_n - lambda_n, where T_n
// is the real-linear derivative of F at v_n.  Conjugated and scaled,
// z_n = B^{-1} conj(lambda_n) and omega_n = conj(mu_n) / 2:
//     At omega + 2c conj(v_n) . Re(v_n^T (dM_W/dW_k) omega) = B z_n,
//     z_{n-1} = 2 omega_n - z_n,        z_N = (dt / 2i) conj(ubar),
// (At = A0 + M_{c|v_n|^2}), the same march as the forward one with the inner
// fixed point linearised about the recorded v_n, and
//     dJ/dV0_k = -2 Re sum_n omega_n^T (dM_V/dV_k) v_n.
// The adjoint step is not a subdomain problem with a fixed interface operator
// (its matrix changes with v_n), so the gradient is taken of the monodomain
// scheme, which the converged SWR solution reproduces: the whole grid is one
// system spread over a thread-block cluster.
// ---------------------------------------------------------------------------

// Tables and factorisation of the one-system grid (first call only).
swr_status mono_setup(swr_plan_t p) {
    if (p->d_mono) return SWR_OK;
    const int nx = p->nx;
    const int L = chunks_for(nx, 4) + 1 <= 16 * 256 ? 4 : 8;
    if (chunks_for(nx, L) + 1 > 16 * 256) return SWR_ERR_UNSUPPORTED;
    swr_status st = SWR_OK;
    const int tab[4] = {nx, 0, 0, 0};
    MarchSys sys{};
    sys.sub = 0;
    sys.flags = SYS_WRITE_UT;
    sys.nt = p->nt;
    sys.in_l = sys.in_r = sys.out_a = sys.out_b = -1;
    if ((st = dalloc(&p->d_mono, 4)) || (st = dalloc(&p->d_mdg, nx)) ||
        (st = dalloc(&p->d_mod, nx)) || (st = dalloc(&p->d_sys_mono, 1)))
        return st;
    CK(cudaMemcpyAsync(p->d_mono, tab, sizeof(tab), cudaMemcpyHostToDevice, p->s));
    CK(cudaMemcpyAsync(p->d_sys_mono, &sys, sizeof(sys), cudaMemcpyHostToDevice, p->s));
    swr_launch_assemble_static(p->d_V, 1, p->d_mono, p->d_mono + 1, p->d_mono + 2, p->d_mono + 3,
                               nx, p->h, p->d.dt, p->sigma0, p->inv_ik, p->d_mdg, p->d_mod, p->s);
    CK(cudaGetLastError());
    if (swr_factor_alloc(p->fsM, 1, L, chunks_for(nx, L), p->s) != 0) return SWR_ERR_NOMEM;
    if (swr_launch_factor(p->fsM, 1, p->d_mono, p->d_mono + 2, p->d_mdg, p->d_mod, p->d_status,
                          p->s) != 0) {
        cudaGetLastError();
        return SWR_ERR_CUDA;
    }
    // two-level separator data with a reduced system over the whole CTA (thousands of
    // separators); without it the march keeps the cluster-wide PCR
    if (swr_launch_factor_tl(p->fsM, 1, p->d_mono + 2, p->d_mdg, p->d_mod, p->d_status, p->s,
                             true) == -1) {
        cudaGetLastError();
        return SWR_ERR_CUDA;
    }
    CK(cudaStreamSynchronize(p->s));
    return SWR_OK;
}

// One march of the nonlinear scheme over the one-system grid for nrun steps:
// mode 0 from u0 to uT, 1 also records v_n of every step into the slab, 2 the
// adjoint march reading it (see above).
swr_status mono_nl_march(swr_plan_t p, int mode, const double2* u0, double2* uT, int nrun) {
    const FactorSet& fs = p->fsM;
    const int tps = fs.P + 1;
    MarchCfg c;
    c.L = fs.L;
    c.G = 1;
    c.C = std::max((tps + 255) / 256, std::min(16, tps / 64));
    c.C = std::max(1, std::min(c.C, std::max(1, p->nsm / 2)));
    c = shape_of(c, tps, 1);
    if (c.C > 16 || c.T > 256) return SWR_ERR_UNSUPPORTED;
    MarchArgs a{};
    a.nt = nrun;
    a.C = c.C;
    a.G = 1;
    a.T = c.T;
    a.nsys = 1;
    a.sys = p->d_sys_mono;
    a.sub_n = p->d_mono;
    a.sub_goff = p->d_mono + 1;
    a.sub_tc = p->d_mono + 3;
    a.u0 = u0;
    a.uT = uT;
    a.two_sigma = p->two_sigma;
    a.inv_ik = p->inv_ik;
    a.status = p->d_status;
    a.gstride = nrun;
    a.nxrec = p->nx;
    a.vrec = p->d_slab;
    a.vfwd = p->d_slab;
    a.gint = p->d_gint;
    a.gl = p->d_gl;
    a.gr = p->d_gr;
    a.h12 = p->h / 12.0;
    a.two_level = p->two_level;
    const double kappa = 2.0 / p->d.dt * (p->h / 6.0);
    const int pi = prof_begin(p, 3, (long long)p->nx * nrun);
    const int rc = swr_launch_march_nl(fs, a, (p->h / 12.0) / kappa, p->d.nl_coef, p->d.nl_tol,
                                       p->d.nl_maxit, nullptr, 1, p->s, mode, p->d_pit);
    prof_end(p, pi);
    if (rc == -2) return SWR_ERR_UNSUPPORTED;
    if (rc) return launch_fail("nonlinear adjoint march", __LINE__);
    return SWR_OK;
}

extern "C" {

const char* swr_status_string(swr_status s) {
    switch (s) {
        case SWR_OK: return "SWR_OK";
        case SWR_ERR_ARG: return "SWR_ERR_ARG: invalid argument";
        case SWR_ERR_SINGULAR: return "SWR_ERR_SINGULAR: zero pivot in A - B";
        case SWR_ERR_NOT_CONVERGED: return "SWR_ERR_NOT_CONVERGED: iteration cap reached";
        case SWR_ERR_NONFINITE: return "SWR_ERR_NONFINITE: NaN or Inf";
        case SWR_ERR_TIMEOUT: return "SWR_ERR_TIMEOUT: bounded device wait gave up";
        case SWR_ERR_NOMEM: return "SWR_ERR_NOMEM: device allocation failed";
        case SWR_ERR_CUDA: return "SWR_ERR_CUDA: CUDA runtime error";
        case SWR_ERR_STATE: return "SWR_ERR_STATE: call order violated";
        case SWR_ERR_UNSUPPORTED:
            return "SWR_ERR_UNSUPPORTED: combination not supported by the library";
    }
    return "unknown swr_status";
}

int64_t swr_kernel_launch_count(void) { return (int64_t)g_launches.load(); }

swr_status swr_test_wait_hook(int64_t max_polls, int32_t withhold) {
    return swr_set_wait_hook((long long)max_polls, (int)withhold) == 0 ? SWR_OK : SWR_ERR_CUDA;
}

void swr_destroy(swr_plan_t p) {
    if (!p) return;
    cudaStreamSynchronize(p->s);
    cudaFree(p->d_n); cudaFree(p->d_goff); cudaFree(p->d_loff); cudaFree(p->d_tc);
    cudaFree(p->d_dg); cudaFree(p->d_od); cudaFree(p->d_dg0); cudaFree(p->d_od0);
    for (int k = 0; k < 5; ++k) {
        swr_factor_free(p->fsL[k]);
        swr_factor_free(p->fs0L[k]);
    }
    cudaFree(p->d_beta); cudaFree(p->d_s02hist); cudaFree(p->d_gconv);
    cudaFree(p->d_inst); cudaFree(p->d_blk_inst); cudaFree(p->d_if_inst);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (auto& e : p->gev)
        if (e) cudaEventDestroy(e);
    for (auto& k : p->packings) {
        cudaFree(k.d_start);
        cudaFree(k.d_rag);
    }
    cudaFree(p->d_ckpt); cudaFree(p->d_slab); cudaFree(p->d_ya); cudaFree(p->d_yb); cudaFree(p->d_hseg);
    cudaFree(p->d_dy); cudaFree(p->d_gy); cudaFree(p->d_gint); cudaFree(p->d_gl);
    cudaFree(p->d_gr); cudaFree(p->d_part); cudaFree(p->d_sys_seg);
    cudaFree(p->d_mono); cudaFree(p->d_mdg); cudaFree(p->d_mod); cudaFree(p->d_sys_mono);
    swr_factor_free(p->fsM);
    cudaFree(p->d_u0); cudaFree(p->d_V); cudaFree(p->d_Vbar); cudaFree(p->d_iface); cudaFree(p->d_iface0);
    cudaFree(p->d_lag0); cudaFree(p->d_lag0_0); cudaFree(p->d_hist); cudaFree(p->d_gtmp);
    cudaFree(p->d_gtmp2); cudaFree(p->d_trace);
    cudaFree(p->d_sys_build); cudaFree(p->d_sys_R); cudaFree(p->d_sys_final);
    cudaFree(p->d_status); cudaFree(p->d_scal); cudaFree(p->d_pit);
    cudaFree(p->d_urec); cudaFree(p->d_rec_base);
    cudaFree(p->d_W); cudaFree(p->d_spec); cudaFree(p->d_spec0); cudaFree(p->d_Gw);
    cudaFree(p->d_Pwin); cudaFree(p->d_hspec); cudaFree(p->d_hspec0);
    cudaFree(p->d_xspec);
    cudaFree(p->d_kap); cudaFree(p->d_kout); cudaFree(p->d_rho); cudaFree(p->d_long);
    Workspace& w = p->ws;
    cudaFree(w.V); cudaFree(w.w); cudaFree(w.z); cudaFree(w.r); cudaFree(w.H); cudaFree(w.cs);
    cudaFree(w.sn); cudaFree(w.sv); cudaFree(w.y); cudaFree(w.h); cudaFree(w.partial);
    cudaFree(w.res);
    for (auto& e : p->ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : p->pev)
        if (e) cudaEventDestroy(e);
    delete p;
}

// Validate and set up one plan over count problem instances (count = 1: swr_plan).
static swr_status plan_create(const swr_desc* ds, int count, const swr_tuning* tuning,
                              swr_plan_t* out, void* stream) {
    NvtxRange nvtx_range("swr_plan");
    if (!out) return SWR_ERR_ARG;
    *out = nullptr;
    if (!ds || count < 1) return SWR_ERR_ARG;
    if (tuning) {
        const swr_tuning& u = *tuning;
        if (!(u.chunk_L == 0 || u.chunk_L == 2 || u.chunk_L == 4 || u.chunk_L == 8 ||
              u.chunk_L == 12 || u.chunk_L == 16) ||
            u.debug < 0)
            return SWR_ERR_ARG;
    }
    const swr_desc* d = &ds[0];
    for (int i = 0; i < count; ++i) {
        const swr_desc& e = ds[i];
        if (e.nx < 3 || e.nt < 1 || !(e.dt > 0.0) || e.nsub < 2 || !(e.b0 > e.a0))
            return SWR_ERR_ARG;
    }
    if (d->vkind < 0 || d->vkind > 2 || d->tc < SWR_TC_ROBIN || d->tc > SWR_TC_S14)
        return SWR_ERR_ARG;
    // the higher-order conditions: V(x) only (their kernels are time invariant there)
    if (d->tc >= SWR_TC_S03 &&
        (d->vkind != SWR_V_STATIC || d->precond == SWR_PC_ZERO_POTENTIAL ||
         d->precond == SWR_PC_MEAN_POTENTIAL))
        return SWR_ERR_UNSUPPORTED;
    if (d->solver < 0 || d->solver > 4 || d->precond < 0 || d->precond > 3) return SWR_ERR_ARG;
    if (d->solver == SWR_SOLVER_BICGSTAB && d->vkind == SWR_V_NONLINEAR) return SWR_ERR_ARG;
    if (d->solver == SWR_SOLVER_CAUSAL && d->vkind != SWR_V_STATIC) return SWR_ERR_ARG;
    if (d->vkind == SWR_V_NONLINEAR && d->solver == SWR_SOLVER_GMRES) return SWR_ERR_ARG;
    if (d->vkind == SWR_V_TIME && d->solver == SWR_SOLVER_FIXED_POINT) return SWR_ERR_ARG;
    if (d->vkind == SWR_V_TIME && (long long)(d->nt + 1) * d->nx > (1LL << 31)) return SWR_ERR_ARG;
    if (d->precond == SWR_PC_CAUSAL && d->vkind != SWR_V_STATIC) return SWR_ERR_ARG;
    const double h0 = (d->b0 - d->a0) / (d->nx - 1);
    if (count > 1) {
        // a batch shares everything but the grid extent, the step count and the partition
        if (d->vkind != SWR_V_STATIC) return SWR_ERR_UNSUPPORTED;
        for (int i = 1; i < count; ++i) {
            const swr_desc& e = ds[i];
            const double hi = (e.b0 - e.a0) / (e.nx - 1);
            if (std::fabs(hi - h0) > 1e-12 * h0 || e.dt != d->dt || e.vkind != d->vkind ||
                e.tc != d->tc || e.tc_re != d->tc_re || e.tc_im != d->tc_im ||
                e.solver != d->solver || e.restart != d->restart || e.maxit != d->maxit ||
                e.tol_abs != d->tol_abs || e.precond != d->precond || e.pc_sweeps != d->pc_sweeps)
                return SWR_ERR_ARG;
        }
    }
    swr_plan_t p = new (std::nothrow) swr_plan_s();
    if (!p) return SWR_ERR_NOMEM;
    p->d = *d;
    if (tuning) p->tune = *tuning;
    t_debug = p->tune.debug;
    p->d.node_off = nullptr;
    if (p->d.restart <= 0) p->d.restart = 30;
    if (p->d.restart > 200) p->d.restart = 200;   // Gram-Schmidt kernels take <= 256 vectors
    if (p->d.maxit <= 0) p->d.maxit = 2000;
    if (!(p->d.tol_abs > 0.0)) p->d.tol_abs = 1e-10;
    if (p->d.nl_maxit <= 0) p->d.nl_maxit = 50;
    if (!(p->d.nl_tol > 0.0)) p->d.nl_tol = 1e-13;
    if (p->d.nl_coef == 0.0) p->d.nl_coef = 1.0;
    p->causal_sweeps = (d->pc_sweeps >= 0) ? std::min(d->pc_sweeps, 16) : 0;
    p->auto_sweeps = d->pc_sweeps < 0 && d->vkind == SWR_V_STATIC &&
                     (d->precond == SWR_PC_CAUSAL || d->solver == SWR_SOLVER_CAUSAL);
    p->s = (cudaStream_t)stream;
    p->ninst = count;
    p->batched = count > 1;
    p->h = h0;
    // instances: partitions, subdomain tables, interface and column offsets
    int ntot = 0, nmax = 0, xoff = 0, sub = 0, ifc = 0, blk = 0, ntmax = 0;
    long long foff = 0, coff = 0;
    for (int i = 0; i < count; ++i) {
        const swr_desc& e = ds[i];
        const int Ni = e.nsub;
        std::vector<int> off(Ni + 1);
        if (e.node_off) {
            for (int j = 0; j <= Ni; ++j) off[j] = e.node_off[j];
        } else {
            const int E = e.nx - 1, base = E / Ni, extra = E % Ni;
            off[0] = 0;
            for (int j = 0; j < Ni; ++j) off[j + 1] = off[j] + base + (j < extra ? 1 : 0);
        }
        bool ok = off[0] == 0 && off[Ni] == e.nx - 1;
        for (int j = 0; j < Ni && ok; ++j) ok = (off[j + 1] - off[j] >= 2);
        if (!ok) {
            delete p;
            return SWR_ERR_ARG;
        }
        if (count == 1) p->off = off;
        for (int j = 0; j < Ni; ++j) {
            const int nj = off[j + 1] - off[j] + 1;
            p->n.push_back(nj);
            p->goff.push_back(xoff + off[j]);
            p->loff.push_back(ntot);
            p->tc.push_back((j > 0 ? 1 : 0) | (j < Ni - 1 ? 2 : 0));
            ntot += nj;
            nmax = std::max(nmax, nj);
        }
        InstInfo I{};
        I.N = Ni;
        I.nt = e.nt;
        I.sub0 = sub;
        I.if0 = ifc;
        I.blk0 = blk;
        I.foff = foff;
        I.coff = coff;
        p->inst.push_back(I);
        p->inst_nx.push_back(e.nx);
        p->inst_xoff.push_back(xoff);
        sub += Ni;
        ifc += Ni - 1;
        blk += 2 * Ni - 2;
        foff += (long long)(2 * Ni - 2) * e.nt;
        coff += (long long)4 * Ni * e.nt;
        xoff += e.nx;
        ntmax = std::max(ntmax, e.nt);
    }
    if (foff + coff >= (1LL << 31)) {   // march systems address fluxes with 32-bit offsets
        delete p;
        return SWR_ERR_ARG;
    }
    p->N = sub;
    p->nx = xoff;
    p->nt = ntmax;
    p->nblk = blk;
    p->nif = ifc;
    p->nb = foff;
    p->ncols = coff;
    p->ntot = ntot;
    p->nmax = nmax;
    const double kappa = 2.0 / d->dt * (p->h / 6.0);
    p->inv_ik = make_double2(0.0, -1.0 / kappa);   // 1/(i kappa)
    if (d->tc >= SWR_TC_S02) {
        // S_0^2 (Section 2.2): S-bar v_n = c2 sum_{s<=n} beta_{n-s} v_s with
        // c2 = e^{-i pi/4} sqrt(2/dt); the s = n term, c2 beta_0 = c2, is the
        // boundary matrix entry sigma0
        const double r = std::sqrt(2.0 / d->dt) * std::sqrt(0.5);
        p->c2 = make_double2(r, -r);
        p->sigma0 = p->c2;
        p->two_sigma = make_double2(2.0 * r, -2.0 * r);
        p->c2_ik = cmul_h(p->c2, p->inv_ik);
    } else {
        p->sigma0 = make_double2(d->tc_re, d->tc_im);
        p->two_sigma = make_double2(2.0 * d->tc_re, 2.0 * d->tc_im);
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (p->nsm <= 0) p->nsm = 152;
    p->forceL = p->tune.chunk_L;                 // 0, 2, 4, 8, 12 or 16 (validated)
    p->autotune = p->tune.autotune >= 0;
    p->two_level = p->tune.two_level >= 0 ? 1 : 0;
    swr_status st = SWR_OK;
    const size_t nb = (size_t)p->nb;
    if (!st) st = dalloc(&p->d_n, p->N);
    if (!st) st = dalloc(&p->d_goff, p->N);
    if (!st) st = dalloc(&p->d_loff, p->N);
    if (!st) st = dalloc(&p->d_tc, p->N);
    if (!st) st = dalloc(&p->d_dg, ntot);
    if (!st) st = dalloc(&p->d_od, ntot);
    if (!st) st = dalloc(&p->d_u0, p->nx);
    if (!st) st = dalloc(&p->d_iface, nb + (size_t)p->ncols);
    if (!st) st = dalloc(&p->d_lag0, 4 * p->N);
    if (!st) st = dalloc(reinterpret_cast<char**>(&p->d_hist), swr_causal_scratch_bytes(p->N));
    if (!st && !p->batched && p->tune.history_fft >= 0 && p->nt >= kHistFftMinNt) {
        // one set of column-segment spectra per operator the substitution applies to:
        // the plan's own (static V, CAUSAL) and L_0 (zero / mean-potential preconditioner)
        const size_t hs = (size_t)4 * (p->N - 1) * swr_hist_blocks(p->nt) * 64;
        const bool own = d->vkind == SWR_V_STATIC &&
                         (d->precond == SWR_PC_CAUSAL || d->solver == SWR_SOLVER_CAUSAL);
        const bool pot = d->precond == SWR_PC_ZERO_POTENTIAL ||
                         d->precond == SWR_PC_MEAN_POTENTIAL;
        if (own) st = dalloc(&p->d_hspec, hs);
        if (!st && pot) st = dalloc(&p->d_hspec0, hs);
        if (!st && (own || pot)) st = dalloc(&p->d_xspec, hs);
    }
    if (!st) st = dalloc(&p->d_gtmp, nb);
    if (!st) st = dalloc(&p->d_gtmp2, nb);
    if (!st) st = dalloc(&p->d_trace, (size_t)p->N * 2 * p->nt);
    if (!st) st = dalloc(&p->d_status, 1);
    if (!st) st = dalloc(&p->d_scal, 4);
    if (!st) st = dalloc(&p->d_pit, 1);
    if (!st) {
        const size_t nV = (d->vkind == SWR_V_TIME) ? (size_t)(p->nt + 1) * p->nx : p->nx;
        st = dalloc(&p->d_V, nV);
    }
    if (!st && (d->precond == SWR_PC_ZERO_POTENTIAL || d->precond == SWR_PC_MEAN_POTENTIAL)) {
        st = dalloc(&p->d_Vbar, p->nx);
        if (!st) st = dalloc(&p->d_dg0, ntot);
        if (!st) st = dalloc(&p->d_od0, ntot);
        if (!st) st = dalloc(&p->d_iface0, nb + (size_t)p->ncols);
        if (!st) st = dalloc(&p->d_lag0_0, 4 * p->N);
    }
    if (!st) {
        if (cudaMemcpy(p->d_n, p->n.data(), sizeof(int) * p->N, cudaMemcpyHostToDevice) ||
            cudaMemcpy(p->d_goff, p->goff.data(), sizeof(int) * p->N, cudaMemcpyHostToDevice) ||
            cudaMemcpy(p->d_loff, p->loff.data(), sizeof(int) * p->N, cudaMemcpyHostToDevice) ||
            cudaMemcpy(p->d_tc, p->tc.data(), sizeof(int) * p->N, cudaMemcpyHostToDevice) ||
            cudaMemset(p->d_status, 0, sizeof(int)) ||
            cudaMemset(p->d_pit, 0, sizeof(unsigned long long)))
            st = SWR_ERR_CUDA;
    }
    if (!st) {
        // FFT Toeplitz applies: transform length M >= 2 nt - 1 (a power of two), for
        // 16 <= nt and M <= 4096 (three M-point buffers in shared memory)
        const bool on = p->tune.toeplitz_fft >= 0;
        int M = 1;
        while (M < 2 * p->nt - 1) M <<= 1;
        const bool want0 =
            d->precond == SWR_PC_ZERO_POTENTIAL || d->precond == SWR_PC_MEAN_POTENTIAL;
        const bool want = d->vkind == SWR_V_STATIC || want0;
        if (on && want && p->nt >= 16 && M <= 4096) {
            std::vector<double2> W(M / 2);
            for (int k = 0; k < M / 2; ++k) {
                const double a = 2.0 * M_PI * (double)k / (double)M;
                W[k] = make_double2(std::cos(a), -std::sin(a));
            }
            const size_t ns = (size_t)4 * p->N * M;
            if (dalloc(&p->d_W, (size_t)M / 2) == SWR_OK &&
                (d->vkind != SWR_V_STATIC || dalloc(&p->d_spec, ns) == SWR_OK) &&
                (!want0 || dalloc(&p->d_spec0, ns) == SWR_OK) &&
                cudaMemcpy(p->d_W, W.data(), sizeof(double2) * (M / 2), cudaMemcpyHostToDevice) ==
                    cudaSuccess) {
                p->fftM = M;
            } else {
                cudaGetLastError();
                cudaFree(p->d_W); cudaFree(p->d_spec); cudaFree(p->d_spec0);
                p->d_W = p->d_spec = p->d_spec0 = nullptr;
            }
        }
    }
    if (!st && d->vkind == SWR_V_STATIC &&
        (d->tc == SWR_TC_ROBIN ? (d->tc_re != 0.0 || d->tc_im != 0.0) : p->nt < 4260)) {
        // u(T) by superposition: Phi_l, Phi_r (nt x n_j each) and U_d per subdomain, if
        // they take at most a quarter of the free memory
        const bool on = p->tune.superpose >= 0;
        long long tot = 0;
        std::vector<long long> base(p->N, 0);
        for (const InstInfo& I : p->inst)
            for (int j = 0; j < I.N; ++j) {
                base[I.sub0 + j] = tot;
                tot += (2LL * I.nt + 1) * p->n[I.sub0 + j];
            }
        size_t fr = 0, all = 0;
        if (on && cudaMemGetInfo(&fr, &all) == cudaSuccess &&
            (size_t)tot * sizeof(double2) <= fr / 4 && dalloc(&p->d_urec, (size_t)tot) == SWR_OK &&
            dalloc(&p->d_rec_base, (size_t)p->N) == SWR_OK &&
            cudaMemcpy(p->d_rec_base, base.data(), sizeof(long long) * p->N,
                       cudaMemcpyHostToDevice) == cudaSuccess) {
            p->superpose = true;
            p->rec_base = base;
        } else {
            cudaGetLastError();
            cudaFree(p->d_urec);
            cudaFree(p->d_rec_base);
            p->d_urec = nullptr;
            p->d_rec_base = nullptr;
        }
    }
    if (!st) {
        auto vb = build_systems(p, true);
        p->nsys_build = (int)vb.size();
        for (size_t k = 0; k < vb.size(); ++k) {
            const long long w = (long long)p->n[vb[k].sub] * vb[k].nt;
            p->work_build += w;
            if ((int)k >= p->N) p->work_build_imp += w;
        }
        for (const InstInfo& I : p->inst)
            for (int j = 0; j < I.N; ++j) p->work_R += (long long)p->n[I.sub0 + j] * I.nt;
        st = upload_systems(&p->d_sys_build, vb, p);
    }
    const bool force_long = p->tune.long_march >= 1;   // the grid-wide march for any V(x) plan
    if (!st && (force_long || chunks_for(p->nmax, 16) + 1 > 16 * march_tmax(MK_STATIC, 16))) {
        // a subdomain longer than one cluster can hold (16 CTAs x 256 chunks of 16 nodes):
        // the grid-wide march, V(x) and single instances only
        if (d->vkind != SWR_V_STATIC || p->batched) {
            st = SWR_ERR_UNSUPPORTED;
        } else {
            p->long_march = true;
            p->long_bytes = swr_long_scratch_bytes(std::max(p->nsys_build, p->N), 16,
                                                   chunks_for(p->nmax, 16));
            st = dalloc(reinterpret_cast<char**>(&p->d_long), p->long_bytes);
        }
    }
    if (!st && d->tc >= SWR_TC_S03) {
        // per-end kernels of the higher-order conditions (formed from V at every build)
        const size_t ne = (size_t)2 * p->N;
        st = dalloc(&p->d_kap, ne * (p->nt + 1));
        if (!st) st = dalloc(&p->d_kout, ne * (p->nt + 1));
        if (!st) st = dalloc(&p->d_rho, ne);
    }
    if (!st && d->tc >= SWR_TC_S02) {
        // beta_s = (-1)^s alpha_s, alpha_{2k} = alpha_{2k+1} = prod_{i<=k} (2i-1)/(2i):
        // the coefficients of sqrt((1-z)/(1+z)) (Section 2.2)
        std::vector<double> beta(p->nt + 1);
        double alpha = 1.0;
        for (int k = 0; k <= p->nt; ++k) {
            if (k > 0 && k % 2 == 0) alpha *= (double)(k - 1) / (double)k;
            beta[k] = (k % 2 == 0) ? alpha : -alpha;
        }
        st = dalloc(&p->d_beta, p->nt + 1);
        if (!st && cudaMemcpy(p->d_beta, beta.data(), sizeof(double) * (p->nt + 1),
                              cudaMemcpyHostToDevice) != cudaSuccess)
            st = SWR_ERR_CUDA;
        if (!st)
            st = dalloc(&p->d_s02hist, (size_t)std::max(p->nsys_build, p->N) * 2 * (p->nt + 1));
    }
    if (!st) st = dalloc(&p->d_gconv, nb);
    if (!st && p->batched) {
        // instance tables of the interface kernels, and the instance groups that one
        // cooperative launch of the causal substitution can hold
        std::vector<int> bi(p->nblk), ii(p->nif);
        for (int i = 0; i < p->ninst; ++i) {
            const InstInfo& I = p->inst[i];
            for (int b = 0; b < 2 * I.N - 2; ++b) bi[I.blk0 + b] = i;
            for (int k = 0; k < I.N - 1; ++k) ii[I.if0 + k] = i;
        }
        st = dalloc(&p->d_inst, p->ninst);
        if (!st) st = dalloc(&p->d_blk_inst, p->nblk);
        if (!st) st = dalloc(&p->d_if_inst, p->nif);
        if (!st && (cudaMemcpy(p->d_inst, p->inst.data(), sizeof(InstInfo) * p->ninst,
                               cudaMemcpyHostToDevice) ||
                    cudaMemcpy(p->d_blk_inst, bi.data(), sizeof(int) * p->nblk,
                               cudaMemcpyHostToDevice) ||
                    cudaMemcpy(p->d_if_inst, ii.data(), sizeof(int) * p->nif,
                               cudaMemcpyHostToDevice)))
            st = SWR_ERR_CUDA;
        const int cap = swr_causal_capacity(p->nt);
        int k0 = 0, cnt = 0;
        for (int i = 0; i < p->ninst && !st; ++i) {
            const int ni = p->inst[i].N - 1;
            if (ni > cap) st = SWR_ERR_UNSUPPORTED;
            if (cnt + ni > cap) {
                p->causal_groups.push_back({k0, cnt});
                k0 += cnt;
                cnt = 0;
            }
            cnt += ni;
        }
        if (cnt > 0) p->causal_groups.push_back({k0, cnt});
    }
    if (!st) st = upload_systems(&p->d_sys_R, apply_systems(p, 0), p);
    if (!st) st = upload_systems(&p->d_sys_final, apply_systems(p, SYS_WRITE_UT | SYS_TRACE), p);
    if (!st) {
        for (auto& e : p->ev)
            if (cudaEventCreate(&e) != cudaSuccess) st = SWR_ERR_CUDA;
        for (auto& e : p->pev)
            if (!st && cudaEventCreate(&e) != cudaSuccess) st = SWR_ERR_CUDA;
    }
    if (st) {
        swr_destroy(p);
        return st;
    }
    *out = p;
    return SWR_OK;
}

swr_status swr_plan(const swr_desc* d, swr_plan_t* out, void* stream) {
    return plan_create(d, 1, nullptr, out, stream);
}

swr_status swr_plan_ex(const swr_desc* d, const swr_tuning* tuning, swr_plan_t* out,
                       void* stream) {
    return plan_create(d, 1, tuning, out, stream);
}

swr_status swr_plan_batch(const swr_desc* descs, int32_t count, swr_plan_t* out, void* stream) {
    return plan_create(descs, count, nullptr, out, stream);
}

swr_status swr_plan_batch_ex(const swr_desc* descs, int32_t count, const swr_tuning* tuning,
                             swr_plan_t* out, void* stream) {
    return plan_create(descs, count, tuning, out, stream);
}

void swr_tuning_defaults(swr_tuning* t) {
    if (t) *t = swr_tuning{};
}

// Everything a build does after the inputs are in place and the first build's
// tuning is done: assembly, factorisations, the d / first-column marches and
// the preconditioner's operator.  Stream work only (no host synchronisation),
// so that it can be captured into a CUDA graph.
static swr_status build_body(swr_plan_t p, bool do_assemble) {
    cudaStream_t s = p->s;
    const size_t nb = (size_t)p->nb;
    swr_status st = SWR_OK;
    if (do_assemble && (st = assemble(p, p->d_V, p->d_dg, p->d_od))) return st;
    if (p->d.vkind == SWR_V_TIME) {
        // chunk tables for the per-step refactorising march (the factors of the
        // t = 0 matrix computed alongside are not used)
        const int kt = march_kind(p, false);
        const int Lt = march_config(p, p->N, kt).L;
        if (kt == MK_TSTAT)   // every step's matrix, W = (V(t_{n-1}) + V(t_n)) / 2
            st = factor_steps_for(p, p->fsL[lidx(Lt)], Lt, p->nt);
        else
            st = factor_for(p, p->fsL[lidx(Lt)], Lt, p->d_V, p->d_dg, p->d_od);
        if (st) return st;
        CK(cudaMemsetAsync(p->d_iface, 0, sizeof(double2) * (nb + (size_t)p->ncols), s));
        // d = R 0 (Section 4.1; valid for V(t,x)): the first N systems of the build list
        st = run_march(p, false, p->d_sys_build, p->N, nullptr, p->d_iface, nullptr, nullptr,
                       p->d_u0, p->work_R);
        if (st) return st;
    } else if (p->d.vkind == SWR_V_NONLINEAR) {
        // constant matrix (2i/dt) M - S + M_{V0} - B: factor once (Eq. AvMNL)
        const int La = march_config(p, p->N, MK_NL).L;
        if ((st = factor_for(p, p->fsL[lidx(La)], La, p->d_V, p->d_dg, p->d_od))) return st;
    } else {
        // factorisations for the chunk lengths the marches of this plan will use
        const int Lb = march_config(p, p->nsys_build).L, La = march_config(p, p->N).L;
        if ((st = factor_for(p, p->fsL[lidx(Lb)], Lb, p->d_V, p->d_dg, p->d_od))) return st;
        if (La != Lb && (st = factor_for(p, p->fsL[lidx(La)], La, p->d_V, p->d_dg, p->d_od)))
            return st;
        CK(cudaMemsetAsync(p->d_iface, 0, sizeof(double2) * (nb + (size_t)p->ncols), s));
        // Algorithm 3, step 1: d and the first columns, 3 marches per interior subdomain
        st = run_march(p, false, p->d_sys_build, p->nsys_build, nullptr, p->d_iface, nullptr,
                       nullptr, p->d_u0, p->work_build);
        if (st) return st;
        const double2* cols = p->d_iface + nb;
        LK(p_lag0(p, cols, p->d_lag0));
        if (p->d_hspec) LK(swr_launch_hist_spectra(p->N, p->nt, cols, p->d_hspec, s));
        if (p->fftM)
            LK(swr_launch_col_spectra(p->N, p->nt, cols, p->d_spec, p->fftM, p->d_W, s,
                                      p->batched ? p->d_inst : nullptr, p->ninst));
        if (p->causal_H > 0)
            LK(swr_launch_lag0_window(p->N, p->nt, cols, p->d_lag0, p->d_Gw, p->causal_H, s,
                                      p->batched ? p->d_inst : nullptr, p->d_if_inst, p->nif));
    }
    if (p->d.precond == SWR_PC_ZERO_POTENTIAL || p->d.precond == SWR_PC_MEAN_POTENTIAL) {
        const double* Vp = nullptr;                       // V = 0 (Section 5)
        if (p->d.precond == SWR_PC_MEAN_POTENTIAL) {
            LK(swr_launch_row_mean(p->d_V, p->d.vkind == SWR_V_TIME ? p->nt + 1 : 1, p->nx,
                                   p->d_Vbar, s));
            Vp = p->d_Vbar;
        }
        if ((st = assemble(p, Vp, p->d_dg0, p->d_od0))) return st;
        const int L0 = march_config(p, p->nsys_build - p->N).L;
        if ((st = factor_for(p, p->fs0L[lidx(L0)], L0, Vp, p->d_dg0, p->d_od0))) return st;
        CK(cudaMemsetAsync(p->d_iface0, 0, sizeof(double2) * (nb + (size_t)p->ncols), s));
        // impulse marches only (the first N systems of the build list are the d marches)
        st = run_march(p, true, p->d_sys_build + p->N, p->nsys_build - p->N, nullptr,
                       p->d_iface0, nullptr, nullptr, p->d_u0, p->work_build_imp);
        if (st) return st;
        LK(p_lag0(p, p->d_iface0 + nb, p->d_lag0_0));
        if (p->d_hspec0)
            LK(swr_launch_hist_spectra(p->N, p->nt, p->d_iface0 + nb, p->d_hspec0, s));
        if (p->fftM)
            LK(swr_launch_col_spectra(p->N, p->nt, p->d_iface0 + nb, p->d_spec0, p->fftM,
                                      p->d_W, s, p->batched ? p->d_inst : nullptr, p->ninst));
        p->have_L0 = true;
    }
    return SWR_OK;
}

swr_status swr_build_interface(swr_plan_t p, const double* V, const double* u0) {
    t_debug = p ? p->tune.debug : 0;
    NvtxRange nvtx_range("swr_build_interface");
    if (!p || !V || !u0) return SWR_ERR_ARG;
    p->nl_rec = false;
    cudaStream_t s = p->s;
    const size_t nb = (size_t)p->nb;
    const size_t nV = (p->d.vkind == SWR_V_TIME) ? (size_t)(p->nt + 1) * p->nx : p->nx;
    CK(cudaEventRecord(p->ev[0], s));
    CK(cudaMemsetAsync(p->d_status, 0, sizeof(int), s));
    CK(cudaMemcpyAsync(p->d_V, V, sizeof(double) * nV, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(p->d_u0, u0, sizeof(double2) * p->nx, cudaMemcpyDeviceToDevice, s));
    swr_status st = SWR_OK;
    if (p->tune.graph < 0) p->use_graph = false;
    const bool direct = !p->built || !p->use_graph;
    if (direct && (st = assemble(p, p->d_V, p->d_dg, p->d_od))) return st;
    if (p->d.vkind == SWR_V_TIME && p->tdep_pre < 0) {
        // per-step factorisations need nt copies of the factors (about 110 bytes
        // per node and step); take them while they use at most half the free memory
        bool on = p->nt >= 2;
        if (p->tune.tdep_precomp < 0) on = false;
        // the refactorising march has no S_0^2 history terms
        if (p->d.tc == SWR_TC_S02) on = p->nt >= 2;
        if (on) {
            size_t fr = 0, tot = 0;
            CK(cudaMemGetInfo(&fr, &tot));
            const size_t need =
                (size_t)p->nt * swr_factor_step_bytes(p->N, 4, chunks_for(p->nmax, 4));
            on = need <= fr / 2;
        }
        p->tdep_pre = on ? 1 : 0;
    }
    if (p->autotune && !p->built) {
        // first build: measure the launch shapes of every march this plan makes
        const int k = march_kind(p, false);
        if ((st = tune_march(p, k, false, p->d_sys_R, p->N, p->d_iface, p->d_V, p->d_dg, p->d_od)))
            return st;
        if (k == MK_STATIC &&
            (st = tune_march(p, k, false, p->d_sys_build, p->nsys_build, p->d_iface, p->d_V,
                             p->d_dg, p->d_od)))
            return st;
        if (p->d.precond == SWR_PC_ZERO_POTENTIAL || p->d.precond == SWR_PC_MEAN_POTENTIAL) {
            const double* Vp = nullptr;
            if (p->d.precond == SWR_PC_MEAN_POTENTIAL) {
                LK(swr_launch_row_mean(p->d_V, p->d.vkind == SWR_V_TIME ? p->nt + 1 : 1, p->nx,
                                       p->d_Vbar, s));
                Vp = p->d_Vbar;
            }
            if ((st = assemble(p, Vp, p->d_dg0, p->d_od0))) return st;
            if ((st = tune_march(p, MK_STATIC, true, p->d_sys_build + p->N, p->nsys_build - p->N,
                                 p->d_iface, Vp, p->d_dg0, p->d_od0)))
                return st;
        }
        // the probes wrote into d_iface; the build below starts the clock again
        CK(cudaMemsetAsync(p->d_iface, 0, sizeof(double2) * (nb + (size_t)p->ncols), s));
        CK(cudaEventRecord(p->ev[0], s));
    }
    if (!p->built || !p->use_graph) {
        st = build_body(p, false);
        if (st) return st;
    } else if (p->gexec) {
        // replay the captured build
        CK(cudaGraphLaunch(p->gexec, s));
        g_launches += p->graph_kernels;
        p->graph_pending = true;
    } else {
        // second build: capture it, then launch the graph (later builds replay it)
        for (auto& e : p->gev)
            if (!e && cudaEventCreate(&e) != cudaSuccess) p->use_graph = false;
        bool ok = p->use_graph;
        const long long k0 = g_launches.load();
        if (ok) ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) == cudaSuccess;
        if (ok) {
            p->capturing = true;
            p->gcount = 0;
            st = build_body(p, true);
            p->capturing = false;
            cudaGraph_t gr = nullptr;
            const bool ended = cudaStreamEndCapture(s, &gr) == cudaSuccess && gr;
            if (st || !ended) {
                if (gr) cudaGraphDestroy(gr);
                cudaGetLastError();
                ok = false;
            } else if (cudaGraphInstantiate(&p->gexec, gr, 0) != cudaSuccess) {
                cudaGraphDestroy(gr);
                cudaGetLastError();
                p->gexec = nullptr;
                ok = false;
            } else {
                p->graph = gr;
                p->graph_kernels = g_launches.load() - k0;
            }
        }
        g_launches -= g_launches.load() - k0;   // captured launches ran nowhere yet
        if (ok) {
            CK(cudaGraphLaunch(p->gexec, s));
            g_launches += p->graph_kernels;
            p->graph_pending = true;
        } else {
            // capture is not available here: build directly from now on
            p->use_graph = false;
            p->gcount = 0;
            if ((st = build_body(p, true))) return st;
        }
    }
    CK(cudaEventRecord(p->ev[1], s));
    st = read_status(p);
    if (st) return st;
    if (!p->built && p->auto_sweeps) {
        // The substitution's same-step coupling of neighbouring interfaces is the
        // corner entries cB_k = X^{k+1,2}[0], cD_k = X^{k,3}[0] of the subdomain
        // inverses, of relative size f = max_k max(|cB_k|, |cD_k|) ||D_k^{-1}||_inf.
        // The window form resolves it to f^{H+1}: H is the smallest width with
        // f^{H+1} <= 1e-16 (then P^{-1} is (I - L)^{-1} to rounding and GMRES needs
        // one iteration); f^9 > 1e-16 (narrow subdomains) takes one block-Jacobi
        // sweep instead, f <= 1e-16 neither.
        double f = 0.0;
        for (const InstInfo& I : p->inst) {
            if (I.N < 3) continue;
            std::vector<double2> c0((size_t)4 * I.N);
            CK(cudaMemcpy2DAsync(c0.data(), sizeof(double2), p->d_iface + p->nb + I.coff,
                                 sizeof(double2) * I.nt, sizeof(double2), (size_t)4 * I.N,
                                 cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int k = 0; k + 1 < I.N; ++k) {
                const double2 a = c0[4 * (k + 1) + 0], b = c0[4 * k + 3];
                const double2 det = make_double2(1.0 - (a.x * b.x - a.y * b.y),
                                                 -(a.x * b.y + a.y * b.x));
                const double na = std::hypot(a.x, a.y), nbv = std::hypot(b.x, b.y);
                const double dinv = std::max(1.0 + na, 1.0 + nbv) / std::hypot(det.x, det.y);
                double c = 0.0;
                if (k + 2 < I.N) c = std::max(c, std::hypot(c0[4 * (k + 1) + 1].x, c0[4 * (k + 1) + 1].y));
                if (k >= 1) c = std::max(c, std::hypot(c0[4 * k + 2].x, c0[4 * k + 2].y));
                f = std::max(f, c * dinv);
            }
        }
        int H = 0;
        if (f > 1e-16) {
            H = 1;
            while (H <= 8 && std::pow(f, H + 1) > 1e-16) ++H;
        }
        p->causal_sweeps = 0;
        p->causal_H = 0;
        if (H > 8) {
            p->causal_sweeps = 1;
        } else if (H >= 1) {
            if (!p->d_Gw && (st = dalloc(&p->d_Gw, (size_t)p->nif * (2 * 8 + 1) * 4))) return st;
            if (!p->d_Pwin && (st = dalloc(&p->d_Pwin, (size_t)p->nb))) return st;
            p->causal_H = H;
            LK(swr_launch_lag0_window(p->N, p->nt, p->d_iface + p->nb, p->d_lag0, p->d_Gw, H, s,
                                      p->batched ? p->d_inst : nullptr, p->d_if_inst, p->nif));
            CK(cudaStreamSynchronize(s));
        }
    }
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, p->ev[0], p->ev[1]));
    p->t_build_ms = ms;
    p->built = true;
    return SWR_OK;
}

swr_status swr_solve(swr_plan_t p, double* g_, int32_t g_is_initial, double* uT_, swr_info* info) {
    t_debug = p ? p->tune.debug : 0;
    NvtxRange nvtx_range("swr_solve");
    if (!p) return SWR_ERR_ARG;
    if (!p->built) return SWR_ERR_STATE;
    p->nl_rec = false;
    cudaStream_t s = p->s;
    swr_info loc{};
    double2* g = g_ ? reinterpret_cast<double2*>(g_) : p->d_gtmp2;
    const bool init = g_ && g_is_initial;
    CK(cudaMemsetAsync(p->d_status, 0, sizeof(int), s));
    CK(cudaEventRecord(p->ev[1], s));
    swr_status st;
    if (p->d.vkind == SWR_V_NONLINEAR)
        st = nl_fixed_point(p, g, init, &loc);
    else if (p->d.solver == SWR_SOLVER_CAUSAL)
        st = causal_direct(p, g, init, &loc);
    else if (p->d.solver == SWR_SOLVER_BICGSTAB)
        st = bicgstab(p, p->d_iface, p->d.tol_abs, g, init, &loc);
    else if (p->d.solver == SWR_SOLVER_GMRES)
        st = gmres(p, p->d_iface, p->d.tol_abs, g, init, &loc);
    else
        st = fixed_point(p, g, init, p->d.solver == SWR_SOLVER_CLASSICAL, &loc);
    if (st != SWR_OK && st != SWR_ERR_NOT_CONVERGED) return st;
    p->solved = false;
    CK(cudaMemcpyAsync(p->d_gconv, g, sizeof(double2) * (size_t)p->nb,
                       cudaMemcpyDeviceToDevice, s));
    CK(cudaEventRecord(p->ev[2], s));
    double2* uT = uT_ ? reinterpret_cast<double2*>(uT_) : nullptr;
    if (p->superpose) {
        // u(T) from the build marches' states (the march is linear and time invariant);
        // the interface mismatch from w = L g + d and g
        if (uT)
            LK(swr_launch_superpose(p->d_urec, p->d_rec_base, p->d_sys_final, p->N, p->d_n,
                                    p->d_goff, p->d_tc, p->nmax, g, uT, s));
        if (p_toeplitz(p, p->d_iface + p->nb, g, p->d_iface, p->d_gtmp, 1))
            return launch_fail("toeplitz", __LINE__);
        if (p->d.tc == SWR_TC_ROBIN) {
            const double as = std::hypot(p->two_sigma.x, p->two_sigma.y);
            LK(swr_launch_jump_res(p->d_gtmp, g, p->N, p->nt, as > 0.0 ? 1.0 / as : 0.0,
                                   p->d_scal, s, p->batched ? p->d_inst : nullptr, p->d_if_inst,
                                   p->nif));
        } else {   // the mismatch trace through the flux update's convolution
            LK(swr_launch_jump_conv(p->d_gtmp, g, p->N, p->nt, p->d_kout, p->nt + 1, p->c2,
                                    p->d_beta, p->d_scal, s, p->batched ? p->d_inst : nullptr,
                                    p->d_if_inst, p->nif));
        }
    } else {
        // final march (last step of Algorithms 1-3).  Nonlinear plans with Robin or Neumann
        // ends also record v_n of every step when the record (nt x nx values) takes at most
        // an eighth of the free device memory: that is the forward trajectory the gradient
        // is linearised about (the converged SWR solution is the monodomain one), so
        // swr_adjoint with one checkpoint segment skips its forward re-march.
        double2* vrec = nullptr;
        if (st == SWR_OK && p->d.vkind == SWR_V_NONLINEAR && p->d.tc < SWR_TC_S02 &&
            !p->batched && !p->long_march) {
            if (p->adj_K != p->nt) {
                size_t fr = 0, tot = 0;
                const size_t need = ((size_t)p->nt + 1) * (size_t)p->nx * sizeof(double2);
                if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && need <= fr / 8) {
                    cudaFree(p->d_ckpt);
                    cudaFree(p->d_slab);
                    p->d_ckpt = p->d_slab = nullptr;
                    p->adj_K = 0;
                    swr_status sa = dalloc(&p->d_ckpt, (size_t)p->nx);
                    if (!sa) sa = dalloc(&p->d_slab, (size_t)p->nt * p->nx);
                    if (sa) {   // no record: the adjoint re-marches the forward scheme
                        cudaFree(p->d_ckpt);
                        cudaFree(p->d_slab);
                        p->d_ckpt = p->d_slab = nullptr;
                    } else {
                        p->adj_K = p->nt;
                    }
                }
                cudaGetLastError();
            }
            if (p->adj_K == p->nt) vrec = p->d_slab;
        }
        swr_status st2 = run_march(p, false, p->d_sys_final, p->N, g, p->d_gtmp, uT, p->d_trace,
                                   p->d_u0, p->work_R, vrec);
        if (st2) return st2;
        p->nl_rec = (vrec != nullptr);
        LK(p_jump(p));
    }
    CK(cudaEventRecord(p->ev[3], s));
    double jump = 0.0;
    CK(cudaMemcpyAsync(&jump, p->d_scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    swr_status st3 = read_status(p);
    if (st3) return st3;
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, p->ev[1], p->ev[2]);
    cudaEventElapsedTime(&b, p->ev[2], p->ev[3]);
    loc.interface_jump = jump;
    loc.t_build_ms = p->t_build_ms;
    loc.t_solve_ms = a;
    loc.t_final_ms = b;
    long long sweeps = (p->superpose ? 0 : 1) +
                       (p->d.solver == SWR_SOLVER_CLASSICAL ? loc.iterations : 0);
    loc.march_point_steps = sweeps * p->work_R;   // nodes x steps of one pass over all instances
    if (info) *info = loc;
    p->solved = (st == SWR_OK);
    return st;
}

swr_status swr_apply_R(swr_plan_t p, const double* g_in, double* g_out) {
    t_debug = p ? p->tune.debug : 0;
    NvtxRange nvtx_range("swr_apply_R");
    if (!p || !g_in || !g_out || g_in == g_out) return SWR_ERR_ARG;
    if (!p->built) return SWR_ERR_STATE;
    CK(cudaMemsetAsync(g_out, 0, sizeof(double2) * (size_t)p->nb, p->s));
    swr_status st = run_march(p, false, p->d_sys_R, p->N, reinterpret_cast<const double2*>(g_in),
                              reinterpret_cast<double2*>(g_out), nullptr, nullptr, p->d_u0,
                              p->work_R);
    if (st) return st;
    return read_status(p);
}

swr_status swr_apply_interface(swr_plan_t p, const double* x, double* y) {
    t_debug = p ? p->tune.debug : 0;
    NvtxRange nvtx_range("swr_apply_interface");
    if (!p || !x || !y || x == y) return SWR_ERR_ARG;
    if (!p->built) return SWR_ERR_STATE;
    if (p->d.vkind != SWR_V_STATIC) return SWR_ERR_UNSUPPORTED;
    if (p_toeplitz(p, p->d_iface + p->nb, reinterpret_cast<const double2*>(x), nullptr,
                   reinterpret_cast<double2*>(y), 0))
        return SWR_ERR_UNSUPPORTED;
    CK(cudaStreamSynchronize(p->s));
    return SWR_OK;
}

swr_status swr_get_interface(swr_plan_t p, double* d, double* cols) {
    t_debug = p ? p->tune.debug : 0;
    if (!p) return SWR_ERR_ARG;
    if (!p->built) return SWR_ERR_STATE;
    const size_t nb = (size_t)p->nb;
    if (d) CK(cudaMemcpyAsync(d, p->d_iface, sizeof(double2) * nb, cudaMemcpyDeviceToDevice, p->s));
    if (cols)
        CK(cudaMemcpyAsync(cols, p->d_iface + nb, sizeof(double2) * p->ncols,
                           cudaMemcpyDeviceToDevice, p->s));
    CK(cudaStreamSynchronize(p->s));
    return SWR_OK;
}

swr_status swr_apply_precond(swr_plan_t p, const double* y, double* x) {
    t_debug = p ? p->tune.debug : 0;
    NvtxRange nvtx_range("swr_apply_precond");
    if (!p || !y || !x || x == y) return SWR_ERR_ARG;
    if (!p->built) return SWR_ERR_STATE;
    if (!has_precond(p)) return SWR_ERR_STATE;
    // the status word reports this call's device errors (a bounded wait that gave up)
    CK(cudaMemsetAsync(p->d_status, 0, sizeof(int), p->s));
    swr_status st = apply_M(p, reinterpret_cast<const double2*>(y), reinterpret_cast<double2*>(x));
    if (st) return st;
    return read_status(p);
}

swr_status swr_get_stats(swr_plan_t p, swr_stats* out, int32_t reset) {
    t_debug = p ? p->tune.debug : 0;
    if (!p) return SWR_ERR_ARG;
    CK(cudaStreamSynchronize(p->s));
    prof_flush(p);
    if (out) {
        *out = p->stats;
        out->march_variant = p->built ? march_kind(p, false) : -1;
        out->march_factor_bytes_per_step = 0;
        if (out->march_variant == MK_TSTAT) {
            const FactorSet& fs = p->fsL[lidx(march_config(p, p->N, MK_TSTAT).L)];
            out->march_factor_bytes_per_step =
                (int64_t)sizeof(double2) * (fs.fstride + fs.sstride + fs.pstride);
        }
        unsigned long long pit = 0;
        CK(cudaMemcpy(&pit, p->d_pit, sizeof(pit), cudaMemcpyDeviceToHost));
        out->march_point_iterations = (int64_t)pit;
        out->superposed = p->superpose ? 1 : 0;
        out->toeplitz_fft_length = p->fftM;
        out->causal_sweeps = p->causal_sweeps;
        out->causal_window = p->causal_H;
    }
    if (reset) {
        p->stats = swr_stats{};
        CK(cudaMemsetAsync(p->d_pit, 0, sizeof(unsigned long long), p->s));
        CK(cudaStreamSynchronize(p->s));
    }
    return SWR_OK;
}

swr_status swr_misfit(swr_plan_t p, const double* uT_, const double* target_, double* ubar_,
                      double* J) {
    t_debug = p ? p->tune.debug : 0;
    if (!p || !uT_ || !target_ || !J) return SWR_ERR_ARG;
    if (!p->d_part && dalloc(&p->d_part, 160)) return SWR_ERR_NOMEM;
    LK(swr_launch_misfit(reinterpret_cast<const double2*>(uT_),
                         reinterpret_cast<const double2*>(target_), p->nx, p->h,
                         reinterpret_cast<double2*>(ubar_), p->d_part, p->d_part + 150, p->s));
    CK(cudaMemcpyAsync(J, p->d_part + 150, sizeof(double), cudaMemcpyDeviceToHost, p->s));
    CK(cudaStreamSynchronize(p->s));
    return SWR_OK;
}

// Gradient of J(V) through the converged SWR solution (which is the monodomain
// Crank-Nicolson solution u_N).  With the M-weighted cotangent ubar (dJ =
// Re(ubar^H M du_N)), the discrete adjoint of u_n = 2 A^{-1} B u_{n-1} - u_{n-1}
// (A = (2i/dt) M - S + M_V complex symmetric, B = (2i/dt) M) conjugated and
// scaled, z_n = B^{-1} conj(lambda_n), obeys the same map backwards:
//     z_N = (dt / 2i) conj(ubar),   z_{n-1} = 2 A^{-1} B z_n - z_n,
// so the adjoint is an SWR solve of the same interface problem (same L, same
// preconditioner) from the initial state z_N, marched as y_m = z_{N-m}, and
//     dJ/dV_k = -2 Re sum_n (v^y_{N-n+1})^T (dM_V/dV_k) v_n,
// v^y_m, v_n the midpoint values of the two marches.  The forward v_n are
// recomputed segment by segment from checkpoints of u every K steps (the
// segment is recorded, then the adjoint march over the mirrored steps reads it).
swr_status swr_adjoint(swr_plan_t p, const double* ubar_, double* dJdV_, int32_t ckpt_every) {
    t_debug = p ? p->tune.debug : 0;
    NvtxRange nvtx_range("swr_adjoint");
    if (!p || !ubar_ || !dJdV_) return SWR_ERR_ARG;
    if (!p->built || !p->solved) return SWR_ERR_STATE;
    // the nonlinear gradient is taken of the monodomain scheme (any transmission
    // condition and solver); the linear one runs the adjoint interface solve
    const bool nl = (p->d.vkind == SWR_V_NONLINEAR);
    cudaStream_t s = p->s;
    const int nt = p->nt, nx = p->nx, N = p->N;
    const bool tdep = (p->d.vkind == SWR_V_TIME);
    if (p->batched || p->long_march || (!nl && p->d.tc > SWR_TC_S02)) return SWR_ERR_UNSUPPORTED;
    // V(t,x): the adjoint walks every step's factors backwards, so they must be stored
    // (the streamed variant) with chunks short enough for the gradient march (L <= 8)
    if (tdep && (march_kind(p, false) != MK_TSTAT || march_config(p, N, MK_TSTAT).L > 8))
        return SWR_ERR_UNSUPPORTED;
    const size_t nb = (size_t)p->nblk * nt;
    // checkpoint interval: the caller's, else every step recorded (one segment, no
    // re-march of the forward) when the record of nt steps takes at most an eighth of
    // the free device memory, else 50
    int Kdef = 50;
    if (ckpt_every <= 0 && p->adj_K == nt) {
        Kdef = nt;   // the record of nt steps is already allocated (and may hold the solve's)
    } else if (ckpt_every <= 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess &&
            (size_t)nt * (size_t)nx * sizeof(double2) <= fr / 8)
            Kdef = nt;
        cudaGetLastError();
    }
    const int K = std::max(1, std::min(ckpt_every > 0 ? ckpt_every : Kdef, nt));
    const int C = (nt + K - 1) / K;
    swr_status st = SWR_OK;
    if (p->adj_K != K) {
        p->nl_rec = false;
        cudaFree(p->d_ckpt);
        cudaFree(p->d_slab);
        p->d_ckpt = p->d_slab = nullptr;
        p->adj_K = 0;
        if ((st = dalloc(&p->d_ckpt, (size_t)C * nx))) return st;
        if ((st = dalloc(&p->d_slab, (size_t)K * nx))) return st;
        p->adj_K = K;
    }
    const bool s02 = (p->d.tc == SWR_TC_S02);
    if (s02 && !p->d_hseg) {
        // the segments' end traces over the whole time axis: forward, adjoint
        if ((st = dalloc(&p->d_hseg, (size_t)2 * N * 2 * (nt + 1)))) return st;
    }
    if (!p->d_ya) {
        if ((st = dalloc(&p->d_ya, nx)) || (st = dalloc(&p->d_yb, nx)) ||
            (st = dalloc(&p->d_dy, nb)) || (st = dalloc(&p->d_gy, nb)) ||
            (st = dalloc(&p->d_gint, nx)) || (st = dalloc(&p->d_gl, nx)) ||
            (st = dalloc(&p->d_gr, nx)) ||
            (st = upload_systems(&p->d_sys_seg, apply_systems(p, SYS_WRITE_UT))))
            return st;
    }
    CK(cudaMemsetAsync(p->d_status, 0, sizeof(int), s));
    if (nl) {
        if ((st = mono_setup(p))) return st;
        CK(cudaMemcpyAsync(p->d_ckpt, p->d_u0, sizeof(double2) * nx, cudaMemcpyDeviceToDevice, s));
        for (int c = 1; c < C; ++c)
            if ((st = mono_nl_march(p, 0, p->d_ckpt + (size_t)(c - 1) * nx,
                                    p->d_ckpt + (size_t)c * nx, K)))
                return st;
        LK(swr_launch_adj_seed(reinterpret_cast<const double2*>(ubar_), 0.5 * p->d.dt, nx,
                               p->d_ya, s));
        CK(cudaMemsetAsync(p->d_gint, 0, sizeof(double) * nx, s));
        CK(cudaMemsetAsync(p->d_gl, 0, sizeof(double) * nx, s));
        CK(cudaMemsetAsync(p->d_gr, 0, sizeof(double) * nx, s));
        double2* ycur = p->d_ya;
        double2* ynext = p->d_yb;
        // one segment with the solve's record of v_n: the adjoint march alone
        const bool rec = (C == 1 && p->nl_rec);
        for (int c = C - 1; c >= 0; --c) {
            const int Kc = std::min(K, nt - c * K);
            if ((!rec && (st = mono_nl_march(p, 1, p->d_ckpt + (size_t)c * nx, nullptr, Kc))) ||
                (st = mono_nl_march(p, 2, ycur, ynext, Kc)))
                return st;
            std::swap(ycur, ynext);
        }
        LK(swr_launch_grad_combine(p->d_gint, p->d_gl, p->d_gr, nx, dJdV_, s));
        CK(cudaStreamSynchronize(s));
        return read_status(p);
    }
    if (tdep) {
        // V(t,x): W_n changes every step, so the adjoint march (the forward map run
        // backwards, z_{n-1} = 2 A_n^{-1} B z_n - z_n) takes the factors of A_N, ...,
        // A_1 in that order: its SWR problem is the forward one with the time axis
        // reversed, solved matrix-free like the forward one (Algorithm 2) with the same
        // time-invariant preconditioner.  Each adjoint step's potential form is
        // dJ/dW_n, which goes to the rows n and n-1 of dJ/dV (W_n = (V_n + V_{n-1})/2).
        const MarchCfg cfg0 = march_config(p, N, MK_TSTAT);          // forward segments
        const MarchCfg cfga = march_config(p, N, MK_ADJ, cfg0.L);    // record / gradient
        auto segT = [&](const MarchCfg& cfg, int mode, const double2* gin, int t0, int nrun,
                        int fstep0, const double2* u0, double2* uT,
                        const double2* vfwd) -> swr_status {
            SegArgs sa;
            sa.mode = mode;
            sa.t0 = t0;
            sa.gstride = nt;
            sa.vrec = p->d_slab;
            sa.vfwd = vfwd;
            sa.gint = p->d_gint;
            sa.gl = p->d_gl;
            sa.gr = p->d_gr;
            sa.fstep0 = fstep0;
            if (s02) {
                sa.hist = p->d_hseg + (mode == 2 ? (size_t)N * 2 * (nt + 1) : 0);
                sa.ht0 = t0;
            }
            const int pi = prof_begin(p, 0, (long long)nx * nrun);
            const int rc = launch_cfg(p, cfg, MK_TSTAT, false, p->d_sys_seg, N, gin, nullptr, uT,
                                      nullptr, u0, nrun, sa);
            prof_end(p, pi);
            if (rc == -2) return SWR_ERR_UNSUPPORTED;
            if (rc) return launch_fail("adjoint segment march (time-dependent)", __LINE__);
            return SWR_OK;
        };
        // 1. forward checkpoints
        CK(cudaMemcpyAsync(p->d_ckpt, p->d_u0, sizeof(double2) * nx, cudaMemcpyDeviceToDevice, s));
        for (int c = 1; c < C; ++c)
            if ((st = segT(cfg0, 0, p->d_gconv, (c - 1) * K, K, (c - 1) * K,
                           p->d_ckpt + (size_t)(c - 1) * nx, p->d_ckpt + (size_t)c * nx,
                           nullptr)))
                return st;
        // 2. the adjoint's time-reversed interface problem: d_y = R_rev 0, then
        //    (I - L_rev) g_y = d_y by the plan's GMRES, matrix-free
        LK(swr_launch_adj_seed(reinterpret_cast<const double2*>(ubar_), 0.5 * p->d.dt, nx,
                               p->d_ya, s));
        CK(cudaMemsetAsync(p->d_dy, 0, sizeof(double2) * nb, s));
        p->cur_rev = 1;
        st = run_march(p, false, p->d_sys_build, N, nullptr, p->d_dy, nullptr, nullptr, p->d_ya,
                       p->work_R);
        double dn = 0.0, dny = 0.0;
        if (!st) st = norm2(p, p->d_iface, (long long)nb, &dn);
        if (!st) st = norm2(p, p->d_dy, (long long)nb, &dny);
        if (!st) {
            const double tol = (dn > 0.0) ? p->d.tol_abs * dny / dn : p->d.tol_abs;
            p->cur_u0 = p->d_ya;
            p->cur_d = p->d_dy;
            swr_info loc{};
            st = gmres(p, p->d_dy, tol, p->d_gy, false, &loc);
        }
        p->cur_rev = 0;
        p->cur_u0 = nullptr;
        p->cur_d = nullptr;
        if (st != SWR_OK) return st;
        // 3. segments from the last to the first: record the forward v of the segment,
        //    then one launch per adjoint step (its potential form is that step's
        //    dJ/dW_n), adding it into the rows of dJ/dV
        CK(cudaMemsetAsync(p->d_gint, 0, sizeof(double) * nx, s));
        CK(cudaMemsetAsync(p->d_gl, 0, sizeof(double) * nx, s));
        CK(cudaMemsetAsync(p->d_gr, 0, sizeof(double) * nx, s));
        CK(cudaMemsetAsync(dJdV_, 0, sizeof(double) * (size_t)(nt + 1) * nx, s));
        double2* ycur = p->d_ya;
        double2* ynext = p->d_yb;
        for (int c = C - 1; c >= 0; --c) {
            const int t0 = c * K, Kc = std::min(K, nt - t0);
            if ((st = segT(cfga, 1, p->d_gconv, t0, Kc, t0, p->d_ckpt + (size_t)c * nx, nullptr,
                           nullptr)))
                return st;
            for (int i = 0; i < Kc; ++i) {
                const int n = t0 + Kc - i;           // forward step of this adjoint step
                const int ta = nt - n;               // adjoint steps before it
                if ((st = segT(cfga, 2, p->d_gy, ta, 1, n - 1, ycur, ynext,
                               p->d_slab + (size_t)(Kc - 1 - i) * nx)))
                    return st;
                LK(swr_launch_grad_step_tdep(p->d_gint, p->d_gl, p->d_gr, nx, n, dJdV_, s));
                std::swap(ycur, ynext);
            }
        }
        CK(cudaStreamSynchronize(s));
        return read_status(p);
    }
    // launch shape of the segment marches (chunk length <= 8 for the gradient sums)
    if (p->autotune) {
        if ((st = tune_march(p, MK_ADJ, false, p->d_sys_R, N, p->d_dy, p->d_V, p->d_dg, p->d_od)))
            return st;
    }
    const MarchCfg cfg = march_config(p, N, MK_ADJ);
    if (p->fsL[lidx(cfg.L)].L != cfg.L &&
        (st = factor_for(p, p->fsL[lidx(cfg.L)], cfg.L, p->d_V, p->d_dg, p->d_od)))
        return st;
    auto seg = [&](int mode, const double2* gin, int t0, int nrun, const double2* u0,
                   double2* uT) -> swr_status {
        SegArgs sa;
        sa.mode = mode;
        sa.t0 = t0;
        sa.gstride = nt;
        if (s02) {   // forward traces for modes 0 and 1, the adjoint's for mode 2
            sa.hist = p->d_hseg + (mode == 2 ? (size_t)N * 2 * (nt + 1) : 0);
            sa.ht0 = t0;
        }
        sa.vrec = p->d_slab;
        sa.vfwd = p->d_slab;
        sa.gint = p->d_gint;
        sa.gl = p->d_gl;
        sa.gr = p->d_gr;
        const long long work = (long long)nx * nrun;
        const int pi = prof_begin(p, 0, work);
        const int rc = launch_cfg(p, cfg, MK_ADJ, false, p->d_sys_seg, N, gin, nullptr, uT,
                                  nullptr, u0, nrun, sa);
        prof_end(p, pi);
        if (rc) return launch_fail("adjoint segment march", __LINE__);
        return SWR_OK;
    };
    // 1. forward checkpoints: ckpt[c] = u after c K steps
    CK(cudaMemcpyAsync(p->d_ckpt, p->d_u0, sizeof(double2) * nx, cudaMemcpyDeviceToDevice, s));
    for (int c = 1; c < C; ++c)
        if ((st = seg(0, p->d_gconv, (c - 1) * K, K, p->d_ckpt + (size_t)(c - 1) * nx,
                      p->d_ckpt + (size_t)c * nx)))
            return st;
    // 2. adjoint initial state and its interface problem: d_y = R_y 0, (I - L) g_y = d_y
    LK(swr_launch_adj_seed(reinterpret_cast<const double2*>(ubar_), 0.5 * p->d.dt, nx, p->d_ya, s));
    CK(cudaMemsetAsync(p->d_dy, 0, sizeof(double2) * nb, s));
    if ((st = run_march(p, false, p->d_sys_build, N, nullptr, p->d_dy, nullptr, nullptr, p->d_ya,
                        p->work_R)))
        return st;
    double dn = 0.0, dny = 0.0;
    if ((st = norm2(p, p->d_iface, (long long)nb, &dn)) || (st = norm2(p, p->d_dy, (long long)nb, &dny)))
        return st;
    // the forward solve's accuracy relative to its right-hand side
    const double tol = (dn > 0.0) ? p->d.tol_abs * dny / dn : p->d.tol_abs;
    swr_info loc{};
    st = gmres(p, p->d_dy, tol, p->d_gy, false, &loc);
    if (st != SWR_OK) return st;
    // 3. segments from the last to the first: record the forward v, then march the
    //    adjoint over the mirrored steps and accumulate the potential form
    CK(cudaMemsetAsync(p->d_gint, 0, sizeof(double) * nx, s));
    CK(cudaMemsetAsync(p->d_gl, 0, sizeof(double) * nx, s));
    CK(cudaMemsetAsync(p->d_gr, 0, sizeof(double) * nx, s));
    double2* ycur = p->d_ya;
    double2* ynext = p->d_yb;
    for (int c = C - 1; c >= 0; --c) {
        const int t0 = c * K, Kc = std::min(K, nt - t0);
        if ((st = seg(1, p->d_gconv, t0, Kc, p->d_ckpt + (size_t)c * nx, nullptr))) return st;
        if ((st = seg(2, p->d_gy, nt - t0 - Kc, Kc, ycur, ynext))) return st;
        std::swap(ycur, ynext);
    }
    LK(swr_launch_grad_combine(p->d_gint, p->d_gl, p->d_gr, nx, dJdV_, s));
    CK(cudaStreamSynchronize(s));
    return read_status(p);
}

}  // extern "C"
