// swr_causal_solve_noalloc: the causal block forward substitution x = (I - L)^{-1} y
// for callers that cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc once it is running, for
// example a solver embedded in a host application that reserves all device
// memory up front with its own pool, or a latency-critical loop where the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable.
// Such callers own x, y and the Toeplitz first columns, but have nowhere to put
// the substitution's working arrays.  This entry point keeps them in a
// fixed-size array in the library's own device memory instead.
//
// The scratch is a file-scope __device__ array: every GPU that loads the
// library holds it (about 260 KB) until the process exits.  Host code must not
// hand the array's name to a kernel: on the host it is only a stand-in symbol.
// Its device address is looked up with cudaGetSymbolAddress once per device,
// with that device current, the first time the entry point runs there, and again
// only if the device's context has changed since (after a cudaDeviceReset the
// array lives at a new address in the new context).
#include <cuda.h>   // CUcontext / CUresult types of cuCtxGetId (found at run time)

#include <mutex>

#include "swr_internal.cuh"

namespace {

constexpr int kNoallocMaxSub = 1024;     // largest supported number of subdomains N
constexpr int kNoallocMaxDevices = 64;
constexpr size_t kLag0Elems = (size_t)4 * kNoallocMaxSub;
// causal substitution scratch for N = 1024: 4(N-1) complex sweep values, then N
// progress counters and the abort flag kProgStride ints apart
constexpr size_t kCausalBytes =
    sizeof(double2) * 4 * (kNoallocMaxSub - 1) + sizeof(int) * kNoallocMaxSub * kProgStride;
constexpr size_t kCausalElems = (kCausalBytes + sizeof(double2) - 1) / sizeof(double2);

std::mutex g_setup_mutex;
double2* g_scratch_addr[kNoallocMaxDevices] = {};
unsigned long long g_scratch_ctx[kNoallocMaxDevices] = {};

// Unique id of the current context (cuCtxGetId, looked up through the runtime so
// that the library needs no link to the driver library); 0 when unavailable, in
// which case the address is looked up on every call.
unsigned long long current_context_id() {
    typedef CUresult (*ctx_id_fn)(CUcontext, unsigned long long*);
    static ctx_id_fn fn = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        cudaGetLastError();
        fn = reinterpret_cast<ctx_id_fn>(f);
        looked_up = true;
    }
    unsigned long long id = 0;
    if (!fn || fn(nullptr, &id) != CUDA_SUCCESS) return 0;
    return id;
}

}  // namespace

// 2x2 lag-0 inverses, then the causal substitution scratch, then one status word
static __device__ __align__(256) double2 g_noalloc_scratch[kLag0Elems + kCausalElems + 1];

extern "C" swr_status swr_causal_solve_noalloc(int32_t nsub, int32_t nt, int32_t sweeps,
                                               const double* cols, const double* y, double* x,
                                               void* stream) {
    if (nsub < 2 || nsub > kNoallocMaxSub || nt < 1 || sweeps < 0 || sweeps > 16 || !cols || !y ||
        !x || x == y)
        return SWR_ERR_ARG;
    if (swr_causal_scratch_bytes(nsub) > kCausalBytes) return SWR_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SWR_ERR_CUDA;
    if (dev < 0 || dev >= kNoallocMaxDevices) return SWR_ERR_UNSUPPORTED;
    double2* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        const unsigned long long ctx = current_context_id();
        if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
            void* addr = nullptr;
            if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || !addr) {
                cudaGetLastError();
                g_scratch_addr[dev] = nullptr;
                return SWR_ERR_CUDA;
            }
            g_scratch_addr[dev] = static_cast<double2*>(addr);
            g_scratch_ctx[dev] = current_context_id();   // the lookup made one current
        }
        scratch = g_scratch_addr[dev];
    }
    double2* lag0 = scratch;
    double2* causal = scratch + kLag0Elems;
    int* status = reinterpret_cast<int*>(scratch + kLag0Elems + kCausalElems);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double2* c = reinterpret_cast<const double2*>(cols);
    // The lag-0 inverses and sweep values are written before they are read in
    // every call; the status word (and, inside the launcher, the progress
    // counters and abort flag) must start at zero and are cleared here.
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return SWR_ERR_CUDA;
    if (swr_launch_lag0_setup(nsub, nt, c, lag0, s) != 0) {
        cudaGetLastError();
        return SWR_ERR_CUDA;
    }
    const int rc = swr_launch_causal(nsub, nt, c, lag0, reinterpret_cast<const double2*>(y),
                                     reinterpret_cast<double2*>(x), sweeps, causal, status, s);
    if (rc == -2) return SWR_ERR_UNSUPPORTED;
    if (rc != 0) {
        cudaGetLastError();
        return SWR_ERR_CUDA;
    }
    int st = 0;
    if (cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SWR_ERR_CUDA;
    if (st & ST_TIMEOUT) return SWR_ERR_TIMEOUT;
    return SWR_OK;
}
