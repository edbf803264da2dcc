// lbrmt_noalloc.cu -- total mass without any device allocation.
//
// lbrmt_total_mass_noalloc serves callers that cannot allocate device memory
// at the point where they need the diagnostic: a loop running after its
// device memory pool has been frozen, a host that handed all device memory to
// another allocator, or a real-time loop in which an allocation (and the
// synchronisation it may bring) is not allowed.  It computes the same quantity
// as the reduction behind lbrmt_total_mass, but keeps its per-block partial
// sums in the file-scope array below instead of memory the library allocates.
#include <cuda.h>

#include <mutex>

#include "lbrmt.h"
#include "lbrmt_sim.cuh"

namespace {

constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_CHUNK = 16384;       // nodes summed by one block
constexpr int NOALLOC_MAX_BLOCKS = 2048;   // partial sums held in the array: 16 KiB
constexpr long long NOALLOC_MAX_NODES = (long long)NOALLOC_CHUNK * NOALLOC_MAX_BLOCKS;

// Shared by every call on a device and kept until the process exits.  In host
// code this name is only a stand-in for the device array: kernels receive the
// device address looked up below, never the host symbol.
static __device__ __align__(256) double g_mass_partials[NOALLOC_MAX_BLOCKS];

constexpr int MAX_DEVICES = 64;
std::mutex g_lock;
double *g_partials_addr[MAX_DEVICES] = {nullptr};
CUcontext g_partials_ctx[MAX_DEVICES] = {nullptr};  // context the address belongs to

// cuCtxGetCurrent through the runtime's driver entry point (no link to libcuda).
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
    }
    return fn;
}

// Device address of g_mass_partials on the current device.  It is looked up
// on the first call on a device (that call must not be inside a stream
// capture) and again whenever the device's context has changed since (after a
// cudaDeviceReset the old address is no longer valid).
cudaError_t partials_address(int dev, double **out) {
    std::lock_guard<std::mutex> guard(g_lock);
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    CUcontext ctx = nullptr;
    CtxGetCurrentFn cur = ctx_get_current();
    if (cur && cur(&ctx) != CUDA_SUCCESS) ctx = nullptr;
    if (!g_partials_addr[dev] || !ctx || ctx != g_partials_ctx[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_mass_partials);
        if (e != cudaSuccess) return e;
        g_partials_addr[dev] = static_cast<double *>(p);
        g_partials_ctx[dev] = ctx;
    }
    *out = g_partials_addr[dev];
    return cudaSuccess;
}

// Block b sums rho - rho_f over nodes [b C, (b+1) C): the nine stored values plus
// the rest base (Delta rho of the step that wrote them, on registered tiles).
template <class R, class S>
__global__ void __launch_bounds__(NOALLOC_THREADS) noalloc_mass_partials(lbrmt::SimParams sp, const S *f, const int *reg,
                                                                         const R *pool, double *partials) {
    const long long P = sp.P;
    __shared__ double sh[NOALLOC_THREADS];
    const long long begin = (long long)blockIdx.x * NOALLOC_CHUNK;
    const long long end = begin + NOALLOC_CHUNK < P ? begin + NOALLOC_CHUNK : P;
    double acc = 0.0;
    for (long long c = begin + threadIdx.x; c < end; c += NOALLOC_THREADS) {
        double s = 0.0;
        for (int q = 0; q < 9; q++) s += (double)lbrmt::ldS<S, R>(f + q * P + c, sp, q);
        s += lbrmt::rest_base_d<R>(sp, reg, pool, (int)(c % sp.nx), (int)(c / sp.nx));
        acc += s;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int k = NOALLOC_THREADS / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(NOALLOC_THREADS) noalloc_mass_final(const double *partials, int n, double base,
                                                                      double *out) {
    __shared__ double sh[NOALLOC_THREADS];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += NOALLOC_THREADS) acc += partials[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int k = NOALLOC_THREADS / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = base + sh[0];
}

}  // namespace

extern "C" lbrmt_status lbrmt_total_mass_noalloc(lbrmt_sim *s, int sim_index, double *dev_out) {
    if (!s || !dev_out || sim_index != 0) return LBRMT_ERR_ARG;
    if (!s->inited) {
        s->err = "lbrmt_total_mass_noalloc needs an initialised simulation (call lbrmt_init first)";
        return LBRMT_ERR_STATE;
    }
    const long long P = s->sp.P;
    if (P > NOALLOC_MAX_NODES) {
        s->err = "lbrmt_total_mass_noalloc handles at most 33554432 nodes (2048 partial sums of 16384 nodes)";
        return LBRMT_ERR_ARG;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && dev != s->device) {
        s->err = "lbrmt_total_mass_noalloc: make the simulation's device current first";
        return LBRMT_ERR_ARG;
    }
    double *partials = nullptr;
    if (e == cudaSuccess) e = partials_address(dev, &partials);
    if (e != cudaSuccess) {
        s->err = std::string("lbrmt_total_mass_noalloc: scratch lookup: ") + cudaGetErrorString(e);
        return LBRMT_ERR_CUDA;
    }
    const int nblocks = (int)((P + NOALLOC_CHUNK - 1) / NOALLOC_CHUNK);
    const int cur = (int)(s->steps & 1);
    const void *f = s->d.f[cur];
    const int *reg = s->d.reg_count[1 - cur];
    const void *pool = s->d.pool[1 - cur];
    // each block overwrites its partial sum, so nothing in the array needs clearing
    switch (s->cfg.precision) {
    case LBRMT_FP64:
        noalloc_mass_partials<double, double><<<nblocks, NOALLOC_THREADS, 0, s->stream>>>(
            s->sp, (const double *)f, reg, (const double *)pool, partials);
        break;
    case LBRMT_FP16_STORE:
        noalloc_mass_partials<float, __half><<<nblocks, NOALLOC_THREADS, 0, s->stream>>>(
            s->sp, (const __half *)f, reg, (const float *)pool, partials);
        break;
    case LBRMT_BF16_STORE:
        noalloc_mass_partials<float, __nv_bfloat16><<<nblocks, NOALLOC_THREADS, 0, s->stream>>>(
            s->sp, (const __nv_bfloat16 *)f, reg, (const float *)pool, partials);
        break;
    default:
        noalloc_mass_partials<float, float><<<nblocks, NOALLOC_THREADS, 0, s->stream>>>(
            s->sp, (const float *)f, reg, (const float *)pool, partials);
        break;
    }
    noalloc_mass_final<<<1, NOALLOC_THREADS, 0, s->stream>>>(partials, nblocks, s->sp.rho_f * (double)P, dev_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        s->err = std::string("lbrmt_total_mass_noalloc: launch: ") + cudaGetErrorString(e);
        return LBRMT_ERR_CUDA;
    }
    return LBRMT_OK;
}
