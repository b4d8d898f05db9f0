// mass_static.cu -- pflbm_phi_mass_noalloc: the FP64 phi-mass reduction for
// callers that cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc at all -- for example a
// component running inside a framework whose memory pool owns the whole
// device, or a latency-critical loop where cudaMalloc (which can synchronise
// the device) is not allowed. Such a caller cannot create a pflbm handle
// either, since creating one allocates the lattice. It can still hold a phi
// field in its own device memory and needs its FP64 sum.
//
// Scratch: the block partials live in a file-scope __device__ array of
// kStaticBlocks doubles (32 KB), which every GPU that loads this library
// keeps until the process exits. Host code may not use the array's name as a
// device address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it; that first
// call should therefore come before any stream capture. The cache is keyed on
// the unique id of the current CUDA context, so after cudaDeviceReset (which
// unloads the module: the array then lives at a new address) the next call
// looks the address up again, and that call too should come before any
// capture. All calls share the one array: calls whose kernels overlap on the
// GPU race on it. No element needs clearing: every call writes each partial
// it later reads.
#include <cuda.h>

#include <mutex>

#include "pflbm_internal.cuh"

namespace {

constexpr int kStaticBlocks = 4096;
constexpr int kThreads = 256;
constexpr int kNodesPerThread = 32;
constexpr long long kNodesPerBlock = (long long)kThreads * kNodesPerThread;   // 8192
constexpr long long kMaxNodes = kStaticBlocks * kNodesPerBlock;              // 33,554,432
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_mass_scratch[kStaticBlocks];

std::mutex g_setup_mutex;
struct ScratchEntry {
    unsigned long long ctx_id;   // id of the context the address belongs to (0: none yet)
    double* ptr;
};
ScratchEntry g_scratch[kMaxDevices] = {};

// Driver entry points, reached through the runtime (no link against libcuda).
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum(double v, double* sh)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = (lane < kThreads / 32) ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// One partial per block of kNodesPerBlock consecutive nodes, fixed order.
__global__ void __launch_bounds__(kThreads) k_phi_mass_partial(const double* __restrict__ phi,
                                                               const uint8_t* __restrict__ zeta, long long n,
                                                               double* __restrict__ partial)
{
    __shared__ double sh[kThreads / 32];
    const long long base = (long long)blockIdx.x * kNodesPerBlock;
    double acc = 0.0;
    for (int j = 0; j < kNodesPerThread; ++j) {
        long long k = base + (long long)j * kThreads + threadIdx.x;
        if (k < n && (!zeta || zeta[k])) acc += phi[k];
    }
    double r = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

__global__ void __launch_bounds__(kThreads) k_phi_mass_final(const double* __restrict__ partial, int nblocks,
                                                             double* __restrict__ out)
{
    __shared__ double sh[kThreads / 32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += kThreads) acc += partial[i];
    double r = block_sum(acc, sh);
    if (threadIdx.x == 0) *out = r;
}

// Unique id of the calling thread's current context; 0 when none is current.
cudaError_t current_context_id(unsigned long long* id)
{
    *id = 0;
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void* a = nullptr;
        void* b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa);
        if (e != cudaSuccess) return e;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb);
        if (e != cudaSuccess) return e;
        if (qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
            return cudaErrorNotSupported;
        g_ctx_get_current = (CtxGetCurrentFn)a;
        g_ctx_get_id = (CtxGetIdFn)b;
    }
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    if (!ctx) return cudaSuccess;
    if (g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}

// Device address of the static scratch for the current device, looked up once
// per context with cudaGetSymbolAddress.
cudaError_t scratch_for_current_device(double** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long id = 0;
    e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    if (id != 0 && g_scratch[dev].ctx_id == id && g_scratch[dev].ptr) {
        *out = g_scratch[dev].ptr;
        return cudaSuccess;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_mass_scratch);   // makes the device's context current
    if (e != cudaSuccess) return e;
    e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    g_scratch[dev].ctx_id = id;
    g_scratch[dev].ptr = (double*)p;
    *out = (double*)p;
    return cudaSuccess;
}

}  // namespace

namespace pfk {
int set_error(int code, const char* msg);
}

extern "C" int pflbm_phi_mass_noalloc(const double* d_phi, const uint8_t* d_zeta, int nx, int ny, double* d_out,
                                      void* stream)
{
    if (!d_phi || !d_out) return pfk::set_error(PFLBM_EINVAL, "pflbm_phi_mass_noalloc: NULL phi or out");
    if (nx < 1 || ny < 1) return pfk::set_error(PFLBM_EINVAL, "pflbm_phi_mass_noalloc: nx and ny must be >= 1");
    const long long n = (long long)nx * ny;
    if (n > kMaxNodes)
        return pfk::set_error(PFLBM_EINVAL,
                              "pflbm_phi_mass_noalloc: nx * ny exceeds the static scratch limit of 33554432 nodes");
    double* scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return pfk::set_error(PFLBM_ECUDA, cudaGetErrorString(e));
    const int nblocks = (int)((n + kNodesPerBlock - 1) / kNodesPerBlock);
    cudaStream_t s = (cudaStream_t)stream;
    k_phi_mass_partial<<<nblocks, kThreads, 0, s>>>(d_phi, d_zeta, n, scratch);
    k_phi_mass_final<<<1, kThreads, 0, s>>>(scratch, nblocks, d_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return pfk::set_error(PFLBM_ECUDA, cudaGetErrorString(e));
    return PFLBM_OK;
}
