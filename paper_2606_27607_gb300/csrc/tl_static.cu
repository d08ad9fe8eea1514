// Root log-likelihood for callers that cannot allocate device memory.
//
// Some host code cannot call cudaMalloc: code running while a CUDA graph is
// being captured by someone else, plug-ins whose host application owns the
// device allocator, or real-time loops that forbid allocation after start-up.
// This entry point evaluates the same quantity as tl_root_loglik for FP32
// four-state root partials held by the caller, and takes its scratch (one
// FP64 partial sum per 32-pattern tile) from a fixed array compiled into the
// library instead of allocating it.
#include <mutex>

#include "tl_internal.cuh"

namespace tl {
namespace {

// Per-tile partial sums: 65,536 tiles of 32 patterns = 2,097,152 patterns at
// most (512 KiB of device memory). The runtime loads this module lazily, so
// a device holds the array from the first use of the module on it (the
// first call of the entry point there) until the process exits.
constexpr int kStaticMaxTiles = 65536;
static __device__ __align__(256) double g_root_partials[kStaticMaxTiles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch[kMaxDevices] = {nullptr};

__global__ void k_root_static(const float* __restrict__ root, const int* __restrict__ exps,
                              const double* __restrict__ pi, const double* __restrict__ catw,
                              const double* __restrict__ patw, int n_patterns, int stride, int R,
                              int n_tiles, double* __restrict__ part) {
    const int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= n_tiles) return;
    const int p = tile * 32 + lane;
    double contrib = 0.0;
    if (p < n_patterns) {
        double L = 0.0;
        for (int r = 0; r < R; ++r) {
            float4 x = *reinterpret_cast<const float4*>(root + ((size_t)r * stride + p) * 4);
            L += catw[r] * (pi[0] * (double)x.x + pi[1] * (double)x.y + pi[2] * (double)x.z +
                            pi[3] * (double)x.w);
        }
        const double e = exps ? (double)exps[p] : 0.0;
        contrib = patw[p] * (log(L) + 0.69314718055994530942 * e);
    }
    for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
    if (lane == 0) part[tile] = contrib;
}

// Fixed-order sum of n partials into out (one block of 256 threads).
__global__ void k_sum_static(const double* __restrict__ part, int n, double* __restrict__ out) {
    __shared__ double s[256];
    double acc = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) acc += part[j];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// Device address of this device's copy of the scratch array. Host code only
// sees a host-side stand-in for the symbol, so the address is looked up once
// per device (with that device current) and cached. The lookup is the set-up
// of the first call on a device (it may load the module and reserve the
// array), which is why that call belongs before any stream capture; the
// cached address is that of the primary context and is stale after
// cudaDeviceReset.
int scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(nullptr, e, "tl_root_loglik_static: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(nullptr, TL_ERR_UNSUPPORTED, "tl_root_loglik_static: device %d >= %d", dev,
                    kMaxDevices);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_root_partials);
        if (e != cudaSuccess)
            return cuda_check(nullptr, e, "tl_root_loglik_static: cudaGetSymbolAddress");
        g_scratch[dev] = static_cast<double*>(p);
    }
    *out = g_scratch[dev];
    return TL_OK;
}

}  // namespace
}  // namespace tl

extern "C" int tl_root_loglik_static(const float* root_partials, const int32_t* exponents,
                                     const double* pi, const double* cat_weights,
                                     const double* pattern_weights, int n_patterns,
                                     int pattern_stride, int n_categories, double* out_logl,
                                     void* stream) {
    using namespace tl;
    if (!root_partials || !pi || !cat_weights || !pattern_weights || !out_logl)
        return fail(nullptr, TL_ERR_ARG, "tl_root_loglik_static: null pointer");
    if (n_categories < 1 || n_categories > kMaxCat)
        return fail(nullptr, TL_ERR_ARG, "tl_root_loglik_static: 1 <= n_categories <= %d", kMaxCat);
    if (n_patterns < 1 || pattern_stride < n_patterns)
        return fail(nullptr, TL_ERR_ARG, "tl_root_loglik_static: need 1 <= n_patterns <= stride");
    const long long tiles = ((long long)n_patterns + 31) / 32;
    if (tiles > kStaticMaxTiles)
        return fail(nullptr, TL_ERR_UNSUPPORTED,
                    "tl_root_loglik_static: %d patterns exceed the built-in scratch limit of %d",
                    n_patterns, kStaticMaxTiles * 32);
    if (reinterpret_cast<uintptr_t>(root_partials) % 16 != 0)
        return fail(nullptr, TL_ERR_ARG, "tl_root_loglik_static: root_partials not 16-byte aligned");
    double* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int threads = 128;
    const int blocks = (int)((tiles * 32 + threads - 1) / threads);
    // every tile's partial is written before it is read, so nothing in the
    // scratch array needs clearing between calls
    k_root_static<<<blocks, threads, 0, s>>>(root_partials, exponents, pi, cat_weights,
                                             pattern_weights, n_patterns, pattern_stride,
                                             n_categories, (int)tiles, scratch);
    k_sum_static<<<1, 256, 0, s>>>(scratch, (int)tiles, out_logl);
    return cuda_check(nullptr, cudaGetLastError(), "tl_root_loglik_static");
}
