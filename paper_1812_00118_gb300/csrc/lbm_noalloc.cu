// Field diagnostics that allocate nothing.
//
// The same deterministic FP64 reduction as lbm_diagnostics (block partials in
// a fixed order, then one block sums the partials in a fixed order), but its
// scratch -- the per-block partials -- lives in a file-scope device array
// instead of memory obtained from cudaMalloc.  It serves callers that must
// not allocate device memory: a host framework whose allocator owns all
// device memory, or a real-time loop that may not touch the allocator.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>

#include "lbm.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;
constexpr long long kChunk = (long long)kThreads * kPerThread;   // nodes per block
constexpr int kMaxBlocks = LBM_NOALLOC_MAX_NODES / (int)kChunk;

// Four partials per block.  Held by every device that loads the library until
// the process exits; shared by all calls on that device.
__device__ __align__(256) double g_partials[kMaxBlocks * 4];

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block b reduces nodes [b*kChunk, (b+1)*kChunk) and writes its four partials.
__global__ void partial_kernel(const double* __restrict__ phi, const double* __restrict__ P,
                               const double* __restrict__ v0, const double* __restrict__ v1,
                               const double* __restrict__ v2, long long n, double rho_L, double rho_dif,
                               double* __restrict__ part) {
    __shared__ double sh[4][kThreads / 32];
    double s_phi = 0, s_rho = 0, m_v = 0, bad = 0;
    const long long base = blockIdx.x * kChunk;
    for (int k = 0; k < kPerThread; ++k) {
        const long long i = base + (long long)k * kThreads + threadIdx.x;
        if (i >= n) break;
        const double f = phi[i], p = P[i];
        const double a = v0 ? v0[i] : 0.0, b = v1 ? v1[i] : 0.0, c = v2 ? v2[i] : 0.0;
        s_phi += f;
        s_rho += rho_L + f * rho_dif;
        const double m = sqrt(a * a + b * b + c * c);
        if (!isfinite(f) || !isfinite(p) || !isfinite(m)) bad += 1;
        else m_v = fmax(m_v, m);
    }
    s_phi = warp_sum(s_phi); s_rho = warp_sum(s_rho); m_v = warp_max(m_v); bad = warp_sum(bad);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh[0][wid] = s_phi; sh[1][wid] = s_rho; sh[2][wid] = m_v; sh[3][wid] = bad; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r0 = 0, r1 = 0, r2 = 0, r3 = 0;
        for (int w = 0; w < kThreads / 32; ++w) { r0 += sh[0][w]; r1 += sh[1][w]; r2 = fmax(r2, sh[2][w]); r3 += sh[3][w]; }
        part[blockIdx.x * 4 + 0] = r0;
        part[blockIdx.x * 4 + 1] = r1;
        part[blockIdx.x * 4 + 2] = r2;
        part[blockIdx.x * 4 + 3] = r3;
    }
}

// One warp: lane k < 4 folds column k of the partials in block order.
__global__ void finish_kernel(const double* __restrict__ part, int nb, double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k >= 4) return;
    double r = 0;
    for (int b = 0; b < nb; ++b) {
        const double v = part[b * 4 + k];
        r = (k == 2) ? fmax(r, v) : r + v;
    }
    out[k] = r;
}

// Device address of g_partials, looked up at set-up once per device and
// context (host code may not use the symbol's name as a device pointer).  The
// context is part of the key: after cudaDeviceReset the device gets a new
// context, and the array a new address.
constexpr int kMaxDevices = 64;
struct Scratch {
    CUcontext ctx = nullptr;
    double* addr = nullptr;
};
Scratch g_scratch[kMaxDevices];

using CtxGetCurrent = CUresult (*)(CUcontext*);
CtxGetCurrent ctx_get_current() {
    static CtxGetCurrent fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrent)f;
    }
    return fn;
}

}  // namespace

extern "C" int lbm_field_sums_noalloc(const double* phi, const double* P, const double* v0, const double* v1,
                                      const double* v2, long long n, double rho_L, double rho_dif, double* out,
                                      void* cuda_stream) {
    if (!phi || !P || !out || n < 0) return LBM_EINVAL;
    if (n > (long long)LBM_NOALLOC_MAX_NODES) return LBM_EINVAL;
    // an error left by earlier, unrelated work is reported, not cleared
    if (cudaPeekAtLastError() != cudaSuccess) return LBM_ECUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ECUDA;
    // set-up: look the array up on the first call on this device, and again
    // whenever the current context is not the one of the last lookup (the
    // lookup also creates the device's primary context if none is current)
    CtxGetCurrent get = ctx_get_current();
    CUcontext ctx = nullptr;
    if (get && get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
    Scratch& sc = g_scratch[dev];
    if (!sc.addr || !ctx || sc.ctx != ctx) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess) return LBM_ECUDA;
        if (get && get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
        sc.addr = (double*)p;
        sc.ctx = ctx;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int nb = (int)((n + kChunk - 1) / kChunk);
    if (nb > 0)
        partial_kernel<<<nb, kThreads, 0, s>>>(phi, P, v0, v1, v2, n, rho_L, rho_dif, sc.addr);
    // every partial the finish reads was written above: nothing to clear first
    finish_kernel<<<1, 32, 0, s>>>(sc.addr, nb, out);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
