// Host side of liblbm: the C-ABI declared in include/lbm.h.
//
// Owns the A/B population buffers, derives the model constants of Section 2
// from the user parameters, maps user axes to the internal (march-along-z)
// axes, and launches the kernels of lbm_kernels.cuh on the context stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_tma.cuh"

using namespace lbm;

namespace lbm {
const KernelTable* table_for(int lattice, int store) {
    switch (lattice * 4 + store) {
        case 0: return table_l0_s0();
        case 1: return table_l0_s1();
        case 2: return table_l0_s2();
        case 3: return table_l0_s3();
        case 4: return table_l1_s0();
        case 5: return table_l1_s1();
        case 6: return table_l1_s2();
        case 7: return table_l1_s3();
        default: return nullptr;
    }
}
}  // namespace lbm


namespace {

constexpr double kT = 1.0 / 3.0;

int check_cuda(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ECUDA; }


size_t elem_size(int store) {
    switch (store) {
        case LBM_F64: return 8;
        case LBM_F32: return 4;
        case LBM_F16S: case LBM_BF16S: return 2;
        default: return 0;
    }
}

// Model constants (Section 2): tau_phi = M/T + 1/2 (Eq. 1), theta = (M/T)(...)/W
// (Eq. 4), beta = 48 sigma/W and kappa = 3 sigma W/2 (Eq. 8), tau = nu/T + 1/2
// and the interpolation of 1/tau (Eq. 9).
int derive(const lbm_params& u, int lattice, Phys* out) {
    if (!(u.M > 0) || !(u.W > 0) || !(u.sigma >= 0) || !(u.rho_L > 0) || !(u.rho_H > 0) ||
        !(u.nu_L > 0) || !(u.nu_H > 0) || !(u.eps > 0))
        return LBM_EINVAL;
    if (u.force_mode != 0 && u.force_mode != 1) return LBM_EINVAL;
    // every real parameter finite (an infinite viscosity or density, or a
    // NaN shift of the 16-bit storage, would only show as a diverged state)
    const double reals[] = {u.M, u.W, u.sigma, u.rho_L, u.rho_H, u.nu_L, u.nu_H, u.g[0], u.g[1], u.g[2],
                            u.eps, u.P_ref, u.g_scale, u.C_dtheta};
    for (double v : reals)
        if (!std::isfinite(v)) return LBM_EINVAL;
    if (u.g_scale < 0) return LBM_EINVAL;
    if (elem_size(u.store) == 0) return LBM_EINVAL;
    Phys p{};
    p.inv_tau_phi = 1.0 / (u.M / kT + 0.5);
    p.theta_coef = (u.M / kT) / u.W;
    p.beta = 48.0 * u.sigma / u.W;
    p.kappa = 1.5 * u.sigma * u.W;
    p.rho_L = u.rho_L;
    p.rho_dif = u.rho_H - u.rho_L;
    const double tau_L = u.nu_L / kT + 0.5, tau_H = u.nu_H / kT + 0.5;
    p.om_L = 1.0 / tau_L;
    p.om_dif = 1.0 / tau_H - 1.0 / tau_L;
    if (lattice == LBM_D2Q9) {   // user (x, y) -> internal (x, z)
        p.g[0] = u.g[0]; p.g[1] = 0.0; p.g[2] = u.g[1];
    } else {
        p.g[0] = u.g[0]; p.g[1] = u.g[1]; p.g[2] = u.g[2];
    }
    p.force_mode = u.force_mode;
    p.rho_bar = 0.0;
    p.eps = u.eps;
    p.hocorr = u.hocorr ? 1 : 0;
    const bool shifted = u.store == LBM_F16S || u.store == LBM_BF16S;
    p.h_shift = shifted ? 0.5 : 0.0;
    p.g_shift = shifted ? u.P_ref / kT : 0.0;
    p.g_scale = shifted && u.g_scale > 0 ? u.g_scale : 1.0;
    p.g_inv_scale = 1.0 / p.g_scale;
    p.dtheta_coef = u.C_dtheta * (u.M / kT) * u.W * u.W;   // Eq. 14, F of the header
    *out = p;
    return LBM_OK;
}

int ensure_scratch(lbm_ctx* c) {
    if (c->fields && c->partial) return LBM_OK;
    if (!c->fields) {
        cudaError_t e = cudaMallocAsync((void**)&c->fields, sizeof(double) * 5 * (size_t)c->G.N, c->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->fields = nullptr;
            return LBM_ENOMEM;
        }
    }
    c->n_partial_blocks = 1024;
    cudaError_t e = cudaMallocAsync((void**)&c->partial, sizeof(double) * 8 * c->n_partial_blocks, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(c->fields, c->stream);
        c->fields = nullptr;
        c->partial = nullptr;
        return LBM_ENOMEM;
    }
    return LBM_OK;
}

double* f_phi(lbm_ctx* c) { return c->fields; }
double* f_P(lbm_ctx* c) { return c->fields + c->G.N; }
double* f_u(lbm_ctx* c, int a) { return c->fields + (2 + a) * c->G.N; }

// phi, P, u of the current state into the scratch fields.
int compute_fields(lbm_ctx* c) {
    int rc = ensure_scratch(c);
    if (rc) return rc;
    if (check_cuda(c->K->phi(c->h[c->cur], c->G, c->P, f_phi(c), c->stream))) return LBM_ECUDA;
    if (check_cuda(c->K->macro(c->g[c->cur], c->G, c->P, f_phi(c), f_P(c), f_u(c, 0), f_u(c, 1), f_u(c, 2),
                               c->stream)))
        return LBM_ECUDA;
    c->launches += 2;
    return LBM_OK;
}

// internal component index of user velocity component d
int internal_axis(const lbm_ctx* c, int d) { return (c->lattice == LBM_D2Q9 && d == 1) ? 2 : d; }

// ---------------------------------------------------------------- reductions
// Block partials in a fixed order, then one block sums the partials in a
// fixed order: the result is deterministic for a given grid.
constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// out[b*4 + {0,1,2,3}] = sum phi, sum rho, max |u|, non-finite count of block b
__global__ void diag_partial_kernel(const double* __restrict__ phi, const double* __restrict__ P,
                                    const double* __restrict__ ux, const double* __restrict__ uy,
                                    const double* __restrict__ uz, long long N, double rho_L, double rho_dif,
                                    double* out) {
    __shared__ double sh[4][kRedThreads / 32];
    double s_phi = 0, s_rho = 0, m_u = 0, bad = 0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const double f = phi[n];
        const double a = ux[n], b = uy[n], d = uz[n], p = P[n];
        s_phi += f;
        s_rho += rho_L + f * rho_dif;
        const double um = sqrt(a * a + b * b + d * d);
        if (!isfinite(f) || !isfinite(p) || !isfinite(um)) bad += 1;
        else m_u = fmax(m_u, um);
    }
    s_phi = warp_sum(s_phi); s_rho = warp_sum(s_rho); m_u = warp_max(m_u); bad = warp_sum(bad);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh[0][wid] = s_phi; sh[1][wid] = s_rho; sh[2][wid] = m_u; sh[3][wid] = bad; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r0 = 0, r1 = 0, r2 = 0, r3 = 0;
        for (int w = 0; w < kRedThreads / 32; ++w) { r0 += sh[0][w]; r1 += sh[1][w]; r2 = fmax(r2, sh[2][w]); r3 += sh[3][w]; }
        out[blockIdx.x * 4 + 0] = r0; out[blockIdx.x * 4 + 1] = r1;
        out[blockIdx.x * 4 + 2] = r2; out[blockIdx.x * 4 + 3] = r3;
    }
}

// sum / max of nb partial rows of width `width` (columns in max_mask use max)
__global__ void finish_kernel(const double* __restrict__ part, int nb, int width, int max_mask, double* out) {
    if (threadIdx.x >= (unsigned)width) return;
    const int k = threadIdx.x;
    double r = 0;
    for (int b = 0; b < nb; ++b) {
        const double v = part[b * width + k];
        r = ((max_mask >> k) & 1) ? fmax(r, v) : r + v;
    }
    out[k] = r;
}

// Laplace partials: sum P and count for r < r_in, and for r > r_out.
__global__ void laplace_partial_kernel(const double* __restrict__ P, Geom G, double cx, double cy, double cz,
                                       double r_in, double r_out, double* out) {
    __shared__ double sh[4][kRedThreads / 32];
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < G.N; n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % G.NX), y = (int)((n / G.NX) % G.NY), z = (int)(n / ((long long)G.NX * G.NY));
        double d[3] = {x - cx, y - cy, z - cz};
        const int nn[3] = {G.NX, G.NY, G.NZ};
        double r2 = 0;
        for (int a = 0; a < 3; ++a) {
            double v = d[a];
            if (!G.wall[a]) v = v - nn[a] * floor(v / nn[a] + 0.5);
            if (nn[a] > 1) r2 += v * v;
        }
        const double r = sqrt(r2);
        if (r < r_in) { a0 += P[n]; a1 += 1; }
        if (r > r_out) { a2 += P[n]; a3 += 1; }
    }
    a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2); a3 = warp_sum(a3);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh[0][wid] = a0; sh[1][wid] = a1; sh[2][wid] = a2; sh[3][wid] = a3; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r[4] = {0, 0, 0, 0};
        for (int w = 0; w < kRedThreads / 32; ++w) for (int k = 0; k < 4; ++k) r[k] += sh[k][w];
        for (int k = 0; k < 4; ++k) out[blockIdx.x * 4 + k] = r[k];
    }
}

// Re-imposition of the total of phi: block partials of sum a (fixed order),
// then delta = (target - sum) / N in one thread.
constexpr int kFixBlocks = 1024;

__global__ void sum_partial_kernel(const double* __restrict__ a, long long n, double* __restrict__ part) {
    __shared__ double sh[kRedThreads];
    double s = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        s += a[k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void phi_delta_kernel(const double* __restrict__ part, int nb, double target, long long n,
                                 double* __restrict__ delta) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b];
    *delta = (target - s) / (double)n;
}

// rho u = rho(phi) u
__global__ void rho_times_u_kernel(const double* __restrict__ phi, const double* __restrict__ u, long long N,
                                   double rho_L, double rho_dif, double* out) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n < N) out[n] = (rho_L + phi[n] * rho_dif) * u[n];
}

int partial_blocks(const lbm_ctx* c) {
    long long b = (c->G.N + kRedThreads - 1) / kRedThreads;
    return (int)(b < c->n_partial_blocks ? b : c->n_partial_blocks);
}

// FP64 sums of the scratch fields -> host out[4]
int reduce_diag(lbm_ctx* c, double out[4]) {
    const int nb = partial_blocks(c);
    double* res = c->partial + 4 * (size_t)c->n_partial_blocks;
    diag_partial_kernel<<<nb, kRedThreads, 0, c->stream>>>(f_phi(c), f_P(c), f_u(c, 0), f_u(c, 1), f_u(c, 2),
                                                          c->G.N, c->P.rho_L, c->P.rho_dif, c->partial);
    finish_kernel<<<1, 32, 0, c->stream>>>(c->partial, nb, 4, 1 << 2, res);
    c->launches += 2;
    if (check_cuda(cudaGetLastError())) return LBM_ECUDA;
    if (check_cuda(cudaMemcpyAsync(out, res, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream))) return LBM_ECUDA;
    return check_cuda(cudaStreamSynchronize(c->stream));
}

// Total of phi restored to phi_target (FP64 sums on the GPU, uniform shift of
// the rest population); stream-ordered, no host synchronisation.
int phi_fix(lbm_ctx* c) {
    if (check_cuda(c->K->phi(c->h[c->cur], c->G, c->P, f_phi(c), c->stream))) return LBM_ECUDA;
    long long nb = (c->G.N + kRedThreads - 1) / kRedThreads;
    if (nb > kFixBlocks) nb = kFixBlocks;
    sum_partial_kernel<<<(unsigned)nb, kRedThreads, 0, c->stream>>>(f_phi(c), c->G.N, c->d_fix);
    phi_delta_kernel<<<1, 32, 0, c->stream>>>(c->d_fix, (int)nb, c->phi_target, c->G.N, c->d_fix + kFixBlocks);
    if (check_cuda(cudaGetLastError())) return LBM_ECUDA;
    if (check_cuda(c->K->shift_rest(c->h[c->cur], c->G, c->P, c->d_fix + kFixBlocks, c->stream))) return LBM_ECUDA;
    c->launches += 4;
    return LBM_OK;
}

int copy_field(lbm_ctx* c, double* dst, const double* src, size_t n, int on_device) {
    return check_cuda(cudaMemcpyAsync(dst, src, n * sizeof(double),
                                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
}

// rho_bar for force_mode 1 from the current state's phi (scratch fields must be fresh)
int update_rho_bar(lbm_ctx* c) {
    double d[4];
    int rc = reduce_diag(c, d);
    if (rc) return rc;
    c->P.rho_bar = c->P.rho_L + c->P.rho_dif * d[0] / (double)c->G.N;
    return LBM_OK;
}

}  // namespace

namespace lbm {

// Everything of lbm_create but the device buffers: checks, model constants,
// internal geometry (ghost-padded, base 0) and kernel table.
int ctx_setup(lbm_ctx* c, const lbm_grid* grid, int lattice, const lbm_params* params, void* cuda_stream,
              int flags) {
    if (flags & ~LBM_CREATE_GHOST_BAND) return LBM_EINVAL;
    if (!grid || !params) return LBM_EINVAL;
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19) return LBM_EINVAL;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return LBM_EINVAL;
    if (lattice == LBM_D2Q9 && grid->nz != 1) return LBM_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (grid->bc[a] != LBM_PERIODIC && grid->bc[a] != LBM_WALL) return LBM_EINVAL;
    Phys P;
    int rc = derive(*params, lattice, &P);
    if (rc) return rc;
    c->lattice = lattice;
    c->store = params->store;
    c->dim = lattice == LBM_D2Q9 ? 2 : 3;
    c->grid = *grid;
    c->params = *params;
    c->P = P;
    c->stream = (cudaStream_t)cuda_stream;
    c->elem = elem_size(params->store);
    if (lattice == LBM_D2Q9) {
        c->G.NX = grid->nx; c->G.NY = 1; c->G.NZ = grid->ny;
        c->G.wall[0] = grid->bc[0] == LBM_WALL; c->G.wall[1] = 0; c->G.wall[2] = grid->bc[1] == LBM_WALL;
        c->K = table_for(0, params->store);
        c->lz = 16;
    } else {
        c->G.NX = grid->nx; c->G.NY = grid->ny; c->G.NZ = grid->nz;
        for (int a = 0; a < 3; ++a) c->G.wall[a] = grid->bc[a] == LBM_WALL;
        c->K = table_for(1, params->store);
        c->lz = 16;
    }
    // ghost padding (see lbm_kernels.cuh), on walled axes only unless the
    // ghost band is asked for: x ghosts of 32 bytes (at least 2 cells); y
    // ghosts 2 cells (D3Q19); one ghost plane at each z end.  Rows are padded
    // to 32 bytes either way.  A periodic axis needs no ghost cell (the pulls
    // wrap), and leaving them out keeps the 256-byte L2 fetches of the step
    // kernel from bringing in padding: at 128^3 the rows are then exactly
    // two 256-byte blocks.
    {
        const bool band = (flags & LBM_CREATE_GHOST_BAND) != 0;
        const int A32 = (int)(32 / c->elem);            // elements per 32 bytes
        c->G.GX = (band || c->G.wall[0]) ? (A32 > 2 ? A32 : 2) : 0;
        c->G.GY = lattice == LBM_D2Q9 ? 0 : ((band || c->G.wall[1]) ? 2 : 0);
        c->G.GZ = (band || c->G.wall[2]) ? 1 : 0;
        // extents in 64 bits, checked before they are narrowed: the kernels
        // index one population array with 32-bit offsets (PX * PY * PZ < 2^31)
        const long long px = ((long long)c->G.NX + A32 - 1) / A32 * A32 + 2LL * c->G.GX;
        const long long py = (long long)c->G.NY + 2LL * c->G.GY;
        const long long pz = (long long)c->G.NZ + 2LL * c->G.GZ;
        const long long pxy = px * py;                 // < 2^63: each factor < 2^32
        if (pxy >= (1LL << 31) || pxy * pz >= (1LL << 31)) return LBM_EINVAL;
        c->G.PX = (int)px;
        c->G.PY = (int)py;
        c->G.PZ = (int)pz;
        c->G.PXY = (int)pxy;
        c->G.NP = pxy * pz;
    }
    c->G.N = (long long)c->G.NX * c->G.NY * c->G.NZ;
    if (!c->K) return LBM_EINVAL;
    // default: per-thread loads in phases (the fastest tiles on the measured
    // grids; lbm_autotune picks per grid): D2Q9 at 8 CTAs per SM; D3Q19 at 7
    // CTAs per SM (72 registers) and 16 planes, which keeps a grid like 128^3
    // (1024 CTAs) in one wave, and for FP32 storage from 2^24 nodes on, where
    // the grid runs in several waves anyway, at 6 CTAs per SM (80 registers,
    // fewer spills) and 32 planes (256 x 256 x 512: 1.988 against 2.068 ms per
    // step; the 16-bit forms are faster at 7 CTAs per SM: 1.776 against 1.820)
    if (lattice == LBM_D2Q9) {
        c->tile = 1;
    } else if (params->store == LBM_F32 && c->G.N >= (1LL << 24)) {
        c->tile = 3;
        c->lz = 32;
    } else {
        c->tile = 8;
    }
    return LBM_OK;
}

}  // namespace lbm

extern "C" {

int lbm_checked_status(void* stream) {
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return LBM_ECUDA;
    int worst = 0;
    for (int lat = 0; lat < 2; ++lat)
        for (int st = 0; st < 4; ++st) {
            const int v = table_for(lat, st)->checked_status();
            if (v < 0) return LBM_ECUDA;
            if (v > worst) worst = v;
        }
    return worst ? LBM_ECHECKED : LBM_OK;
}

int lbm_is_checked_build(void) {
#ifdef LBM_CHECKED
    return 1;
#else
    return 0;
#endif
}

const char* lbm_strerror(int s) {
    switch (s) {
        case LBM_OK: return "ok";
        case LBM_EINVAL: return "invalid argument";
        case LBM_ENOMEM: return "device allocation failed";
        case LBM_ECUDA: return "CUDA call failed";
        case LBM_EDIVERGED: return "simulation diverged (non-finite value or |u| > 0.3)";
        case LBM_ETIMEOUT: return "bounded device wait timed out";
        case LBM_ENOTSUP: return "not supported";
        case LBM_ECHECKED: return "an offset check of a checked build failed";
        default: return "unknown status";
    }
}

int lbm_lattice_info(int lattice, int* Q, int* c, double* w) {
    if (lattice == LBM_D2Q9) {
        using L = Lattice<0>;
        if (Q) *Q = L::Q;
        for (int i = 0; i < L::Q; ++i) {
            if (c) { c[3 * i] = L::cx[i]; c[3 * i + 1] = L::cz[i]; c[3 * i + 2] = 0; }
            if (w) w[i] = L::w[i];
        }
        return LBM_OK;
    }
    if (lattice == LBM_D3Q19) {
        using L = Lattice<1>;
        if (Q) *Q = L::Q;
        for (int i = 0; i < L::Q; ++i) {
            if (c) { c[3 * i] = L::cx[i]; c[3 * i + 1] = L::cy[i]; c[3 * i + 2] = L::cz[i]; }
            if (w) w[i] = L::w[i];
        }
        return LBM_OK;
    }
    return LBM_EINVAL;
}

int lbm_create(const lbm_grid* grid, int lattice, const lbm_params* params, void* cuda_stream, lbm_ctx** out) {
    return lbm_create_ex(grid, lattice, params, cuda_stream, 0, out);
}

int lbm_create_ex(const lbm_grid* grid, int lattice, const lbm_params* params, void* cuda_stream, int flags,
                  lbm_ctx** out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ENOMEM;
    int rc = ctx_setup(c, grid, lattice, params, cuda_stream, flags);
    if (rc) { delete c; return rc; }
    const int Q = lattice == LBM_D2Q9 ? 9 : 19;
    const size_t bytes = c->elem * (size_t)Q * (size_t)c->G.NP;
    for (int b = 0; b < 2; ++b) {
        if (cudaMallocAsync(&c->h[b], bytes, c->stream) != cudaSuccess ||
            cudaMallocAsync(&c->g[b], bytes, c->stream) != cudaSuccess) {
            cudaGetLastError();
            lbm_destroy(c);
            return LBM_ENOMEM;
        }
        cudaMemsetAsync(c->h[b], 0, bytes, c->stream);
        cudaMemsetAsync(c->g[b], 0, bytes, c->stream);
    }
    if (cudaMallocAsync((void**)&c->d_err, sizeof(int), c->stream) != cudaSuccess) {
        cudaGetLastError();
        lbm_destroy(c);
        return LBM_ENOMEM;
    }
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) { lbm_destroy(c); return LBM_ECUDA; }
    *out = c;
    return LBM_OK;
}

int lbm_layout(const lbm_grid* grid, int lattice, const lbm_params* params, int flags, long long out[6]) {
    if (!out) return LBM_EINVAL;
    lbm_ctx c;                       // set-up only: no device call, nothing allocated
    int rc = ctx_setup(&c, grid, lattice, params, nullptr, flags);
    if (rc) return rc;
    const long long Q = lattice == LBM_D2Q9 ? 9 : 19;
    const long long pops = 4LL * Q * c.G.NP * (long long)c.elem;    // h and g, two buffers each
    out[0] = c.G.PX;
    out[1] = c.G.PY;
    out[2] = c.G.PZ;
    out[3] = c.G.NP;
    out[4] = pops;
    // plus the error flag, and the scratch fields and reduction partials the
    // first lbm_init_fields / lbm_macro / lbm_diagnostics allocate
    out[5] = pops + (long long)sizeof(int) + 5LL * (long long)sizeof(double) * c.G.N +
             8LL * (long long)sizeof(double) * 1024;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
    if (!c || c->owner) return;
    for (int b = 0; b < 2; ++b) {
        if (c->h[b]) cudaFreeAsync(c->h[b], c->stream);
        if (c->g[b]) cudaFreeAsync(c->g[b], c->stream);
    }
    if (c->fields) cudaFreeAsync(c->fields, c->stream);
    if (c->d_err) cudaFreeAsync(c->d_err, c->stream);
    if (c->partial) cudaFreeAsync(c->partial, c->stream);
    if (c->d_fix) cudaFreeAsync(c->d_fix, c->stream);
    cudaStreamSynchronize(c->stream);
    delete c;
}

int lbm_init_fields(lbm_ctx* c, const double* phi, const double* u, const double* P, int on_device) {
    return lbm_init_fields_ex(c, phi, u, P, on_device, 0);
}

int lbm_init_fields_ex(lbm_ctx* c, const double* phi, const double* u, const double* P, int on_device, int flags) {
    lbm::NvtxRange range("lbm_init_fields");
    if (!c || !phi || !u || !P || (flags & ~LBM_INIT_NONEQ)) return LBM_EINVAL;
    const long long N = c->G.N;
    int rc = ensure_scratch(c);
    if (rc) return rc;
    // stage the inputs in the scratch fields (internal component order)
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (check_cuda(cudaMemcpyAsync(f_phi(c), phi, N * sizeof(double), kind, c->stream))) return LBM_ECUDA;
    if (check_cuda(cudaMemcpyAsync(f_P(c), P, N * sizeof(double), kind, c->stream))) return LBM_ECUDA;
    if (check_cuda(cudaMemsetAsync(f_u(c, 0), 0, 3 * N * sizeof(double), c->stream))) return LBM_ECUDA;
    for (int d = 0; d < c->dim; ++d)
        if (check_cuda(cudaMemcpyAsync(f_u(c, internal_axis(c, d)), u + d * N, N * sizeof(double), kind, c->stream)))
            return LBM_ECUDA;
    {   // total of phi (kept for the re-imposition) and rho_bar from the given phi
        double d[4];
        rc = reduce_diag(c, d);
        if (rc) return rc;
        c->phi_target = d[0];
        if (c->P.force_mode == 1) c->P.rho_bar = c->P.rho_L + c->P.rho_dif * d[0] / (double)N;
    }
    c->phi_fix_count = 0;
    // the state is written into the current buffer (for a grid of a batch,
    // the buffer all its grids hold the state in)
    const int b = c->cur;
    if (check_cuda(c->K->init(c->h[b], c->g[b], c->G, c->P, f_phi(c), f_u(c, 0), f_u(c, 1), f_u(c, 2), f_P(c),
                              (flags & LBM_INIT_NONEQ) ? 1 : 0, c->stream)))
        return LBM_ECUDA;
    c->ghosts[b] = true;   // the initialisation writes the periodic images too
    c->diverged = false;
    if (check_cuda(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream))) return LBM_ECUDA;
    c->launches += 1;
    return check_cuda(cudaStreamSynchronize(c->stream));
}

static int step_impl(lbm_ctx* c, int n, cudaEvent_t* ev);

int lbm_step(lbm_ctx* c, int n) {
    lbm::NvtxRange range("lbm_step");
    return step_impl(c, n, nullptr);
}

int lbm_step_profiled(lbm_ctx* c, int n, double* kernel_ms) {
    if (!c || n < 0 || !kernel_ms || c->owner) return LBM_EINVAL;
    cudaEvent_t* ev = (cudaEvent_t*)calloc(2 * (size_t)(n > 0 ? n : 1), sizeof(cudaEvent_t));
    if (!ev) return LBM_ENOMEM;
    int rc = LBM_OK;
    for (int k = 0; k < 2 * n && !rc; ++k) rc = check_cuda(cudaEventCreate(&ev[k]));
    if (!rc) rc = step_impl(c, n, ev);
    if (!rc && n > 0) rc = check_cuda(cudaEventSynchronize(ev[2 * n - 1]));
    double total = 0;
    for (int k = 0; k < n && !rc; ++k) {
        float ms = 0;
        rc = check_cuda(cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]));
        total += ms;
    }
    for (int k = 0; k < 2 * n; ++k)
        if (ev[k]) cudaEventDestroy(ev[k]);
    free(ev);
    *kernel_ms = total;
    return rc;
}

static int step_impl(lbm_ctx* c, int n, cudaEvent_t* ev) {
    if (!c || n < 0 || c->owner) return LBM_EINVAL;
    if (c->diverged) return LBM_EDIVERGED;
    const bool tma = c->K->tile_tma[c->tile] != 0;
    if (tma && c->maps_tile != c->tile) {
        for (int b = 0; b < 2; ++b)
            if (check_cuda(c->K->make_maps(c->tile, &c->maps[b], c->h[b], c->g[b], c->G))) return LBM_ECUDA;
        c->maps_tile = c->tile;
    }
    StepArgs a;
    a.G = c->G;
    a.p = c->P;
    a.tile = c->tile;
    a.lz = c->lz;
    a.stream = c->stream;
    a.error_flag = c->d_err;
    a.wait_polls = c->wait_polls;
    for (int s = 0; s < n; ++s) {
        const int i = c->cur, o = 1 - c->cur;
        a.hin = c->h[i]; a.gin = c->g[i]; a.hout = c->h[o]; a.gout = c->g[o];
        a.maps = &c->maps[i];
        // bulk-copy tiles read the ghost band unwrapped: it must hold the
        // periodic images (per-thread-load tiles wrap their pulls instead)
        if (tma && !c->ghosts[i]) {
            if (check_cuda(c->K->halo(c->h[i], c->g[i], c->G, c->stream))) return LBM_ECUDA;
            c->ghosts[i] = true;
            c->launches += 1;
        }
        if (ev) cudaEventRecord(ev[2 * s], c->stream);
        if (check_cuda(c->K->step(a))) return LBM_ECUDA;
        if (ev) cudaEventRecord(ev[2 * s + 1], c->stream);
        c->launches += 1;
        c->ghosts[o] = false;
        if (tma) {
            if (check_cuda(c->K->halo(c->h[o], c->g[o], c->G, c->stream))) return LBM_ECUDA;
            c->ghosts[o] = true;
            c->launches += 1;
        }
        c->cur = o;
        if (c->phi_fix_every > 0 && ++c->phi_fix_count >= c->phi_fix_every) {
            if (phi_fix(c)) return LBM_ECUDA;
            c->phi_fix_count = 0;
        }
    }
    return LBM_OK;
}

int lbm_macro(lbm_ctx* c, double* phi, double* P, double* rho_u, int on_device) {
    lbm::NvtxRange range("lbm_macro");
    if (!c) return LBM_EINVAL;
    int rc = compute_fields(c);
    if (rc) return rc;
    const long long N = c->G.N;
    if (phi && copy_field(c, phi, f_phi(c), N, on_device)) return LBM_ECUDA;
    if (P && copy_field(c, P, f_P(c), N, on_device)) return LBM_ECUDA;
    if (rho_u) {
        double* dst = rho_u;
        if (!on_device && cudaMallocAsync((void**)&dst, sizeof(double) * c->dim * (size_t)N, c->stream) != cudaSuccess) {
            cudaGetLastError();
            return LBM_ENOMEM;
        }
        const unsigned nb = (unsigned)((N + 255) / 256);
        for (int d = 0; d < c->dim; ++d)
            rho_times_u_kernel<<<nb, 256, 0, c->stream>>>(f_phi(c), f_u(c, internal_axis(c, d)), N, c->P.rho_L,
                                                          c->P.rho_dif, dst + d * N);
        c->launches += c->dim;
        rc = check_cuda(cudaGetLastError());
        if (!on_device) {
            if (!rc) rc = check_cuda(cudaMemcpyAsync(rho_u, dst, sizeof(double) * c->dim * (size_t)N,
                                                     cudaMemcpyDeviceToHost, c->stream));
            cudaFreeAsync(dst, c->stream);
        }
        if (rc) return rc;
    }
    return check_cuda(cudaStreamSynchronize(c->stream));
}

int lbm_get_populations(lbm_ctx* c, double* h, double* g, int on_device) {
    if (!c || !h || !g) return LBM_EINVAL;
    const int Q = c->lattice == LBM_D2Q9 ? 9 : 19;
    const size_t n = (size_t)Q * c->G.N;
    double *dh = h, *dg = g;
    if (!on_device) {
        if (cudaMallocAsync((void**)&dh, n * sizeof(double), c->stream) != cudaSuccess) {
            cudaGetLastError();
            return LBM_ENOMEM;
        }
        if (cudaMallocAsync((void**)&dg, n * sizeof(double), c->stream) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeAsync(dh, c->stream);
            return LBM_ENOMEM;
        }
    }
    int rc = check_cuda(c->K->get(c->h[c->cur], c->g[c->cur], c->G, c->P, dh, dg, c->stream));
    c->launches += 1;
    if (!rc && !on_device) {
        rc = check_cuda(cudaMemcpyAsync(h, dh, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (!rc) rc = check_cuda(cudaMemcpyAsync(g, dg, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    if (!on_device) { cudaFreeAsync(dh, c->stream); cudaFreeAsync(dg, c->stream); }
    int rs = check_cuda(cudaStreamSynchronize(c->stream));
    return rc ? rc : rs;
}

int lbm_set_populations(lbm_ctx* c, const double* h, const double* g, int on_device) {
    if (!c || !h || !g) return LBM_EINVAL;
    const int Q = c->lattice == LBM_D2Q9 ? 9 : 19;
    const size_t n = (size_t)Q * c->G.N;
    const double *dh = h, *dg = g;
    double *th = nullptr, *tg = nullptr;
    if (!on_device) {
        if (cudaMallocAsync((void**)&th, n * sizeof(double), c->stream) != cudaSuccess) {
            cudaGetLastError();
            return LBM_ENOMEM;
        }
        if (cudaMallocAsync((void**)&tg, n * sizeof(double), c->stream) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeAsync(th, c->stream);
            return LBM_ENOMEM;
        }
        cudaMemcpyAsync(th, h, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        cudaMemcpyAsync(tg, g, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        dh = th; dg = tg;
    }
    const int b = c->cur;
    int rc = check_cuda(c->K->set(c->h[b], c->g[b], c->G, c->P, dh, dg, c->stream));
    c->ghosts[b] = true;
    c->diverged = false;
    if (!rc) rc = check_cuda(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    c->launches += 1;
    if (th) { cudaFreeAsync(th, c->stream); cudaFreeAsync(tg, c->stream); }
    if (!rc) {
        rc = compute_fields(c);
        double d[4];
        if (!rc) rc = reduce_diag(c, d);
        if (!rc) {
            c->phi_target = d[0];
            c->phi_fix_count = 0;
            if (c->P.force_mode == 1) c->P.rho_bar = c->P.rho_L + c->P.rho_dif * d[0] / (double)c->G.N;
        }
    }
    int rs = check_cuda(cudaStreamSynchronize(c->stream));
    return rc ? rc : rs;
}

int lbm_diagnostics(lbm_ctx* c, double out[4]) {
    lbm::NvtxRange range("lbm_diagnostics");
    if (!c || !out) return LBM_EINVAL;
    int rc = compute_fields(c);
    if (rc) return rc;
    rc = reduce_diag(c, out);
    if (rc) return rc;
    int err = 0;
    if (check_cuda(cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost))) return LBM_ECUDA;
    if (err) return LBM_ETIMEOUT;
    if (out[3] > 0 || out[2] > 0.3) {
        // sticky: lbm_step refuses to advance a diverged state until it is
        // replaced (lbm_init_fields, lbm_set_populations)
        c->diverged = true;
        return LBM_EDIVERGED;
    }
    return LBM_OK;
}

int lbm_laplace(lbm_ctx* c, const double centre[3], double r_in, double r_out, double* dP) {
    if (!c || !centre || !dP) return LBM_EINVAL;
    int rc = compute_fields(c);
    if (rc) return rc;
    double cc[3] = {centre[0], centre[1], centre[2]};
    if (c->lattice == LBM_D2Q9) { cc[1] = 0.0; cc[2] = centre[1]; }
    const int nb = partial_blocks(c);
    double* res = c->partial + 4 * (size_t)c->n_partial_blocks;
    laplace_partial_kernel<<<nb, kRedThreads, 0, c->stream>>>(f_P(c), c->G, cc[0], cc[1], cc[2], r_in, r_out,
                                                             c->partial);
    finish_kernel<<<1, 32, 0, c->stream>>>(c->partial, nb, 4, 0, res);
    c->launches += 2;
    if (check_cuda(cudaGetLastError())) return LBM_ECUDA;
    double h[4];
    if (check_cuda(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, c->stream))) return LBM_ECUDA;
    if (check_cuda(cudaStreamSynchronize(c->stream))) return LBM_ECUDA;
    if (h[1] <= 0 || h[3] <= 0) return LBM_EINVAL;
    *dP = h[0] / h[1] - h[2] / h[3];
    return LBM_OK;
}

int lbm_autotune(lbm_ctx* c, int steps, int* best_tile, int* best_lz, double* best_ms) {
    if (!c || steps < 1 || c->owner) return LBM_EINVAL;
    // the trials advance the state: keep a copy and restore it afterwards
    const int Q = c->lattice == LBM_D2Q9 ? 9 : 19;
    const size_t bytes = c->elem * (size_t)Q * (size_t)c->G.NP;
    void* save_h = nullptr;
    void* save_g = nullptr;
    if (cudaMallocAsync(&save_h, bytes, c->stream) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ENOMEM;
    }
    if (cudaMallocAsync(&save_g, bytes, c->stream) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(save_h, c->stream);
        return LBM_ENOMEM;
    }
    const bool saved_ghosts = c->ghosts[c->cur];
    const bool saved_diverged = c->diverged;
    const int saved_tile = c->tile, saved_lz = c->lz, saved_fix_count = c->phi_fix_count;
    int rc = check_cuda(cudaMemcpyAsync(save_h, c->h[c->cur], bytes, cudaMemcpyDeviceToDevice, c->stream));
    if (!rc) rc = check_cuda(cudaMemcpyAsync(save_g, c->g[c->cur], bytes, cudaMemcpyDeviceToDevice, c->stream));
    const bool saved = rc == LBM_OK;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int lzs[4] = {4, 8, 16, 32};
    int bt = c->tile, bl = c->lz;
    float bms = 1e30f;
    for (int t = 0; t < c->K->n_tiles && !rc; ++t) {
        if (!c->K->tile_ok(t, c->G)) continue;
        for (int k = 0; k < 4 && !rc; ++k) {
            c->tile = t;
            c->lz = lzs[k];
            rc = lbm_step(c, 2);
            if (rc) break;
            cudaEventRecord(e0, c->stream);
            rc = lbm_step(c, steps);
            cudaEventRecord(e1, c->stream);
            if (rc) break;
            rc = check_cuda(cudaEventSynchronize(e1));
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < bms) { bms = ms; bt = t; bl = lzs[k]; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the state goes back whether or not a trial failed (a failed trial keeps
    // the tile the context had)
    if (saved) {
        int rr = check_cuda(cudaMemcpyAsync(c->h[0], save_h, bytes, cudaMemcpyDeviceToDevice, c->stream));
        if (!rr) rr = check_cuda(cudaMemcpyAsync(c->g[0], save_g, bytes, cudaMemcpyDeviceToDevice, c->stream));
        c->cur = 0;
        c->ghosts[0] = saved_ghosts;
        c->ghosts[1] = false;
        c->diverged = saved_diverged;
        c->phi_fix_count = saved_fix_count;
        if (!rc) rc = rr;
    }
    cudaFreeAsync(save_h, c->stream);
    cudaFreeAsync(save_g, c->stream);
    c->tile = rc ? saved_tile : bt;
    c->lz = rc ? saved_lz : bl;
    if (!rc) rc = check_cuda(cudaStreamSynchronize(c->stream));
    if (best_tile) *best_tile = bt;
    if (best_lz) *best_lz = bl;
    if (best_ms) *best_ms = (double)bms / steps;
    return rc;
}

long long lbm_launch_count(const lbm_ctx* c) { return c ? c->launches : 0; }

void* lbm_stream(const lbm_ctx* c) { return c ? (void*)c->stream : nullptr; }

int lbm_set_phi_correction(lbm_ctx* c, int every) {
    if (!c || every < 0 || c->owner) return LBM_EINVAL;
    if (every > 0) {
        int rc = ensure_scratch(c);
        if (rc) return rc;
        if (!c->d_fix && cudaMallocAsync((void**)&c->d_fix, sizeof(double) * (kFixBlocks + 1), c->stream) != cudaSuccess) {
            cudaGetLastError();
            c->d_fix = nullptr;
            return LBM_ENOMEM;
        }
    }
    c->phi_fix_every = every;
    c->phi_fix_count = 0;
    return LBM_OK;
}

int lbm_set_wall_velocity(lbm_ctx* c, int axis, int side, const double u[3]) {
    if (!c || !u || side < 0 || side > 1) return LBM_EINVAL;
    if (axis < 0 || axis >= c->dim) return LBM_EINVAL;
    if (c->grid.bc[axis] != LBM_WALL) return LBM_EINVAL;       // only walls move
    if (u[axis] != 0.0) return LBM_EINVAL;                      // sliding: no normal component
    for (int d = 0; d < c->dim; ++d)
        if (!std::isfinite(u[d])) return LBM_EINVAL;
    const int ia = internal_axis(c, axis);
    double ui[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < c->dim; ++d) ui[internal_axis(c, d)] = u[d];
    for (int k = 0; k < 3; ++k) c->P.uw[ia][side][k] = ui[k];
    int moving = 0;
    for (int a = 0; a < 3; ++a)
        for (int sd = 0; sd < 2; ++sd)
            for (int k = 0; k < 3; ++k) moving |= c->P.uw[a][sd][k] != 0.0;
    c->P.moving = moving;
    c->pversion += 1;
    return LBM_OK;
}

int lbm_set_wait_limit(lbm_ctx* c, long long polls) {
    if (!c || polls < 0) return LBM_EINVAL;
    c->wait_polls = (long)polls;
    return LBM_OK;
}

// Step tile shape and z-chunk length (used by the tuner and the tests).
int lbm_set_tile(lbm_ctx* c, int tile, int lz) {
    if (!c || tile < 0 || tile >= c->K->n_tiles || lz < 1 || c->owner) return LBM_EINVAL;
    if (!c->K->tile_ok(tile, c->G)) return LBM_ENOTSUP;
    c->tile = tile;
    c->lz = lz;
    return LBM_OK;
}

int lbm_get_tile(const lbm_ctx* c, int* tile, int* lz, int* tx, int* ty) {
    if (!c) return LBM_EINVAL;
    if (tile) *tile = c->tile;
    if (lz) *lz = c->lz;
    if (tx) *tx = c->K->tile_tx[c->tile];
    if (ty) *ty = c->K->tile_ty[c->tile];
    return LBM_OK;
}

}  // extern "C"
