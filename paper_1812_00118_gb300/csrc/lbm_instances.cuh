// Kernel launchers for one lattice, all storage types.  Included by exactly
// one translation unit per lattice (lbm_d2q9.cu, lbm_d3q19.cu) so that the
// two lattices compile in parallel.
#pragma once
#include "lbm_internal.h"

namespace lbm {

template <int LAT, int ST, int TX, int TY, int MINB>
cudaError_t launch_step_tile(const void* hin, const void* gin, void* hout, void* gout, const Geom& G,
                             const Phys& p, int lz, cudaStream_t s) {
    using S = typename Storage<ST>::S;
    dim3 block(TX, TY);
    dim3 grid((G.NX + TX - 1) / TX, (G.NY + TY - 1) / TY, (G.NZ + lz - 1) / lz);
    step_kernel<LAT, ST, TX, TY, MINB><<<grid, block, 0, s>>>(
        dir_ptrs<S, Lattice<LAT>::Q>(hin, gin, hout, gout, G.NP), G, phys_as<typename Storage<ST>::R>(p), lz);
    return cudaGetLastError();
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <int LAT, int ST>
struct Launchers {
    using S = typename Storage<ST>::S;
    static constexpr int Q = Lattice<LAT>::Q;
    static cudaError_t phi(const void* hin, const Geom& G, const Phys& p, double* out, cudaStream_t s) {
        phi_kernel<LAT, ST><<<blocks_for(G.N, 256), 256, 0, s>>>(
            dir_ptrs<S, Q>(hin, hin, nullptr, nullptr, G.NP), G, p, out);
        return cudaGetLastError();
    }
    static cudaError_t macro(const void* gin, const Geom& G, const Phys& p, const double* phi, double* P,
                             double* ux, double* uy, double* uz, cudaStream_t s) {
        macro_kernel<LAT, ST><<<blocks_for(G.N, 256), 256, 0, s>>>(
            dir_ptrs<S, Q>(gin, gin, nullptr, nullptr, G.NP), G, phys_as<double>(p), phi, P, ux, uy, uz);
        return cudaGetLastError();
    }
    static cudaError_t init(void* hout, void* gout, const Geom& G, const Phys& p, const double* phi,
                            const double* ux, const double* uy, const double* uz, const double* P,
                            cudaStream_t s) {
        init_kernel<LAT, ST><<<blocks_for(G.N, 256), 256, 0, s>>>(
            dir_ptrs<S, Q>(hout, gout, hout, gout, G.NP), G, p, phi, ux, uy, uz, P);
        return cudaGetLastError();
    }
    static cudaError_t get(const void* hin, const void* gin, const Geom& G, const Phys& p, double* h, double* g,
                           cudaStream_t s) {
        get_kernel<LAT, ST><<<blocks_for(G.N, 256), 256, 0, s>>>(
            dir_ptrs<S, Q>(hin, gin, nullptr, nullptr, G.NP), G, p, h, g);
        return cudaGetLastError();
    }
    static cudaError_t set(void* hout, void* gout, const Geom& G, const Phys& p, const double* h,
                           const double* g, cudaStream_t s) {
        set_kernel<LAT, ST><<<blocks_for(G.N, 256), 256, 0, s>>>(
            dir_ptrs<S, Q>(hout, gout, hout, gout, G.NP), G, p, h, g);
        return cudaGetLastError();
    }
};

}  // namespace lbm
