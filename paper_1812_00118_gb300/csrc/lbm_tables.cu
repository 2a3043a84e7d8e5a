// Kernel instantiations for ONE (lattice, storage) pair, selected at compile
// time by LBM_LAT (0 = D2Q9, 1 = D3Q19) and LBM_ST (lbm::ST_*).  The build
// compiles this file once per pair so the eight pairs compile in parallel.
#include "lbm_instances.cuh"

#ifndef LBM_LAT
#error "LBM_LAT must be defined"
#endif
#ifndef LBM_ST
#error "LBM_ST must be defined"
#endif

namespace lbm {
namespace {

#if LBM_LAT == 1
// D3Q19: CTA shapes in the x-y plane
cudaError_t step_dispatch(const void* hin, const void* gin, void* hout, void* gout, const Geom& G, const Phys& p,
                          int tile, int lz, cudaStream_t s) {
    switch (tile) {
        case 0: return launch_step_tile<1, LBM_ST, 32, 4, 4>(hin, gin, hout, gout, G, p, lz, s);
        case 1: return launch_step_tile<1, LBM_ST, 32, 8, 2>(hin, gin, hout, gout, G, p, lz, s);
        case 2: return launch_step_tile<1, LBM_ST, 64, 4, 2>(hin, gin, hout, gout, G, p, lz, s);
        case 3: return launch_step_tile<1, LBM_ST, 32, 4, 5>(hin, gin, hout, gout, G, p, lz, s);
        default: return cudaErrorInvalidValue;
    }
}
const KernelTable kTable = {step_dispatch, Launchers<1, LBM_ST>::phi, Launchers<1, LBM_ST>::macro,
                            Launchers<1, LBM_ST>::init, Launchers<1, LBM_ST>::get, Launchers<1, LBM_ST>::set,
                            4, {32, 32, 64, 32}, {4, 8, 4, 4}};
#else
// D2Q9: the 2-D grid is stored as (nx, 1, ny); CTAs are rows along x
cudaError_t step_dispatch(const void* hin, const void* gin, void* hout, void* gout, const Geom& G, const Phys& p,
                          int tile, int lz, cudaStream_t s) {
    switch (tile) {
        case 0: return launch_step_tile<0, LBM_ST, 128, 1, 4>(hin, gin, hout, gout, G, p, lz, s);
        case 1: return launch_step_tile<0, LBM_ST, 256, 1, 2>(hin, gin, hout, gout, G, p, lz, s);
        case 2: return launch_step_tile<0, LBM_ST, 64, 1, 8>(hin, gin, hout, gout, G, p, lz, s);
        case 3: return launch_step_tile<0, LBM_ST, 32, 1, 8>(hin, gin, hout, gout, G, p, lz, s);
        default: return cudaErrorInvalidValue;
    }
}
const KernelTable kTable = {step_dispatch, Launchers<0, LBM_ST>::phi, Launchers<0, LBM_ST>::macro,
                            Launchers<0, LBM_ST>::init, Launchers<0, LBM_ST>::get, Launchers<0, LBM_ST>::set,
                            4, {128, 256, 64, 32}, {1, 1, 1, 1}};
#endif

}  // namespace

const KernelTable* LBM_TABLE_NAME(LBM_LAT, LBM_ST)() { return &kTable; }

}  // namespace lbm
