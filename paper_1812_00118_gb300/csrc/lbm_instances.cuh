// Kernel launchers of one (lattice, storage) pair.  Included by
// lbm_tables.cu, which the build compiles once per pair (LBM_LAT, LBM_ST) so
// that the eight pairs compile in parallel.
#pragma once
#include <cudaTypedefs.h>

#include <new>

#include "lbm_internal.h"
#include "lbm_tma.cuh"

namespace lbm {

// Values a launcher computes once per device and kernel variant (resident
// CTAs, function attributes): kept per device ordinal, since two devices of
// one process may differ.  Slot value 0 means "not computed yet".
constexpr int kMaxDevices = 64;
struct PerDevice {
    int v[kMaxDevices][2] = {};
};

template <typename F>
cudaError_t per_device(PerDevice& cache, int variant, F compute, int* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return compute(out);
    int& c = cache.v[dev][variant];
    if (c == 0) {
        int val = 0;
        e = compute(&val);
        if (e != cudaSuccess) return e;
        c = val + 1;
    }
    *out = c - 1;
    return cudaSuccess;
}

// Resident-slot count of a kernel on the current device: SMs x occupancy.
template <typename K>
cudaError_t resident_slots(K kern, int threads, size_t smem, int* out) {
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    *out = sms * occ;
    return cudaSuccess;
}

// Grid = tile columns x chunks along z.  Chunks of lz planes, or with BAL
// (one-wave launch) as many equal chunks as the resident slots (occupancy x
// SMs, looked up once per instantiation) allow for every column, with at
// least lz planes each.
template <int LAT, int ST, int TX, int TY, int MINB, bool HOIST, bool BAL>
cudaError_t launch_step_tile(const StepArgs& a) {
    using S = typename Storage<ST>::S;
    const Geom& G = a.G;
    const bool walls = G.wall[0] || G.wall[1] || G.wall[2];
    auto kern = walls ? step_kernel<LAT, ST, TX, TY, MINB, HOIST, BAL, true>
                      : step_kernel<LAT, ST, TX, TY, MINB, HOIST, BAL, false>;
    dim3 block(TX, TY);
    dim3 grid((G.NX + TX - 1) / TX, (G.NY + TY - 1) / TY, (G.NZ + a.lz - 1) / a.lz);
    if (BAL) {
        static PerDevice slots_cache;
        int slots = 0;
        cudaError_t e = per_device(slots_cache, walls ? 1 : 0,
                                   [&](int* v) { return resident_slots(kern, TX * TY, 0, v); }, &slots);
        if (e != cudaSuccess) return e;
        long long nzc = slots / ((long long)grid.x * grid.y);
        const long long by_lz = (G.NZ + a.lz - 1) / a.lz;
        if (nzc > by_lz) nzc = by_lz;
        if (nzc < 1) nzc = 1;
        grid.z = (unsigned)nzc;
    }
    const auto d = dir_ptrs<S, Lattice<LAT>::Q>(a.hin, a.gin, a.hout, a.gout, G.NP);
    const auto ph = phys_as<typename Storage<ST>::R>(a.p);
    kern<<<grid, block, 0, a.stream>>>(d, G, ph, a.lz);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- asynchronous-load tiles (FP32)
template <int LAT, int TX, int TY>
constexpr size_t async_smem_bytes() { return sizeof(AsyncSmem<LAT, TX, TY>); }

template <int LAT, int ST, int TX, int TY>
bool async_tile_ok(const Geom&) {
    return ST == ST_F32 && async_smem_bytes<LAT, TX, TY>() <= 227 * 1024;
}

template <int LAT, int ST, int TX, int TY, int MINB>
cudaError_t launch_async_tile(const StepArgs& a) {
    if constexpr (ST != ST_F32) {
        return cudaErrorNotSupported;
    } else {
        const Geom& G = a.G;
        const bool walls = G.wall[0] || G.wall[1] || G.wall[2];
        auto kern = walls ? step_async_kernel<LAT, TX, TY, MINB, true> : step_async_kernel<LAT, TX, TY, MINB, false>;
        constexpr size_t bytes = async_smem_bytes<LAT, TX, TY>();
        static PerDevice attr_cache;
        int done = 0;
        cudaError_t e = per_device(attr_cache, walls ? 1 : 0, [&](int* v) {
            *v = 1;
            return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        }, &done);
        if (e != cudaSuccess) return e;
        dim3 grid((G.NX + TX - 1) / TX, (G.NY + TY - 1) / TY, (G.NZ + a.lz - 1) / a.lz);
        kern<<<grid, dim3(TX, TY), bytes, a.stream>>>(dir_ptrs<float, Lattice<LAT>::Q>(a.hin, a.gin, a.hout, a.gout, G.NP),
                                                      G, phys_as<float>(a.p), a.lz);
        return cudaGetLastError();
    }
}

// ---------------------------------------------------------------- batches
// One CTA per resident slot (occupancy x SMs, looked up once per
// instantiation), at most one per work item.
template <int LAT, int ST, int TX, int MINB, bool HOIST>
cudaError_t launch_batch_tile(const BatchArgs& a) {
    using S = typename Storage<ST>::S;
    using R = typename Storage<ST>::R;
    auto kern = batch_step_kernel<LAT, ST, TX, MINB, HOIST>;
    static PerDevice slots_cache;
    int slots = 0;
    cudaError_t e = per_device(slots_cache, 0, [&](int* v) { return resident_slots(kern, TX, 0, v); }, &slots);
    if (e != cudaSuccess) return e;
    if (a.n_items < 1) return cudaSuccess;
    const int nb = a.n_items < slots ? a.n_items : slots;
    kern<<<nb, TX, 0, a.stream>>>(dir_ptrs<S, Lattice<LAT>::Q>(a.hin, a.gin, a.hout, a.gout, a.NP),
                                  (const BatchCase<R>*)a.cases, (const BatchItem*)a.items, a.n_items, a.counters);
    return cudaGetLastError();
}

template <int ST>
cudaError_t batch_upload(const Geom* G, const Phys* P, int n, void* d_cases, cudaStream_t s) {
    using R = typename Storage<ST>::R;
    BatchCase<R>* h = new (std::nothrow) BatchCase<R>[n > 0 ? n : 1];
    if (!h) return cudaErrorMemoryAllocation;
    for (int i = 0; i < n; ++i) {
        h[i].G = G[i];
        h[i].p = phys_as<R>(P[i]);
    }
    cudaError_t e = cudaMemcpyAsync(d_cases, h, sizeof(BatchCase<R>) * (size_t)n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    delete[] h;
    return e;
}

// ---------------------------------------------------------------- bulk-copy tiles
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    }
    return fn;
}

template <int ST> struct TmaType;
template <> struct TmaType<ST_F64> { static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT64; };
template <> struct TmaType<ST_F32> { static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; };
template <> struct TmaType<ST_F16S> { static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; };
template <> struct TmaType<ST_BF16S> { static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; };

// 4-D view (x, y, z, population) of one ghost-padded population array set.
template <int LAT, int ST, int TX, int TY>
cudaError_t make_maps_tile(TmaMaps* m, const void* h, const void* g, const Geom& G) {
    using C = TmaCfg<LAT, ST, TX, TY>;
    auto enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t es = C::ES;
    cuuint64_t dims[4] = {(cuuint64_t)G.PX, (cuuint64_t)G.PY, (cuuint64_t)G.PZ, (cuuint64_t)Lattice<LAT>::Q};
    cuuint64_t strides[3] = {(cuuint64_t)G.PX * es, (cuuint64_t)G.PXY * es, (cuuint64_t)G.NP * es};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    struct { CUtensorMap* map; const void* base; cuuint32_t rows, k; } jobs[4] = {
        {&m->h3, h, (cuuint32_t)C::RH, 3}, {&m->h1, h, (cuuint32_t)C::RH, 1},
        {&m->g3, g, (cuuint32_t)C::RG, 3}, {&m->g1, g, (cuuint32_t)C::RG, 1}};
    for (auto& jb : jobs) {
        cuuint32_t box[4] = {(cuuint32_t)C::BX, jb.rows, 1, jb.k};
        CUresult r = enc(jb.map, TmaType<ST>::v, 4, const_cast<void*>(jb.base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

template <int LAT, int ST, int TX, int TY>
bool tma_tile_ok(const Geom& G) {
    using C = TmaCfg<LAT, ST, TX, TY>;
    // shared memory of one CTA, box limits, and the periodic images the
    // halo of a tile reads (two cells deep) must exist: a ghost band on
    // every periodic axis (lbm_create_ex with LBM_CREATE_GHOST_BAND)
    if (C::smem_bytes > 227 * 1024 || C::BX > 256 || C::RH > 256) return false;
    if (G.NX < 2 * kRep || (Lattice<LAT>::kHasY && G.NY < 2 * kRep)) return false;
    if (!G.wall[0] && G.GX < kRep) return false;
    if (Lattice<LAT>::kHasY && !G.wall[1] && G.GY < kRep) return false;
    return tensor_map_encoder() != nullptr;
}

template <int LAT, int ST, int TX, int TY, int MINB>
cudaError_t launch_tma_tile(const StepArgs& a) {
    using S = typename Storage<ST>::S;
    using C = TmaCfg<LAT, ST, TX, TY>;
    const bool walls = a.G.wall[0] || a.G.wall[1] || a.G.wall[2];
    auto kern = walls ? step_tma_kernel<LAT, ST, TX, TY, MINB, true> : step_tma_kernel<LAT, ST, TX, TY, MINB, false>;
    static PerDevice slots_cache;
    int slots = 0;
    cudaError_t e = per_device(slots_cache, walls ? 1 : 0, [&](int* v) {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::smem_bytes);
        return r != cudaSuccess ? r : resident_slots(kern, TX * TY, C::smem_bytes, v);
    }, &slots);
    if (e != cudaSuccess) return e;
    const Geom& G = a.G;
    const int chunk = a.lz > 0 ? a.lz : 8;
    const long long work = (long long)((G.NX + TX - 1) / TX) * ((G.NY + TY - 1) / TY) * ((G.NZ + chunk - 1) / chunk);
    long long grid = slots;
    if (grid > work) grid = work;
    kern<<<(unsigned)grid, dim3(TX, TY), C::smem_bytes, a.stream>>>(
        *a.maps, dir_ptrs<S, Lattice<LAT>::Q>(a.hin, a.gin, a.hout, a.gout, G.NP), G,
        phys_as<typename Storage<ST>::R>(a.p), chunk, a.error_flag, a.wait_polls);
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
            dir_ptrs<S, Q>(gin, gin, nullptr, nullptr, G.NP), G, phys_as<typename Storage<ST>::R>(p), phi, P, ux, uy,
            uz);
        return cudaGetLastError();
    }
    static cudaError_t init(void* hout, void* gout, const Geom& G, const Phys& p, const double* phi,
                            const double* ux, const double* uy, const double* uz, const double* P, int neq,
                            cudaStream_t s) {
        init_kernel<LAT, ST><<<blocks_for(G.N, 256), 256, 0, s>>>(
            dir_ptrs<S, Q>(hout, gout, hout, gout, G.NP), G, phys_as<typename Storage<ST>::R>(p), phi, ux, uy, uz, P,
            neq);
        return cudaGetLastError();
    }
    static cudaError_t get(const void* hin, const void* gin, const Geom& G, const Phys& p, double* h, double* g,
                           cudaStream_t s) {
        get_kernel<LAT, ST><<<blocks_for(G.N, 256), 256, 0, s>>>(
            dir_ptrs<S, Q>(hin, gin, nullptr, nullptr, G.NP), G, p, h, g);
        return cudaGetLastError();
    }
    static cudaError_t halo(void* hout, void* gout, const Geom& G, cudaStream_t s) {
        const int Ry = G.GY < kRep ? G.GY : kRep;
        const long long band = (long long)(G.NX + 2 * kRep) * (G.NY + 2 * Ry);
        const long long n = (band - (long long)G.NX * G.NY) * G.NZ + (G.wall[2] ? 2 * band : 0);
        if (G.wall[0] && (G.wall[1] || G.GY == 0)) return cudaSuccess;   // no periodic x/y axis
        halo_kernel<LAT, ST><<<blocks_for(n, 256), 256, 0, s>>>(dir_ptrs<S, Q>(hout, gout, hout, gout, G.NP), G);
        return cudaGetLastError();
    }
    static cudaError_t shift_rest(void* h, const Geom& G, const Phys& p, const double* delta, cudaStream_t s) {
        shift_rest_kernel<LAT, ST><<<blocks_for(G.N, 256), 256, 0, s>>>((S*)h, G, phys_as<typename Storage<ST>::R>(p),
                                                                         delta);
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
