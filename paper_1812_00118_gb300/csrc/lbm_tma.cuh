// Fused step with bulk tensor copies (TMA) into a shared-memory pipeline.
//
// Same arithmetic as step_kernel (lbm_kernels.cuh); only the way the pulled
// populations reach the threads differs.  The ghost-padded layout makes
// every pull of a tile a dense box of the padded array: for a group of
// velocities with the same (c_y, c_z) the pulled values of a TX x TY tile
// (plus a one-node halo for h) are the box
//     x in [x0 - A, x0 + TX + A), rows y0 - c_y - halo ..., plane z - c_z,
// in population coordinates [first, first + size), where A = 16 bytes of
// storage keeps the box start aligned.  Each thread reads its pulled value
// at column (tx + A - c_x) of its direction's slab.
//
// Pipeline per CTA, planes z0..z1-1 of one tile (q counts h planes from
// z0 - 1): h planes q, q+1, q+2 are resident or in flight in a three-slot
// ring, g planes j, j+1 in a two-slot ring.  Iteration j (plane z = z0 + j):
//   barrier; thread 0 issues h plane q = j+3 and g plane j+1;
//   wait h[j+2] and fill phi of plane z+1 (tile + halo) into the phi ring;
//   wait g[j]; barrier; collide plane z from h[j+1], g[j] and the phi ring.
// Every wait is bounded: on timeout a flag is raised, the CTA waits
// (bounded) for its copies in flight and returns.
//
// Work items are (z chunk, tile) pairs ordered chunk-major, dealt round-robin
// to persistent CTAs: the CTAs running at one time hold neighbouring tiles
// at the same depth, so the halo rows one tile re-reads are still in L2.
#pragma once
#include <cuda.h>

#include "lbm_kernels.cuh"

namespace lbm {

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Bounded wait: false if the phase did not complete within `polls` tries.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long polls) {
    for (long it = 0; it < polls; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// Polls of the wait that drains the copies a failed CTA still has in flight:
// far more than a bulk copy of a few tens of kilobytes takes to land.
constexpr long kDrainPolls = 1L << 22;
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

// ------------------------------------------------------------ layout
// Shared-memory layout of one pipeline stage of one array: for each
// velocity group a block of size * rows * BX elements (direction-major),
// each group starting on a 128-byte boundary.
template <int LAT, int ROWS, int BX, int ES>
struct StageLayout {
    using L = Lattice<LAT>;
    static constexpr int dir_bytes = ROWS * BX * ES;
    __host__ __device__ static constexpr int group_offset(int g) {
        int off = 0;
        for (int k = 0; k < g; ++k) off += (L::groups[k][1] * dir_bytes + 127) / 128 * 128;
        return off;
    }
    static constexpr int bytes = group_offset(L::NG);
    // byte offset of direction i's slab
    __host__ __device__ static constexpr int dir_offset(int i) {
        for (int g = 0; g < L::NG; ++g)
            if (i >= L::groups[g][0] && i < L::groups[g][0] + L::groups[g][1])
                return group_offset(g) + (i - L::groups[g][0]) * dir_bytes;
        return -1;
    }
};

// Tensor maps of the current input buffers: boxes of 3 and of 1 velocity,
// h-shaped (TY + 2 halo rows) and g-shaped (TY rows).
struct TmaMaps {
    CUtensorMap h3, h1, g3, g1;
};

template <int LAT, int ST, int TX, int TY>
struct TmaCfg {
    using L = Lattice<LAT>;
    using S = typename Storage<ST>::S;
    static constexpr int ES = (int)sizeof(S);
    static constexpr int A = 16 / ES;                      // elements per 16 bytes
    static constexpr int HY = L::kHasY ? 1 : 0;
    static constexpr int BX = TX + 2 * A;                  // box width (x)
    static constexpr int RH = TY + 2 * HY;                 // h box rows
    static constexpr int RG = TY;                          // g box rows
    using HL = StageLayout<LAT, RH, BX, ES>;
    using GL = StageLayout<LAT, RG, BX, ES>;
    static constexpr int NHS = 3, NGS = 2;                 // ring slots
    static constexpr int SX = TX + 2, SY = TY + 2 * HY;    // phi tile with halo
    static constexpr int phi_bytes = 4 * SY * SX * (int)sizeof(typename Storage<ST>::R);
    static constexpr int off_h = 0;
    static constexpr int off_g = NHS * HL::bytes;
    static constexpr int off_phi = off_g + NGS * GL::bytes;
    static constexpr int off_bar = (off_phi + phi_bytes + 15) / 16 * 16;
    static constexpr int smem_bytes = off_bar + (NHS + NGS) * 8 + 128;   // + alignment slack
};

// ------------------------------------------------------------ kernel
template <int LAT, int ST, int TX, int TY, int MINB, bool WALLS>
__global__ void __launch_bounds__(TX * TY, MINB)
step_tma_kernel(const __grid_constant__ TmaMaps maps, const DirPtrs<typename Storage<ST>::S, Lattice<LAT>::Q> D,
                Geom G, PhysT<typename Storage<ST>::R> p, int chunk, int* error_flag, long wait_polls) {
    using L = Lattice<LAT>;
    using St = Storage<ST>;
    using S = typename St::S;
    using R = typename St::R;
    using C = TmaCfg<LAT, ST, TX, TY>;
    constexpr int Q = L::Q;
    constexpr int HY = C::HY;
    constexpr int A = C::A;
    extern __shared__ unsigned char smem_raw[];
    // 128-byte aligned base
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    R(*phis)[C::SY][C::SX] = reinterpret_cast<R(*)[C::SY][C::SX]>(smem + C::off_phi);
    uint64_t* hbar = reinterpret_cast<uint64_t*>(smem + C::off_bar);
    uint64_t* gbar = hbar + C::NHS;

    const int tid = threadIdx.x + TX * threadIdx.y;
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (tid == 0) {
        for (int s = 0; s < C::NHS; ++s) mbar_init(&hbar[s], 1);
        for (int s = 0; s < C::NGS; ++s) mbar_init(&gbar[s], 1);
        fence_barrier_init();
    }
    __syncthreads();

    const int ntx = (G.NX + TX - 1) / TX, nty = (G.NY + TY - 1) / TY;
    const int ntiles = ntx * nty;
    const int nchunks = (G.NZ + chunk - 1) / chunk;
    const long long items = (long long)ntiles * nchunks;   // (chunk, tile), tile fastest
    uint32_t hcount = 0, gcount = 0;                          // ring uses so far (parity = use & 1)
    // uses issued so far (CTA-uniform: every thread follows the issue
    // decisions of thread 0); all but the last use of a slot have been waited
    // for when a wait gives up
    uint32_t hiss = 0, giss = 0;
    bool failed = false;

    // issue the h box set of fill plane zf (unwrapped) into h slot s
    auto issue_h = [&](int x0, int y0, int zf, int s) {
        const int zz = stencil_coord(zf, G.NZ, G.wall[2]);   // plane whose pulls fill this slot
        mbar_arrive_expect_tx(&hbar[s], (uint32_t)(Q * C::HL::dir_bytes));
        unsigned char* base = smem + C::off_h + s * C::HL::bytes;
        Unroll<0, L::NG>::run([&](auto gc) {
            constexpr int g = decltype(gc)::value;
            constexpr int first = L::groups[g][0], cnt = L::groups[g][1], cy = L::groups[g][2], cz = L::groups[g][3];
            constexpr int goff = C::HL::group_offset(g);
            const int row = y0 - HY - cy + G.GY;
            const int plane = pull_plane(G, zz - cz) + G.GZ;
            tma_load_4d(base + goff, cnt == 3 ? &maps.h3 : &maps.h1, x0 + G.GX - A, row, plane, first, &hbar[s]);
        });
    };
    auto issue_g = [&](int x0, int y0, int z, int s) {
        mbar_arrive_expect_tx(&gbar[s], (uint32_t)(Q * C::GL::dir_bytes));
        unsigned char* base = smem + C::off_g + s * C::GL::bytes;
        Unroll<0, L::NG>::run([&](auto gc) {
            constexpr int g = decltype(gc)::value;
            constexpr int first = L::groups[g][0], cnt = L::groups[g][1], cy = L::groups[g][2], cz = L::groups[g][3];
            constexpr int goff = C::GL::group_offset(g);
            const int row = y0 - cy + G.GY;
            const int plane = pull_plane(G, z - cz) + G.GZ;
            tma_load_4d(base + goff, cnt == 3 ? &maps.g3 : &maps.g1, x0 + G.GX - A, row, plane, first, &gbar[s]);
        });
    };
    // phi of the h slot s into phi ring slot r, then mirror halo cells behind walls
    auto fill = [&](int s, int r, int x0, int y0) {
        const S* hb = reinterpret_cast<const S*>(smem + C::off_h + s * C::HL::bytes);
        for (int k = tid; k < C::SX * C::SY; k += TX * TY) {
            const int lx = k % C::SX, ly = k / C::SX;
            PhiSum<R> phi;
            Unroll<0, Q>::run([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                constexpr int off = C::HL::dir_offset(i) / C::ES + A - 1 - L::cx[i];
                constexpr double W = L::w[i];
                phi.add(St::load(hb[off + ly * C::BX + lx], (R)W * p.h_shift, (R)1));
            });
            phis[r][ly][lx] = phi.value();
        }
        if (G.wall[0] || (HY && G.wall[1])) {
            __syncthreads();
            if (G.wall[0]) {
                for (int ly = tid; ly < C::SY; ly += TX * TY) {
                    if (x0 == 0) phis[r][ly][0] = phis[r][ly][1];
                    const int lr = G.NX - x0 + 1;   // first halo column past the last node
                    if (lr < C::SX) phis[r][ly][lr] = phis[r][ly][lr - 1];
                }
            }
            if (HY && G.wall[1]) {
                __syncthreads();
                for (int lx = tid; lx < C::SX; lx += TX * TY) {
                    if (y0 == 0) phis[r][0][lx] = phis[r][1][lx];
                    const int lr = G.NY - y0 + HY;
                    if (lr < C::SY) phis[r][lr][lx] = phis[r][lr - 1][lx];
                }
            }
        }
    };

    for (long long it = blockIdx.x; it < items && !failed; it += gridDim.x) {
        const int tile = (int)(it % ntiles);
        const int z0 = (int)(it / ntiles) * chunk;
        const int z1 = min(z0 + chunk, G.NZ);
        const int LZ = z1 - z0;
        const int x0 = (int)(tile % ntx) * TX, y0 = (int)(tile / ntx) * TY;
        const int x = x0 + tx, y = y0 + ty;
        const bool active = x < G.NX && y < G.NY;
        const int rb = (y + G.GY) * G.PX + x + G.GX;
        const uint32_t hb0 = hcount, gb0 = gcount;
        // prologue: h planes q = 0, 1, 2 (z0-1, z0, z0+1) and g plane 0
        __syncthreads();
        if (tid == 0) {
            fence_proxy_async();
            for (int q = 0; q < 3 && q <= LZ + 1; ++q) issue_h(x0, y0, z0 - 1 + q, (hb0 + q) % 3);
            issue_g(x0, y0, z0, gb0 % 2);
        }
        hiss = hb0 + (uint32_t)min(3, LZ + 2);
        giss = gb0 + 1;
        bool ok = mbar_wait(&hbar[hb0 % 3], ((hb0) / 3) & 1, wait_polls);
        fill(hb0 % 3, 0, x0, y0);
        ok = ok && mbar_wait(&hbar[(hb0 + 1) % 3], ((hb0 + 1) / 3) & 1, wait_polls);
        fill((hb0 + 1) % 3, 1, x0, y0);
        if (__syncthreads_or(!ok)) { failed = true; break; }
        for (int j = 0; j < LZ; ++j) {
            const int z = z0 + j;
            __syncthreads();
            if (tid == 0) {
                fence_proxy_async();
                if (j + 3 <= LZ + 1) issue_h(x0, y0, z0 - 1 + j + 3, (hb0 + j + 3) % 3);
                if (j + 1 < LZ) issue_g(x0, y0, z + 1, (gb0 + j + 1) % 2);
            }
            if (j + 3 <= LZ + 1) hiss = hb0 + (uint32_t)(j + 4);
            if (j + 1 < LZ) giss = gb0 + (uint32_t)(j + 2);
            const uint32_t qh = hb0 + j + 2, qg = gb0 + j;
            ok = mbar_wait(&hbar[qh % 3], (qh / 3) & 1, wait_polls);
            fill(qh % 3, (j + 2) & 3, x0, y0);
            ok = ok && mbar_wait(&gbar[qg % 2], (qg / 2) & 1, wait_polls);
            if (__syncthreads_or(!ok)) { failed = true; break; }
            if (active) {
                const S* hs_ = reinterpret_cast<const S*>(smem + C::off_h + ((hb0 + j + 1) % 3) * C::HL::bytes);
                const S* gs_ = reinterpret_cast<const S*>(smem + C::off_g + (qg % 2) * C::GL::bytes);
                R m0 = 0, mx = 0, my = 0, mz = 0, mxx = 0, myy = 0, mzz = 0, mxy = 0, mxz = 0, myz = 0;
                Unroll<0, Q>::run([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    constexpr int CX = L::cx[i], CY = L::cy[i], CZ = L::cz[i];
                    constexpr int off = C::GL::dir_offset(i) / C::ES + A - CX;
                    constexpr double W = L::w[i];
                    const R v = St::load(gs_[off + ty * C::BX + tx], (R)W * p.g_shift, p.g_inv_scale);
                    m0 += v;
                    if (CX) { mx += (R)CX * v; mxx += v; }
                    if (CY) { my += (R)CY * v; myy += v; }
                    if (CZ) { mz += (R)CZ * v; mzz += v; }
                    if (CX * CY) mxy += (R)(CX * CY) * v;
                    if (CX * CZ) mxz += (R)(CX * CZ) * v;
                    if (CY * CZ) myz += (R)(CY * CZ) * v;
                });
                const int sm = j & 3, s0 = (j + 1) & 3, sp = (j + 2) & 3;
                const int lx = tx + 1, ly = ty + HY;
                NodeState<R> s;
                s.phi = phis[s0][ly][lx];
                R gx = 0, gy = 0, gz = 0, lap = 0;
                Unroll<1, Q>::run([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    constexpr int CX = L::cx[i], CY = L::cy[i], CZ = L::cz[i];
                    constexpr double W = L::w[i];
                    const int slot = CZ == 0 ? s0 : (CZ > 0 ? sp : sm);
                    const R v = phis[slot][ly + CY][lx + CX];
                    const R wv = (R)W * v;
                    if (CX) gx += (R)CX * wv;
                    if (CY) gy += (R)CY * wv;
                    if (CZ) gz += (R)CZ * wv;
                    lap += (R)W * (v - s.phi);
                });
                s.gx = gx * (R)3;
                s.gy = gy * (R)3;
                s.gz = gz * (R)3;
                s.lap = lap * (R)6;
                node_state<R, L::kHasY>(s, p, m0, mx, my, mz, mxx, myy, mzz, mxy, mxz, myz);
                const NodeWrites nw = node_writes<LAT>(G, x, y, z);
                const int own = (z + G.GZ) * G.PXY + rb;
                R hsum = 0;
                Unroll<1, Q>::run([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    constexpr int off = C::HL::dir_offset(i) / C::ES + A - L::cx[i];
                    constexpr double W = L::w[i];
                    const R hv = St::load(hs_[off + (ty + HY) * C::BX + tx], (R)W * p.h_shift, (R)1);
                    R hs, gs;
                    collide_dir<LAT, i, R>(s, p, hv, &hs, &gs);
                    hsum += hs;
                    write_dir<LAT, i, WALLS>(D.hout, G, x, y, z, own, nw, St::store(hs, (R)W * p.h_shift, (R)1));
                    write_dir<LAT, i, WALLS>(D.gout, G, x, y, z, own, nw, St::store(gs, (R)W * p.g_shift, p.g_scale));
                    if constexpr (WALLS) {
                        if (p.moving && nw.wall_adj) {
                            moving_wall_write<LAT, i>(D.hout, G, x, y, z, hs, s.phi, p,
                                                      [&](R v) { return St::store(v, (R)W * p.h_shift, (R)1); });
                            moving_wall_write<LAT, i>(D.gout, G, x, y, z, gs, s.rho, p,
                                                      [&](R v) { return St::store(v, (R)W * p.g_shift, p.g_scale); });
                        }
                    }
                });
                {
                    constexpr double W0 = L::w[0];
                    R hs, gs;
                    collide_dir<LAT, 0, R>(s, p, (R)0, &hs, &gs);
                    write_dir<LAT, 0, WALLS>(D.hout, G, x, y, z, own, nw, St::store(s.phi - hsum, (R)W0 * p.h_shift, (R)1));
                    write_dir<LAT, 0, WALLS>(D.gout, G, x, y, z, own, nw, St::store(gs, (R)W0 * p.g_shift, p.g_scale));
                }
            }
        }
        if (failed) break;
        hcount = hb0 + (uint32_t)(LZ + 2);
        gcount = gb0 + (uint32_t)LZ;
    }
    if (failed) {
        if (tid == 0) atomicExch(error_flag, 1);
        // let copies already in flight land before the CTA's shared memory is
        // released.  Every use of a slot but its last issued one was waited for
        // successfully, so the only phase that can be pending is that of the
        // last issued use u (the (u / slots)-th use of the slot): wait for it,
        // bounded; slots with no use issued have nothing in flight.
        auto drain = [&](uint64_t* bars, uint32_t nslots, uint32_t issued) {
            for (uint32_t s = 0; s < nslots; ++s) {
                if (issued <= s) continue;
                const uint32_t last = issued - 1 - ((issued - 1 - s) % nslots);   // last use of slot s
                mbar_wait(&bars[s], (last / nslots) & 1, kDrainPolls);
            }
        };
        drain(hbar, (uint32_t)C::NHS, hiss);
        drain(gbar, (uint32_t)C::NGS, giss);
    }
}

}  // namespace lbm
