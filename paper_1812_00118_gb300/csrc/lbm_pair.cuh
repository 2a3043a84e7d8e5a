// Fused step, node-pair form: every thread updates two nodes 32 apart in x
// (nodes A = x and B = x + 32 of a 64-node-wide warp strip), with all of the
// per-node arithmetic -- phi, the CD stencils, the moments of g, the local
// state of a4-a5 and both collisions -- on the paired FP32 instructions of
// sm_100 and later (FFMA2 / FADD2 / FMUL2), lane .x for node A and lane .y
// for node B.  The arithmetic is that of collide_node (lbm_kernels.cuh),
// Eqs. 1-13 with the closed-form Pi; only the organisation differs:
//
//   * one instruction updates a quantity of two nodes, so the ~600 FP32
//     instructions per node of the one-node kernel are roughly halved;
//   * the address arithmetic of a pull is shared: node B's address is node
//     A's plus 32 elements (an immediate offset), because pulls along x never
//     wrap here.  Along a periodic x axis the node at x = NX - 1 also writes
//     its outgoing f*_j with c_jx = +1 into the ghost column x = -1, and the
//     node at x = 0 writes f*_j with c_jx = -1 into x = NX (the periodic
//     images the next step pulls); across an x wall the ghost column holds
//     the bounce-back value as in the one-node kernels;
//   * loads stay scalar and fully coalesced (a warp reads 32 consecutive
//     values for node A and the next 32 for node B).
//
// The march is that of march() (lbm_kernels.cuh): a CTA owns a TX x TY
// column (TX = 64 per warp along x, TY rows of warps) and walks along z; per
// plane it fills phi of the next plane (tile plus one-node halo ring) into a
// four-slot shared ring, keeps its own pulled h for the next iteration in a
// shared slab, reduces its pulled g to moments, and after one barrier
// collides and writes.  The halo ring is computed where the tile ends: at
// the tile border, or at x = NX / y = NY for a tile that overhangs the grid
// (the overhanging positions are not nodes and are never stored).
//
// Requires the ghost band to hold the x images before the first pair step
// after a state written by another kernel (lbm_init_fields and
// lbm_set_populations write them; the host runs halo_kernel otherwise), and
// the population arrays to be followed by a tail of kPairTail elements (a
// warp strip overhanging the last row reads, but never uses, values past
// the row end).
#pragma once
#include "lbm_kernels.cuh"

namespace lbm {

// ------------------------------------------------------------ paired FP32
using f2 = float2;
__device__ __forceinline__ f2 sp(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 ad(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 ml(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fm(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
// a - b, rounded once (b * -1 is exact)
__device__ __forceinline__ f2 sb(f2 a, f2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ f2 ng(f2 a) { return make_float2(-a.x, -a.y); }

// c-weighted sums with compile-time integer coefficients: only nonzero terms
template <int C>
__device__ __forceinline__ f2 cmul2(f2 v) {
    if constexpr (C == 1) return v;
    else if constexpr (C == -1) return ng(v);
    else return ml(sp((float)C), v);
}
template <int A, int B, int C>
__device__ __forceinline__ f2 cdot3p(f2 a, f2 b, f2 c) {
    if constexpr (A != 0 && B != 0 && C != 0) return ad(ad(cmul2<A>(a), cmul2<B>(b)), cmul2<C>(c));
    else if constexpr (A != 0 && B != 0) return ad(cmul2<A>(a), cmul2<B>(b));
    else if constexpr (A != 0 && C != 0) return ad(cmul2<A>(a), cmul2<C>(c));
    else if constexpr (B != 0 && C != 0) return ad(cmul2<B>(b), cmul2<C>(c));
    else if constexpr (A != 0) return cmul2<A>(a);
    else if constexpr (B != 0) return cmul2<B>(b);
    else if constexpr (C != 0) return cmul2<C>(c);
    else return sp(0.0f);
}
template <int A, int B, int C>
__device__ __forceinline__ float cdot3s(float a, float b, float c) {
    return (float)A * a + (float)B * b + (float)C * c;
}

// ------------------------------------------------------------ pulled loads
// Two scalar loads of one warp strip: p (node A) and p + 32 (node B), the
// second only if node B is a node (kb).  Cached in L1 (h: re-read by the halo
// ring of the same CTA) or not (g: read once); L2 fetches 256-byte blocks.
template <bool STREAM, typename S>
__device__ __forceinline__ void ld_pair(const S* p, bool ka, bool kb, S& a, S& b);

template <>
__device__ __forceinline__ void ld_pair<false, float>(const float* p, bool ka, bool kb, float& a, float& b) {
    a = 0.0f;
    b = 0.0f;
    asm("{\n\t.reg .pred pa, pb;\n\tsetp.ne.u32 pa, %3, 0;\n\tsetp.ne.u32 pb, %4, 0;\n\t"
        "@pa ld.global.nc.L2::256B.f32 %0, [%2];\n\t"
        "@pb ld.global.nc.L2::256B.f32 %1, [%2+128];\n\t}"
        : "+f"(a), "+f"(b)
        : "l"(p), "r"((unsigned)ka), "r"((unsigned)kb));
}
template <>
__device__ __forceinline__ void ld_pair<true, float>(const float* p, bool ka, bool kb, float& a, float& b) {
    a = 0.0f;
    b = 0.0f;
    asm("{\n\t.reg .pred pa, pb;\n\tsetp.ne.u32 pa, %3, 0;\n\tsetp.ne.u32 pb, %4, 0;\n\t"
        "@pa ld.global.nc.L1::no_allocate.L2::256B.f32 %0, [%2];\n\t"
        "@pb ld.global.nc.L1::no_allocate.L2::256B.f32 %1, [%2+128];\n\t}"
        : "+f"(a), "+f"(b)
        : "l"(p), "r"((unsigned)ka), "r"((unsigned)kb));
}
// 16-bit storage: raw bits through u16 registers
template <>
__device__ __forceinline__ void ld_pair<false, __half>(const __half* p, bool ka, bool kb, __half& a, __half& b) {
    unsigned short va = 0, vb = 0;
    asm("{\n\t.reg .pred pa, pb;\n\tsetp.ne.u32 pa, %3, 0;\n\tsetp.ne.u32 pb, %4, 0;\n\t"
        "@pa ld.global.nc.L2::256B.b16 %0, [%2];\n\t"
        "@pb ld.global.nc.L2::256B.b16 %1, [%2+64];\n\t}"
        : "+h"(va), "+h"(vb)
        : "l"(p), "r"((unsigned)ka), "r"((unsigned)kb));
    a = __ushort_as_half(va);
    b = __ushort_as_half(vb);
}
template <>
__device__ __forceinline__ void ld_pair<true, __half>(const __half* p, bool ka, bool kb, __half& a, __half& b) {
    unsigned short va = 0, vb = 0;
    asm("{\n\t.reg .pred pa, pb;\n\tsetp.ne.u32 pa, %3, 0;\n\tsetp.ne.u32 pb, %4, 0;\n\t"
        "@pa ld.global.nc.L1::no_allocate.L2::256B.b16 %0, [%2];\n\t"
        "@pb ld.global.nc.L1::no_allocate.L2::256B.b16 %1, [%2+64];\n\t}"
        : "+h"(va), "+h"(vb)
        : "l"(p), "r"((unsigned)ka), "r"((unsigned)kb));
    a = __ushort_as_half(va);
    b = __ushort_as_half(vb);
}
template <>
__device__ __forceinline__ void ld_pair<false, __nv_bfloat16>(const __nv_bfloat16* p, bool ka, bool kb,
                                                              __nv_bfloat16& a, __nv_bfloat16& b) {
    unsigned short va = 0, vb = 0;
    asm("{\n\t.reg .pred pa, pb;\n\tsetp.ne.u32 pa, %3, 0;\n\tsetp.ne.u32 pb, %4, 0;\n\t"
        "@pa ld.global.nc.L2::256B.b16 %0, [%2];\n\t"
        "@pb ld.global.nc.L2::256B.b16 %1, [%2+64];\n\t}"
        : "+h"(va), "+h"(vb)
        : "l"(p), "r"((unsigned)ka), "r"((unsigned)kb));
    a = __ushort_as_bfloat16(va);
    b = __ushort_as_bfloat16(vb);
}
template <>
__device__ __forceinline__ void ld_pair<true, __nv_bfloat16>(const __nv_bfloat16* p, bool ka, bool kb,
                                                             __nv_bfloat16& a, __nv_bfloat16& b) {
    unsigned short va = 0, vb = 0;
    asm("{\n\t.reg .pred pa, pb;\n\tsetp.ne.u32 pa, %3, 0;\n\tsetp.ne.u32 pb, %4, 0;\n\t"
        "@pa ld.global.nc.L1::no_allocate.L2::256B.b16 %0, [%2];\n\t"
        "@pb ld.global.nc.L1::no_allocate.L2::256B.b16 %1, [%2+64];\n\t}"
        : "+h"(va), "+h"(vb)
        : "l"(p), "r"((unsigned)ka), "r"((unsigned)kb));
    a = __ushort_as_bfloat16(va);
    b = __ushort_as_bfloat16(vb);
}

// Pulled values of direction I for the pair: the address of node A is the
// plane part zo[1 + c_z] (wrapped or ghost plane), the row part ro[1 + c_y]
// (wrapped or ghost row) and the column xa - c_x (never wrapped: ghost
// column); node B is 32 elements further.
template <int LAT, int I, bool STREAM, int ST>
__device__ __forceinline__ f2 pull_pair(const typename Storage<ST>::S* const* arr, const int* zo, const int* ro,
                                        int xa, bool ka, bool kb, float shift, float inv_scale) {
    using L = Lattice<LAT>;
    using St = Storage<ST>;
    typename St::S a, b;
    ld_pair<STREAM>(arr[I] + (zo[1 + L::cz[I]] + ro[1 + L::cy[I]] + xa - L::cx[I]), ka, kb, a, b);
    return make_float2(St::load(a, shift, inv_scale), St::load(b, shift, inv_scale));
}

// ------------------------------------------------------------ local state of a pair
struct PairNode {
    f2 phi, gx, gy, gz, lap;
    f2 rho, mu, fr;         // F = fr * g (g the uniform body acceleration)
    f2 ux, uy, uz, P;
    f2 usq, ug, uF;
    f2 pxx, pyy, pzz, pxy, pxz, pyz, tr3;
    f2 omega, nx, ny, nz, theta;
};

// node_state (lbm_kernels.cuh) for two nodes; Pi by the same closed form,
// regrouped: sum c c K = T (u v + v u) - s2 u u + rho_dif T (u.grad) I with
// v = (rho_dif + 3 mu) grad + 3 F and s2 = (rho_dif + 3 mu) u.grad + 3 u.F.
// node_state (lbm_kernels.cuh) for two nodes, in three parts so that the
// collision can run its h and g halves with fewer values live at once.
// (1) rho, mu, F = fr g, the velocity (Eq. 13 reading) and P.
template <bool THREE_D>
__device__ __forceinline__ void pair_velocity(PairNode& s, const PhysT<float>& p, f2 m0, f2 mx, f2 my, f2 mz) {
    const float T = 1.0f / 3.0f;
    const f2 rd = sp(p.rho_dif);
    s.rho = fm(s.phi, rd, sp(p.rho_L));
    // mu = beta phi (phi - 1)(phi - 1/2) - kappa lap       (Eq. 8)
    const f2 q = ml(ml(s.phi, ad(s.phi, sp(-1.0f))), ad(s.phi, sp(-0.5f)));
    s.mu = fm(q, sp(p.beta), ml(s.lap, sp(-p.kappa)));
    s.fr = p.force_mode == 0 ? s.rho : ad(s.rho, sp(-p.rho_bar));
    const f2 rho_e = p.hocorr ? fm(s.lap, sp(0.25f * p.rho_dif), s.rho) : s.rho;
    const f2 inv = make_float2(recip(rho_e.x), recip(rho_e.y));
    // rho_e u = m1 + (mu grad phi + F) / 2                 (after Eq. 12, Eq. 13 reading)
    const f2 h = sp(0.5f);
    s.ux = ml(fm(fm(s.mu, s.gx, ml(s.fr, sp(p.g[0]))), h, mx), inv);
    s.uy = THREE_D ? ml(fm(fm(s.mu, s.gy, ml(s.fr, sp(p.g[1]))), h, my), inv) : sp(0.0f);
    s.uz = ml(fm(fm(s.mu, s.gz, ml(s.fr, sp(p.g[2]))), h, mz), inv);
    s.usq = fm(s.ux, s.ux, fm(s.uy, s.uy, ml(s.uz, s.uz)));
    s.ug = fm(s.ux, s.gx, fm(s.uy, s.gy, ml(s.uz, s.gz)));
    const f2 ugv = fm(s.ux, sp(p.g[0]), fm(s.uy, sp(p.g[1]), ml(s.uz, sp(p.g[2]))));
    s.uF = ml(s.fr, ugv);
    // P = T m0 + (T rho_dif / 2) u.grad phi                (after Eq. 12)
    s.P = fm(s.ug, sp(0.5f * T * p.rho_dif), ml(m0, sp(T)));
}

// (2) the interface normal and theta (Eq. 4) + delta theta (Eq. 14).
__device__ __forceinline__ void pair_interface(PairNode& s, const PhysT<float>& p) {
    const f2 g2 = fm(s.gx, s.gx, fm(s.gy, s.gy, ml(s.gz, s.gz)));
    const f2 gm = make_float2(sqrtf(g2.x), sqrtf(g2.y));
    const f2 ig = make_float2(recip(gm.x + p.eps), recip(gm.y + p.eps));
    s.nx = ml(s.gx, ig);
    s.ny = ml(s.gy, ig);
    s.nz = ml(s.gz, ig);
    const f2 d = ad(s.phi, sp(-0.5f));
    s.theta = ml(fm(ml(d, d), sp(-4.0f), sp(1.0f)), sp(p.theta_coef));
    if (p.dtheta_coef != 0.0f) {
        // delta theta = -C (M/T) W^2 max(0, (2 phi - 1) lap phi) |grad phi|
        const f2 t = ml(fm(s.phi, sp(2.0f), sp(-1.0f)), s.lap);
        const f2 f = make_float2(fmaxf(t.x, 0.0f), fmaxf(t.y, 0.0f));
        s.theta = fm(ml(f, gm), sp(-p.dtheta_coef), s.theta);
    }
}

// (3) Pi = m2 - sum c c g^eq by the closed form of node_state, regrouped:
// sum c c K = T (u v + v u) - s2 u u + rho_dif T (u.grad) I with
// v = (rho_dif + 3 mu) grad + 3 F and s2 = (rho_dif + 3 mu) u.grad + 3 u.F;
// then tr(Pi)/3 and 1/tau_mix (Eq. 9, phi clipped).
template <bool THREE_D>
__device__ __forceinline__ void pair_pi(PairNode& s, const PhysT<float>& p, f2 mxx, f2 myy, f2 mzz, f2 mxy, f2 mxz,
                                        f2 myz) {
    const float T = 1.0f / 3.0f;
    const f2 h = sp(0.5f);
    const f2 sK = fm(s.mu, sp(3.0f), sp(p.rho_dif));
    const f2 fr3 = ml(s.fr, sp(3.0f));
    const f2 vx = fm(sK, s.gx, ml(fr3, sp(p.g[0])));
    const f2 vy = fm(sK, s.gy, ml(fr3, sp(p.g[1])));
    const f2 vz = fm(sK, s.gz, ml(fr3, sp(p.g[2])));
    const f2 s2 = fm(sK, s.ug, ml(s.uF, sp(3.0f)));
    const f2 nrp = ng(fm(s2, h, s.rho));                    // -(rho + s2 / 2)
    const f2 Pd = fm(s.ug, sp(-0.5f * T * p.rho_dif), s.P); // P - (1/2) rho_dif T u.grad
    const f2 hT = sp(0.5f * T);
    // diagonal: m_aa - (rho + s2/2) u_a^2 + T u_a v_a - Pd
    s.pxx = sb(fm(ml(s.ux, vx), sp(T), fm(nrp, ml(s.ux, s.ux), mxx)), Pd);
    s.pzz = sb(fm(ml(s.uz, vz), sp(T), fm(nrp, ml(s.uz, s.uz), mzz)), Pd);
    s.pxz = fm(fm(s.ux, vz, ml(s.uz, vx)), hT, fm(nrp, ml(s.ux, s.uz), mxz));
    if (THREE_D) {
        s.pyy = sb(fm(ml(s.uy, vy), sp(T), fm(nrp, ml(s.uy, s.uy), myy)), Pd);
        s.pxy = fm(fm(s.ux, vy, ml(s.uy, vx)), hT, fm(nrp, ml(s.ux, s.uy), mxy));
        s.pyz = fm(fm(s.uy, vz, ml(s.uz, vy)), hT, fm(nrp, ml(s.uy, s.uz), myz));
    } else {
        s.pyy = s.pxy = s.pyz = sp(0.0f);
    }
    s.tr3 = ml(ad(ad(s.pxx, s.pyy), s.pzz), sp(T));
    const f2 pc = make_float2(fminf(fmaxf(s.phi.x, 0.0f), 1.0f), fminf(fmaxf(s.phi.y, 0.0f), 1.0f));
    s.omega = fm(pc, sp(p.om_dif), sp(p.om_L));
}

template <bool THREE_D>
__device__ __forceinline__ void pair_state(PairNode& s, const PhysT<float>& p, f2 m0, f2 mx, f2 my, f2 mz, f2 mxx,
                                           f2 myy, f2 mzz, f2 mxy, f2 mxz, f2 myz) {
    pair_velocity<THREE_D>(s, p, m0, mx, my, mz);
    pair_pi<THREE_D>(s, p, mxx, myy, mzz, mxy, mxz, myz);
    pair_interface(s, p);
}

// Node quantities the direction pairs share: per weight class k (0: the
// axis weight, 1: the diagonal weight), w-scaled terms.
struct PairShared {
    f2 nus[2];      // -1.5 w u.u
    f2 mu3w[2];     // 3 w mu  (via 3 w)
    f2 w3P_F0[2];   // 3 w P - (1 - omega) 4.5 w tr(Pi)/3   (even base of g*)
    f2 om45w[2];    // (1 - omega) 4.5 w
    f2 hocw[2];     // w (3/4) rho_dif lap   (Eq. 13), 0 without the correction
    f2 phw[2];      // phi w
    f2 thw[2];      // theta w
    f2 sK, mu3, uF3neg, neg_ug, fr3;
    f2 omt, itau;   // 1 - 1/tau_phi, 1/tau_phi
    f2 sxy, sxz, syz, pxy2, pxz2, pyz2;   // Pi_aa + Pi_bb, 2 Pi_ab
};

template <int LAT>
__device__ __forceinline__ void pair_shared(const PairNode& s, const PhysT<float>& p, PairShared& q) {
    using L = Lattice<LAT>;
    constexpr int IA = 1, ID = 4;
    static_assert(L::cx[IA] * L::cx[IA] + L::cy[IA] * L::cy[IA] + L::cz[IA] * L::cz[IA] == 1, "axis");
    static_assert(L::cx[ID] * L::cx[ID] + L::cy[ID] * L::cy[ID] + L::cz[ID] * L::cz[ID] == 2, "diagonal");
    constexpr float WA = (float)L::w[IA], WD = (float)L::w[ID];
    const float wk[2] = {WA, WD};
    const f2 om45 = ml(sb(sp(1.0f), s.omega), sp(4.5f));
    const f2 hoc = p.hocorr ? ml(s.lap, sp(0.75f * p.rho_dif)) : sp(0.0f);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const f2 w = sp(wk[k]);
        q.nus[k] = ml(s.usq, sp(-1.5f * wk[k]));
        q.om45w[k] = ml(om45, w);
        q.w3P_F0[k] = sb(ml(s.P, sp(3.0f * wk[k])), ml(q.om45w[k], s.tr3));
        q.hocw[k] = ml(hoc, w);
        q.phw[k] = ml(s.phi, w);
        q.thw[k] = ml(s.theta, w);
        q.mu3w[k] = ml(s.mu, sp(3.0f * wk[k]));
    }
    q.sK = fm(s.mu, sp(3.0f), sp(p.rho_dif));
    q.mu3 = ml(s.mu, sp(3.0f));
    q.uF3neg = ml(s.uF, sp(-3.0f));
    q.neg_ug = ng(s.ug);
    q.fr3 = ml(s.fr, sp(3.0f));
    q.itau = sp(p.inv_tau_phi);
    q.omt = sp(1.0f - p.inv_tau_phi);
    q.sxy = ad(s.pxx, s.pyy);
    q.sxz = ad(s.pxx, s.pzz);
    q.syz = ad(s.pyy, s.pzz);
    q.pxy2 = ml(s.pxy, sp(2.0f));
    q.pxz2 = ml(s.pxz, sp(2.0f));
    q.pyz2 = ml(s.pyz, sp(2.0f));
}

// c_i c_i : Pi for a compile-time velocity (D2Q9 / D3Q19: |c_a| <= 1, at most
// two nonzero components)
template <int CX, int CY, int CZ>
__device__ __forceinline__ f2 ccpi(const PairNode& s, const PairShared& q) {
    constexpr int n = (CX != 0) + (CY != 0) + (CZ != 0);
    if constexpr (n == 1) return CX ? s.pxx : (CY ? s.pyy : s.pzz);
    else if constexpr (CX != 0 && CY != 0) return CX * CY > 0 ? ad(q.sxy, q.pxy2) : sb(q.sxy, q.pxy2);
    else if constexpr (CX != 0 && CZ != 0) return CX * CZ > 0 ? ad(q.sxz, q.pxz2) : sb(q.sxz, q.pxz2);
    else return CY * CZ > 0 ? ad(q.syz, q.pyz2) : sb(q.syz, q.pyz2);
}

// Post-collision values of direction I (lane-wise for the two nodes) and of
// its opposite J, the arithmetic of collide_dir:
//   G - w = E +- O, E = w (4.5 (c.u)^2 - 1.5 u.u), O = 3 w c.u      (Eq. 3)
//   K = (G - w)(rho_dif + 3 mu)(c.grad - u.grad) + 3 w mu (c.grad - u.grad)
//       + 3 G (c.F - u.F)                                            (Eq. 7)
//   g* = rho (G - w) + 3 w P + K/2 + (c.u) w (3/4) rho_dif lap
//        + (1 - 1/tau_mix) 4.5 w (c c : Pi - T tr Pi)                  (Eqs. 6, 10-13)
//   h* = h + (phi G + theta w c.n - h) / tau_phi                      (Eqs. 1-2)
template <int LAT, int I>
__device__ __forceinline__ void collide_pair2(const PairNode& s, const PairShared& q, const PhysT<float>& p,
                                              f2 hi, f2 hj, f2& hsi, f2& hsj, f2& gsi, f2& gsj) {
    using L = Lattice<LAT>;
    constexpr int CX = L::cx[I], CY = L::cy[I], CZ = L::cz[I];
    constexpr int K = (CX * CX + CY * CY + CZ * CZ) == 1 ? 0 : 1;
    constexpr float W = (float)L::w[I];
    const f2 cu = cdot3p<CX, CY, CZ>(s.ux, s.uy, s.uz);
    const f2 cg = cdot3p<CX, CY, CZ>(s.gx, s.gy, s.gz);
    const f2 cn = cdot3p<CX, CY, CZ>(s.nx, s.ny, s.nz);
    const float cgv = cdot3s<CX, CY, CZ>(p.g[0], p.g[1], p.g[2]);
    const f2 E = fm(ml(cu, cu), sp(4.5f * W), q.nus[K]);
    const f2 O = ml(cu, sp(3.0f * W));
    const f2 Gi = ad(E, O), Gj = sb(E, O);               // Gamma - w of I and J
    const f2 Di = ad(cg, q.neg_ug), Dj = sb(q.neg_ug, cg);   // c.grad - u.grad
    const f2 cF3 = ml(q.fr3, sp(cgv));
    const f2 Fi = ad(cF3, q.uF3neg), Fj = sb(q.uF3neg, cF3); // 3 (c.F - u.F)
    // K = (G - w) (sK D + 3 (c.F - u.F)) + w (3 mu D + 3 (c.F - u.F))
    const f2 Ki = fm(Gi, fm(q.sK, Di, Fi), ml(sp(W), fm(q.mu3, Di, Fi)));
    const f2 Kj = fm(Gj, fm(q.sK, Dj, Fj), ml(sp(W), fm(q.mu3, Dj, Fj)));
    const f2 base = fm(ccpi<CX, CY, CZ>(s, q), q.om45w[K], q.w3P_F0[K]);
    const f2 hc = ml(cu, q.hocw[K]);
    gsi = ad(fm(Ki, sp(0.5f), fm(s.rho, Gi, base)), hc);
    gsj = sb(fm(Kj, sp(0.5f), fm(s.rho, Gj, base)), hc);
    const f2 tn = ml(cn, q.thw[K]);
    const f2 heqi = fm(s.phi, Gi, ad(q.phw[K], tn));
    const f2 heqj = fm(s.phi, Gj, sb(q.phw[K], tn));
    hsi = fm(hi, q.omt, ml(heqi, q.itau));
    hsj = fm(hj, q.omt, ml(heqj, q.itau));
}

// The h half of collide_pair2 (Eqs. 1-3): h* of I and J = opp(I).
template <int LAT, int I>
__device__ __forceinline__ void collide_pair_h(const PairNode& s, const PhysT<float>& p, f2 nus, f2 phw, f2 thw,
                                               f2 hi, f2 hj, f2& hsi, f2& hsj) {
    using L = Lattice<LAT>;
    constexpr int CX = L::cx[I], CY = L::cy[I], CZ = L::cz[I];
    constexpr float W = (float)L::w[I];
    const f2 cu = cdot3p<CX, CY, CZ>(s.ux, s.uy, s.uz);
    const f2 cn = cdot3p<CX, CY, CZ>(s.nx, s.ny, s.nz);
    const f2 E = fm(ml(cu, cu), sp(4.5f * W), nus);
    const f2 O = ml(cu, sp(3.0f * W));
    const f2 tn = ml(cn, thw);
    const f2 heqi = fm(s.phi, ad(E, O), ad(phw, tn));
    const f2 heqj = fm(s.phi, sb(E, O), sb(phw, tn));
    hsi = fm(hi, sp(1.0f - p.inv_tau_phi), ml(heqi, sp(p.inv_tau_phi)));
    hsj = fm(hj, sp(1.0f - p.inv_tau_phi), ml(heqj, sp(p.inv_tau_phi)));
}

// The g half of collide_pair2 (Eqs. 3, 6, 7, 10-13): g* of I and J.
template <int LAT, int I>
__device__ __forceinline__ void collide_pair_g(const PairNode& s, const PairShared& q, const PhysT<float>& p,
                                               f2& gsi, f2& gsj) {
    using L = Lattice<LAT>;
    constexpr int CX = L::cx[I], CY = L::cy[I], CZ = L::cz[I];
    constexpr int K = (CX * CX + CY * CY + CZ * CZ) == 1 ? 0 : 1;
    constexpr float W = (float)L::w[I];
    const f2 cu = cdot3p<CX, CY, CZ>(s.ux, s.uy, s.uz);
    const f2 cg = cdot3p<CX, CY, CZ>(s.gx, s.gy, s.gz);
    const float cgv = cdot3s<CX, CY, CZ>(p.g[0], p.g[1], p.g[2]);
    const f2 E = fm(ml(cu, cu), sp(4.5f * W), q.nus[K]);
    const f2 O = ml(cu, sp(3.0f * W));
    const f2 Gi = ad(E, O), Gj = sb(E, O);
    const f2 Di = ad(cg, q.neg_ug), Dj = sb(q.neg_ug, cg);
    const f2 cF3 = ml(q.fr3, sp(cgv));
    const f2 Fi = ad(cF3, q.uF3neg), Fj = sb(q.uF3neg, cF3);
    const f2 Ki = fm(Gi, fm(q.sK, Di, Fi), ml(sp(W), fm(q.mu3, Di, Fi)));
    const f2 Kj = fm(Gj, fm(q.sK, Dj, Fj), ml(sp(W), fm(q.mu3, Dj, Fj)));
    const f2 base = fm(ccpi<CX, CY, CZ>(s, q), q.om45w[K], q.w3P_F0[K]);
    const f2 hc = ml(cu, q.hocw[K]);
    gsi = ad(fm(Ki, sp(0.5f), fm(s.rho, Gi, base)), hc);
    gsj = sb(fm(Kj, sp(0.5f), fm(s.rho, Gj, base)), hc);
}

// ------------------------------------------------------------ march
template <int LAT, int ST, int TX, int TY>
struct PairSmem {
    static constexpr int Q = Lattice<LAT>::Q;
    static constexpr int HY = Lattice<LAT>::kHasY ? 1 : 0;
    static constexpr int SX = TX + 2, SY = TY + 2 * HY;
    static constexpr int NT = TX / 2 * TY;
    float phis[4][SY][SX];
    f2 hown[2][Q][NT];   // the pair's own pulled h of the last two filled planes
};

// Store the pair's value of direction J: own cells (A at `own`, B at own + 32),
// the periodic x images of the x-edge nodes, and with walls the bounce-back
// ghost cells (x unwrapped, and also wrapped where x + c_x leaves a periodic
// x axis, so that the one-node kernels, which wrap x, find it too).
struct PairWrites {
    int own;               // padded index of node A
    int xa, y;             // coordinates of node A (B: xa + 32)
    bool ka, kb;           // A, B are nodes
    bool edge;             // some node of the pair writes an x image or a wall ghost
    bool a_lo, a_hi, b_hi; // x images: A at x = 0, A / B at x = NX - 1 (periodic x)
    bool wa, wb;           // A, B next to a wall
};

// Bounce-back ghost write of one node's post-collision value v of direction J
// (see write_dir), with the momentum of a moving wall taken off (see
// moving_wall_write): x + c_x unwrapped, and wrapped too where it leaves a
// periodic x axis.  s = phi for h, rho for g.
template <int LAT, int J, typename S, typename Store>
__device__ __forceinline__ void wall_ghost1(S* const* arr, const Geom& G, const PhysT<float>& p, int x, int y, int z,
                                            float v, float s, Store store) {
    using L = Lattice<LAT>;
    constexpr int CX = L::cx[J], CY = L::cy[J], CZ = L::cz[J];
    const int t[3] = {x + CX, y + CY, z + CZ};
    const int n[3] = {G.NX, G.NY, G.NZ};
    const int c[3] = {CX, CY, CZ};
    float u0 = 0.0f, u1 = 0.0f, u2 = 0.0f;
    int cnt = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (c[a] == 0 || !G.wall[a]) continue;
        const bool lo = t[a] < 0, hi = t[a] >= n[a];
        if (!lo && !hi) continue;
        u0 += hi ? p.uw[a][1][0] : p.uw[a][0][0];
        u1 += hi ? p.uw[a][1][1] : p.uw[a][0][1];
        u2 += hi ? p.uw[a][1][2] : p.uw[a][0][2];
        ++cnt;
    }
    if (cnt == 0) return;   // no wall crossed
    constexpr float WJ = (float)L::w[J];
    if (p.moving) v -= 6.0f * WJ * s * (((float)CX * u0 + (float)CY * u1 + (float)CZ * u2) / (float)cnt);
    const int yy = wrap1(t[1], G.NY, G.wall[1]), zz = wrap1(t[2], G.NZ, G.wall[2]);
    const auto sv = store(v);
    arr[L::opp(J)][pidx(G, t[0], yy, zz)] = sv;
    if (!G.wall[0] && (t[0] < 0 || t[0] >= G.NX)) arr[L::opp(J)][pidx(G, wrap1(t[0], G.NX, 0), yy, zz)] = sv;
}

template <int LAT, int J, bool WALLS, typename S, typename Store>
__device__ __forceinline__ void write_pair(S* const* arr, const Geom& G, const PhysT<float>& p, int z,
                                           const PairWrites& w, f2 v, f2 s, Store store) {
    using L = Lattice<LAT>;
    constexpr int CX = L::cx[J];
    S* a = arr[J];
    const S va = store(v.x), vb = store(v.y);
    if (w.ka) a[w.own] = va;
    if (w.kb) a[w.own + 32] = vb;
    if (w.edge) {
        if (CX == -1 && w.a_lo) a[w.own + G.NX] = va;            // image at x = NX of node 0
        if (CX == 1 && w.a_hi) a[w.own - G.NX] = va;             // image at x = -1 of node NX - 1
        if (CX == 1 && w.b_hi) a[w.own + 32 - G.NX] = vb;
        if constexpr (WALLS) {
            if (CX != 0 || L::cy[J] != 0 || L::cz[J] != 0) {
                if (w.wa) wall_ghost1<LAT, J>(arr, G, p, w.xa, w.y, z, v.x, s.x, store);
                if (w.wb) wall_ghost1<LAT, J>(arr, G, p, w.xa + 32, w.y, z, v.y, s.y, store);
            }
        }
    }
}

// Moments of the pair's pulled g (over opposite pairs, as g_moments).
struct PairMoments {
    f2 m0, mx, my, mz, mxx, myy, mzz, mxy, mxz, myz;
};

template <int LAT, int ST, int TX, int TY, bool WALLS, bool GFIRST, bool SRING, bool HG>
__device__ __forceinline__ void march_pair(const DirPtrs<typename Storage<ST>::S, Lattice<LAT>::Q>& D,
                                           const Geom& G, const PhysT<float>& p, int x0, int y0, int z0, int z1,
                                           PairSmem<LAT, ST, TX, TY>& sm) {
    using L = Lattice<LAT>;
    using St = Storage<ST>;
    using S = typename St::S;
    using Sm = PairSmem<LAT, ST, TX, TY>;
    constexpr int Q = L::Q, HY = Sm::HY;
    constexpr int WR = TX / 64;   // warps per row
    static_assert(TX % 64 == 0, "pair tiles are 64 nodes per warp along x");
    const int tid = threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    const int row = wid / WR, wc = wid % WR;
    const int lxa = 64 * wc + lane;                    // tile column of node A (B: + 32)
    const int xa = x0 + lxa, y = y0 + row;
    const bool rowok = y < G.NY;
    const bool ka = rowok && xa < G.NX, kb = rowok && xa + 32 < G.NX;
    // where the tile ends: the halo ring sits at lxr (x) and lyb (y)
    const int nxt = min(TX, G.NX - x0), nyt = HY ? min(TY, G.NY - y0) : 1;
    const int lxr = nxt + 1, lyb = HY ? nyt + 1 : 0;
    // row offsets of the pulls (wrapped or ghost rows), fixed for the march
    auto rows_of = [&](int yy, int* ro) {
#pragma unroll
        for (int k = 0; k < 3; ++k) ro[k] = (wrap1(yy - (k - 1), G.NY, G.wall[1]) + G.GY) * G.PX;
    };
    int ro_own[3], ro_top[3], ro_bot[3];
    rows_of(HY ? stencil_coord(y, G.NY, G.wall[1]) : 0, ro_own);
    const int col_a = xa + G.GX;
    // ring rows (pairs): the warps of tile row 0 fill the row above the tile,
    // the warps of the last tile row the row below
    const bool do_top = !SRING && HY && row == 0, do_bot = !SRING && HY && row == TY - 1;
    if (HY) {
        rows_of(stencil_coord(y0 - 1, G.NY, G.wall[1]), ro_top);
        rows_of(stencil_coord(y0 + nyt, G.NY, G.wall[1]), ro_bot);
    }
    const bool ring_a = xa < G.NX && lxa < nxt, ring_b = xa + 32 < G.NX && lxa + 32 < nxt;
    // SRING: the whole halo ring as scalar positions spread over all threads
    // (position k: the row above, the row below, then the side columns),
    // at most kRingRounds per thread; offsets fixed for the march
    constexpr int kRingRounds = 2;
    const int nring = HY ? 2 * nxt + 2 * (lyb + 1) : 2;
    int rg_n = 0, rg_lx[kRingRounds], rg_ly[kRingRounds], rg_col[kRingRounds], rg_ro[kRingRounds][3];
    if (SRING) {
#pragma unroll
        for (int r = 0; r < kRingRounds; ++r) {
            const int k = tid + r * Sm::NT;
            rg_lx[r] = rg_ly[r] = rg_col[r] = 0;
            rg_ro[r][0] = rg_ro[r][1] = rg_ro[r][2] = 0;
            if (k >= nring) continue;
            int lx, ly;
            if (HY && k < nxt) { lx = 1 + k; ly = 0; }
            else if (HY && k < 2 * nxt) { lx = 1 + k - nxt; ly = lyb; }
            else { const int q = k - (HY ? 2 * nxt : 0); lx = (q & 1) ? lxr : 0; ly = q >> 1; }
            rg_lx[r] = lx;
            rg_ly[r] = ly;
            rg_col[r] = stencil_coord(x0 - 1 + lx, G.NX, G.wall[0]) + G.GX;
            rows_of(HY ? stencil_coord(y0 - 1 + ly, G.NY, G.wall[1]) : 0, rg_ro[r]);
            rg_n = r + 1;
        }
    }
    // ring side positions (scalar): lx = 0 and lx = lxr for ly = 0 .. lyb,
    // handled by the lanes of one warp
    constexpr int SIDE_WARP = (HY && TY >= 3) ? WR : (WR > 1 ? WR - 1 : 0);
    const int nside = 2 * (lyb + 1);
    const bool do_side = !SRING && wid == SIDE_WARP && lane < nside;
    int side_lx = 0, side_ly = 0, side_ro[3] = {0, 0, 0}, side_col = 0;
    if (do_side) {
        side_lx = (lane & 1) ? lxr : 0;
        side_ly = lane >> 1;
        const int xs = stencil_coord(x0 - 1 + side_lx, G.NX, G.wall[0]);
        const int ys = HY ? stencil_coord(y0 - 1 + side_ly, G.NY, G.wall[1]) : 0;
        rows_of(ys, side_ro);
        side_col = xs + G.GX;
    }
    auto plane_offsets = [&](int zz, int* zo) {
#pragma unroll
        for (int k = 0; k < 3; ++k) zo[k] = G.base + (pull_plane(G, zz - (k - 1)) + G.GZ) * G.PXY;
    };
    // phi of plane zp into ring slot `slot`, own pulled h into hown[hs]
    auto fill = [&](int zp, int slot, int hs) {
        const int zz = stencil_coord(zp, G.NZ, G.wall[2]);
        int zo[3];
        plane_offsets(zz, zo);
        f2 phi = sp(0.0f);
        Unroll<0, Q>::run([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr float W = (float)L::w[i];
            const f2 v = pull_pair<LAT, i, false, ST>(D.hin, zo, ro_own, col_a, ka, kb, W * p.h_shift, 1.0f);
            sm.hown[hs][i][tid] = v;
            phi = ad(phi, v);
        });
        if (ka) sm.phis[slot][row + HY][lxa + 1] = phi.x;
        if (kb) sm.phis[slot][row + HY][lxa + 33] = phi.y;
        if (HY && (do_top || do_bot)) {
            const int* ro = do_top ? ro_top : ro_bot;
            f2 r = sp(0.0f);
            Unroll<0, Q>::run([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                constexpr float W = (float)L::w[i];
                r = ad(r, pull_pair<LAT, i, false, ST>(D.hin, zo, ro, col_a, ring_a, ring_b, W * p.h_shift, 1.0f));
            });
            const int ly = do_top ? 0 : lyb;
            if (ring_a) sm.phis[slot][ly][lxa + 1] = r.x;
            if (ring_b) sm.phis[slot][ly][lxa + 33] = r.y;
        }
        if (do_side) {
            float r = 0.0f;
            Unroll<0, Q>::run([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                constexpr int CX = L::cx[i], CY = L::cy[i], CZ = L::cz[i];
                constexpr float W = (float)L::w[i];
                const S* ptr = D.hin[i] + (zo[1 + CZ] + side_ro[1 + CY] + side_col - CX);
                r += St::load(ld_keep(ptr), W * p.h_shift, 1.0f);
            });
            sm.phis[slot][side_ly][side_lx] = r;
        }
        if (SRING) {
#pragma unroll
            for (int rr = 0; rr < kRingRounds; ++rr) {
                if (rr >= rg_n) break;
                float r = 0.0f;
                Unroll<0, Q>::run([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    constexpr int CX = L::cx[i], CY = L::cy[i], CZ = L::cz[i];
                    constexpr float W = (float)L::w[i];
                    const S* ptr = D.hin[i] + (zo[1 + CZ] + rg_ro[rr][1 + CY] + rg_col[rr] - CX);
                    r += St::load(ld_keep(ptr), W * p.h_shift, 1.0f);
                });
                sm.phis[slot][rg_ly[rr]][rg_lx[rr]] = r;
            }
        }
    };

    // writes of the pair, fixed for the march but z
    PairWrites wr;
    wr.own = G.base + (y + G.GY) * G.PX + col_a;   // + plane part per z
    wr.xa = xa;
    wr.y = y;
    wr.ka = ka;
    wr.kb = kb;
    wr.a_lo = ka && !G.wall[0] && xa == 0;
    wr.a_hi = ka && !G.wall[0] && xa == G.NX - 1;
    wr.b_hi = kb && !G.wall[0] && xa + 32 == G.NX - 1;
    const bool wy = L::kHasY && G.wall[1] && (y == 0 || y == G.NY - 1);
    const bool wa_xy = WALLS && ka && (wy || (G.wall[0] && (xa == 0 || xa == G.NX - 1)));
    const bool wb_xy = WALLS && kb && (wy || (G.wall[0] && xa + 32 == G.NX - 1));

    fill(z0 - 1, 0, 0);
    fill(z0, 1, 1);
    for (int z = z0; z < z1; ++z) {
        const int j = z - z0;
        int zo[3];
        plane_offsets(z, zo);
        // g of the pair, reduced to moments; GFIRST: the g loads are issued
        // before the phi fill of the next plane, so both latencies overlap
        PairMoments m;
        {
            f2 gv[Q];
            auto load_g = [&]() {
                Unroll<0, Q>::run([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    constexpr float W = (float)L::w[i];
                    gv[i] = pull_pair<LAT, i, true, ST>(D.gin, zo, ro_own, col_a, ka, kb, W * p.g_shift,
                                                        p.g_inv_scale);
                });
            };
            if (GFIRST) {
                load_g();
                fill(z + 1, (j + 2) & 3, j & 1);
            } else {
                fill(z + 1, (j + 2) & 3, j & 1);
                load_g();
            }
            m.m0 = gv[0];
            m.mx = m.my = m.mz = m.mxx = m.myy = m.mzz = m.mxy = m.mxz = m.myz = sp(0.0f);
            Unroll<1, Q>::run([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                constexpr int o = L::op[i];
                if constexpr (i < o) {
                    constexpr int CX = L::cx[i], CY = L::cy[i], CZ = L::cz[i];
                    const f2 s_ = ad(gv[i], gv[o]), d_ = sb(gv[i], gv[o]);
                    m.m0 = ad(m.m0, s_);
                    if (CX) { m.mx = CX > 0 ? ad(m.mx, d_) : sb(m.mx, d_); m.mxx = ad(m.mxx, s_); }
                    if (CY) { m.my = CY > 0 ? ad(m.my, d_) : sb(m.my, d_); m.myy = ad(m.myy, s_); }
                    if (CZ) { m.mz = CZ > 0 ? ad(m.mz, d_) : sb(m.mz, d_); m.mzz = ad(m.mzz, s_); }
                    if (CX * CY) m.mxy = CX * CY > 0 ? ad(m.mxy, s_) : sb(m.mxy, s_);
                    if (CX * CZ) m.mxz = CX * CZ > 0 ? ad(m.mxz, s_) : sb(m.mxz, s_);
                    if (CY * CZ) m.myz = CY * CZ > 0 ? ad(m.myz, s_) : sb(m.myz, s_);
                }
            });
        }
        __syncthreads();
        if (!(ka || kb)) continue;
        const int sm_ = j & 3, s0 = (j + 1) & 3, sp_ = (j + 2) & 3;
        const int hs = (j + 1) & 1;
        PairNode s;
        const int ly = row + HY, lx = lxa + 1;
        s.phi = make_float2(sm.phis[s0][ly][lx], sm.phis[s0][ly][lx + 32]);
        // central differences (stencils after Eq. 12), opposite pairs
        f2 gx = sp(0.0f), gy = sp(0.0f), gz = sp(0.0f), lap = sp(0.0f);
        Unroll<1, Q>::run([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int o = L::op[i];
            if constexpr (i < o) {
                constexpr int CX = L::cx[i], CY = L::cy[i], CZ = L::cz[i];
                constexpr float W = (float)L::w[i];
                const int slot_p = CZ == 0 ? s0 : (CZ > 0 ? sp_ : sm_);
                const int slot_m = CZ == 0 ? s0 : (CZ > 0 ? sm_ : sp_);
                const f2 vp = make_float2(sm.phis[slot_p][ly + CY][lx + CX], sm.phis[slot_p][ly + CY][lx + CX + 32]);
                const f2 vm = make_float2(sm.phis[slot_m][ly - CY][lx - CX], sm.phis[slot_m][ly - CY][lx - CX + 32]);
                const f2 wd = ml(sp(W), sb(vp, vm));
                if (CX) gx = CX > 0 ? ad(gx, wd) : sb(gx, wd);
                if (CY) gy = CY > 0 ? ad(gy, wd) : sb(gy, wd);
                if (CZ) gz = CZ > 0 ? ad(gz, wd) : sb(gz, wd);
                // differences to phi first: lap of a smooth field is small
                lap = fm(sp(W), ad(sb(vp, s.phi), sb(vm, s.phi)), lap);
            }
        });
        s.gx = ml(gx, sp(3.0f));
        s.gy = ml(gy, sp(3.0f));
        s.gz = ml(gz, sp(3.0f));
        s.lap = ml(lap, sp(6.0f));
        const int zoff = (z + G.GZ) * G.PXY;
        PairWrites w = wr;
        w.own += zoff;
        const bool wz = WALLS && G.wall[2] && (z == 0 || z == G.NZ - 1);
        w.wa = WALLS && (wa_xy || (ka && wz));
        w.wb = WALLS && (wb_xy || (kb && wz));
        w.edge = wr.a_lo || wr.a_hi || wr.b_hi || w.wa || w.wb;
        if constexpr (HG) {
            // h half first (needs u, n, theta), then Pi and the g half: fewer
            // values live at once than in the joint collision below
            pair_velocity<L::kHasY>(s, p, m.m0, m.mx, m.my, m.mz);
            pair_interface(s, p);
            constexpr float WA = (float)L::w[1], WD = (float)L::w[4];
            const f2 nus[2] = {ml(s.usq, sp(-1.5f * WA)), ml(s.usq, sp(-1.5f * WD))};
            const f2 phw[2] = {ml(s.phi, sp(WA)), ml(s.phi, sp(WD))};
            const f2 thw[2] = {ml(s.theta, sp(WA)), ml(s.theta, sp(WD))};
            f2 hsum = sp(0.0f);
            Unroll<1, Q>::run([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                constexpr int o = L::op[i];
                if constexpr (i < o) {
                    constexpr int K = (L::cx[i] * L::cx[i] + L::cy[i] * L::cy[i] + L::cz[i] * L::cz[i]) == 1 ? 0 : 1;
                    constexpr float W = (float)L::w[i];
                    const float hsh = W * p.h_shift;
                    auto sh = [&](float v) { return St::store(v, hsh, 1.0f); };
                    f2 hsi, hso;
                    collide_pair_h<LAT, i>(s, p, nus[K], phw[K], thw[K], sm.hown[hs][i][tid], sm.hown[hs][o][tid],
                                           hsi, hso);
                    hsum = ad(hsum, ad(hsi, hso));
                    write_pair<LAT, i, WALLS>(D.hout, G, p, z, w, hsi, s.phi, sh);
                    write_pair<LAT, o, WALLS>(D.hout, G, p, z, w, hso, s.phi, sh);
                }
            });
            {
                constexpr float W0 = (float)L::w[0];
                const float hsh = W0 * p.h_shift;
                write_pair<LAT, 0, WALLS>(D.hout, G, p, z, w, sb(s.phi, hsum), s.phi,
                                          [&](float v) { return St::store(v, hsh, 1.0f); });
            }
            pair_pi<L::kHasY>(s, p, m.mxx, m.myy, m.mzz, m.mxy, m.mxz, m.myz);
            PairShared q;
            pair_shared<LAT>(s, p, q);
            Unroll<1, Q>::run([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                constexpr int o = L::op[i];
                if constexpr (i < o) {
                    constexpr float W = (float)L::w[i];
                    const float gsh = W * p.g_shift;
                    auto sg = [&](float v) { return St::store(v, gsh, p.g_scale); };
                    f2 gsi, gso;
                    collide_pair_g<LAT, i>(s, q, p, gsi, gso);
                    write_pair<LAT, i, WALLS>(D.gout, G, p, z, w, gsi, s.rho, sg);
                    write_pair<LAT, o, WALLS>(D.gout, G, p, z, w, gso, s.rho, sg);
                }
            });
            {
                constexpr float W0 = (float)L::w[0];
                const f2 G0 = ml(s.usq, sp(-1.5f * W0));
                const f2 K0 = fm(G0, fm(q.sK, q.neg_ug, q.uF3neg), ml(sp(W0), fm(q.mu3, q.neg_ug, q.uF3neg)));
                const f2 om45w0 = ml(sb(sp(1.0f), s.omega), sp(4.5f * W0));
                const f2 base = sb(ml(s.P, sp(3.0f * W0)), ml(om45w0, s.tr3));
                const f2 g0 = fm(K0, sp(0.5f), fm(s.rho, G0, base));
                const float gsh = W0 * p.g_shift;
                write_pair<LAT, 0, WALLS>(D.gout, G, p, z, w, g0, s.rho,
                                          [&](float v) { return St::store(v, gsh, p.g_scale); });
            }
            continue;
        }
        pair_state<L::kHasY>(s, p, m.m0, m.mx, m.my, m.mz, m.mxx, m.myy, m.mzz, m.mxy, m.mxz, m.myz);
        PairShared q;
        pair_shared<LAT>(s, p, q);
        // moving directions (opposite pairs), then the rest population, which
        // closes sum_i h*_i = phi at each node (Eq. 1 conserves phi)
        f2 hsum = sp(0.0f);
        Unroll<1, Q>::run([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int o = L::op[i];
            if constexpr (i < o) {
                constexpr float W = (float)L::w[i];
                const float hsh = W * p.h_shift, gsh = W * p.g_shift;
                auto sh = [&](float v) { return St::store(v, hsh, 1.0f); };
                auto sg = [&](float v) { return St::store(v, gsh, p.g_scale); };
                f2 hsi, hso, gsi, gso;
                collide_pair2<LAT, i>(s, q, p, sm.hown[hs][i][tid], sm.hown[hs][o][tid], hsi, hso, gsi, gso);
                hsum = ad(hsum, ad(hsi, hso));
                write_pair<LAT, i, WALLS>(D.hout, G, p, z, w, hsi, s.phi, sh);
                write_pair<LAT, o, WALLS>(D.hout, G, p, z, w, hso, s.phi, sh);
                write_pair<LAT, i, WALLS>(D.gout, G, p, z, w, gsi, s.rho, sg);
                write_pair<LAT, o, WALLS>(D.gout, G, p, z, w, gso, s.rho, sg);
            }
        });
        {
            // rest direction (c = 0): G - w = -1.5 w0 u.u, c c : Pi = 0,
            // K = (G - w)(sK (-u.grad) - 3 u.F) + w0 (3 mu (-u.grad) - 3 u.F)
            constexpr float W0 = (float)L::w[0];
            const f2 G0 = ml(s.usq, sp(-1.5f * W0));
            const f2 K0 = fm(G0, fm(q.sK, q.neg_ug, q.uF3neg), ml(sp(W0), fm(q.mu3, q.neg_ug, q.uF3neg)));
            const f2 om45w0 = ml(sb(sp(1.0f), s.omega), sp(4.5f * W0));
            const f2 base = sb(ml(s.P, sp(3.0f * W0)), ml(om45w0, s.tr3));
            const f2 g0 = fm(K0, sp(0.5f), fm(s.rho, G0, base));
            const f2 h0 = sb(s.phi, hsum);
            const float hsh = W0 * p.h_shift, gsh = W0 * p.g_shift;
            write_pair<LAT, 0, WALLS>(D.hout, G, p, z, w, h0, s.phi, [&](float v) { return St::store(v, hsh, 1.0f); });
            write_pair<LAT, 0, WALLS>(D.gout, G, p, z, w, g0, s.rho,
                                      [&](float v) { return St::store(v, gsh, p.g_scale); });
        }
    }
}

template <int LAT, int ST, int TX, int TY, int MINB, bool WALLS, bool GFIRST, bool SRING, bool HG>
__global__ void __launch_bounds__(TX / 2 * TY, MINB)
step_pair_kernel(const DirPtrs<typename Storage<ST>::S, Lattice<LAT>::Q> D, Geom G, PhysT<float> p, int LZ) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<PairSmem<LAT, ST, TX, TY>*>(smem_raw);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * LZ;
    const int z1 = min(z0 + LZ, G.NZ);
    march_pair<LAT, ST, TX, TY, WALLS, GFIRST, SRING, HG>(D, G, p, x0, y0, z0, z1, sm);
}

}  // namespace lbm
