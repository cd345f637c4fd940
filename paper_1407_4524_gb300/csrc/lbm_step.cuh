// lbm_step.cuh -- the kernels of one time step t -> t+1 (templated on the
// lattice L and the precision policy P; instantiated in lbm_fp64.cu and
// lbm_fp32.cu).
//
// Storage convention: the population buffer of step t holds the
// post-collision values fhat(x, t) (Eq. collision) at every fluid node.
//
// FP64 mode (parity), one stream, per step:
//   k_links  : for every cut link (x_F fluid, x_A = x_F - c_i solid) the wall
//              value fhat_i(x_A, t) of Eq. Fillipova_interpolation, stored in
//              the (otherwise unused) slot i of the solid node x_A, and the
//              link's momentum-exchange contributions (Eqs. flow_force_2,
//              flow_torque_2, ForceInMovementMovingFrame,
//              TorqueInMovementMovingFrame), which by Eq. Equalities need
//              exactly that wall value and fhat_ib(x_F, t);
//   k_bulk   : pull-streaming f_i(x, t+1) = fhat_i(x - c_i, t) (Eq.
//              streaming) -- at cut links the pull reads the wall value --,
//              moments (Eqs. LBMmacroscopics_0/1), BGK collision, store;
//   k_finish : per-body sums of the link contributions in link order into the
//              force/torque row of step t; for moving bodies the covered /
//              uncovered nodes A+ / A- (Sec. 3.2.2): impulsive terms of Eqs.
//              ForceInMovement / TorqueInMovement, refill of uncovered nodes.
// Every formula there has the FP64 CPU oracle's operation order, so the FP64
// mode reproduces it bit for bit.
//
// FP32 / FP16 modes: k_bulk skips the boundary nodes (fluid nodes with a solid
// neighbour), which the boundary-node kernel (lbm_bnd.cuh) steps on a second
// stream; k_finish converts the exact fixed-point per-body sums.  Storage is
// f - w, arithmetic FP32.
//
// Every mode: under the Zou-He edge rule k_bulk also skips the nodes of the
// wall and inlet faces, which k_zouhe steps (pull, closure of the entering
// populations, collision).  k_init / k_load set the state (an equilibrium or
// populations given on the host); k_macros reads rho, u back.
#pragma once

#include <type_traits>

#include "lbm_dev.cuh"

namespace lbm {

constexpr int BULK_THREADS = 128;
constexpr int LINK_THREADS = 256;
constexpr int IMP_THREADS = 128;
constexpr int N_COUNTERS = 16; // entries of the device counter array (StepBufs::counters)

struct StepBufs {
    const void *src; // fhat(t)   (k_links also writes wall values into it)
    void *dst;       // fhat(t+1)
    const void *mac_t;
    void *mac_t1;
    uint8_t *flags;
    const uint16_t *owner_t;
    const BodyDev *bodies;
    const int *moving_ids;
    int n_moving;
    const long long *link_cnt; // per body, current link buffer
    const long long *link_pre; // prefix of link_cnt over bodies (nb + 1 entries)
    const long long *tile_pre; // prefix of per-body link tiles (LINK_THREADS links each)
    const double *poses;       // POSE_STRIDE doubles per body
    const uint32_t *Lcell;
    const uint8_t *Ldir;
    const double *Ldelta;
    double *me;
    const long long *apm_cnt;
    const uint32_t *apm_cell;
    const int8_t *apm_sign;
    double *imp;
    double *series;
    unsigned long long *counters; // [0] fallback links, [1] covered, [2] uncovered,
                                  // [3] links of this step, [4] links of the last step,
                                  // [5] unstable flag, [6] timeout flag,
                                  // [7] free body out of range, [8] extrapolation refills,
                                  // [9], [10] step index t of even / odd steps (k_finish
                                  // of step t writes t + 1 into the other one)
    unsigned long long *acc;      // reduced-precision modes: per body SERIES_ROW fixed-point sums
    long long t;
    int par; // parity of the step: its index is counters[9 + par] on the device
    // free-body schemes (Params::free_scheme 1 / 2): what the end-of-step kernel does
    int phase;                    // PH_ALL, PH_REDUCE, PH_IMP or PH_FIX
    double *imp_prev;             // scheme 1: impulsive terms of the last displacement [nb][6]
    const uint32_t *apm_pred_cell; // scheme 2: covered / uncovered lists of the prediction
    const int8_t *apm_pred_sign;
    const long long *apm_pred_cnt;
};

// end-of-step phases: PH_ALL the series row and the impulsive terms with the
// refill of the step's covered / uncovered lists; the schemes of free bodies
// split it into PH_REDUCE (the row of the link sums; a scheme-1 free body's
// impulsive terms are those of its previous displacement) before the body
// moves, PH_IMP (impulsive terms and refill of the lists of the displacement
// made: prescribed bodies into the row, scheme-1 free bodies kept for the next
// step) after it, and PH_FIX (scheme 2: refill of the nodes the recomputed
// displacement uncovers and the predicted one did not)
constexpr int PH_ALL = 0, PH_REDUCE = 1, PH_IMP = 2, PH_FIX = 3;

// scheme 2: did the predicted displacement of body b uncover node A?
__device__ __forceinline__ bool pred_uncovered(const StepBufs &sb, const BodyDev &B, int b, long long A) {
    const long long n = sb.apm_pred_cnt[b];
    for (long long e = 0; e < n; ++e)
        if (sb.apm_pred_cell[B.apm_off + e] == (uint32_t)A && sb.apm_pred_sign[B.apm_off + e] < 0) return true;
    return false;
}

// =================================================================== exact ==
// FP64, operation order of the oracle (one expression per formula).

template <class L>
__device__ __forceinline__ double feq_x(const Params &p, int i, double rho, const double u[3]) {
    double cu = (double)L::cx(i) * u[0] + (double)L::cy(i) * u[1] + (double)L::cz(i) * u[2];
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double w = L::template w<double>(i);
    if (p.eq == 0) return w * (rho + p.rho0 * (3.0 * cu + 4.5 * cu * cu - 1.5 * usq));
    return w * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
}

template <class L>
__device__ __forceinline__ void moments_x(const Params &p, const double f[], double &rho, double u[3]) {
    double r = 0.0, j0 = 0.0, j1 = 0.0, j2 = 0.0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        r += f[i];
        j0 += (double)L::cx(i) * f[i];
        j1 += (double)L::cy(i) * f[i];
        j2 += (double)L::cz(i) * f[i];
    }
    if (p.has_force) {
        j0 += 0.5 * p.g[0];
        j1 += 0.5 * p.g[1];
        j2 += 0.5 * p.g[2];
    }
    double den = p.eq == 0 ? p.rho0 : r;
    rho = r;
    u[0] = j0 / den;
    u[1] = j1 / den;
    u[2] = j2 / den;
}

template <class L>
__device__ __forceinline__ void collide_x(const Params &p, double f[], double rho, const double u[3]) {
    const double omega = p.omega;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        double fi = f[i];
        double v = fi - omega * (fi - feq_x<L>(p, i, rho, u));
        if (p.has_force) {
            double cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
            double cg = cx * p.g[0] + cy * p.g[1] + cz * p.g[2];
            double ug = u[0] * p.g[0] + u[1] * p.g[1] + u[2] * p.g[2];
            double cu = cx * u[0] + cy * u[1] + cz * u[2];
            v = v + (1.0 - 0.5 * omega) * L::template w<double>(i) * (3.0 * (cg - ug) + 9.0 * cu * cg);
        }
        f[i] = v;
    }
}

// fictitious equilibrium g_ib of Eq. Fillipova_equilibrium
__device__ __forceinline__ double geq_x(const Params &p, const LatTab &tb, int ib, double rhoF,
                                        const double ubf[3], const double uF[3]) {
    double c0 = tb.c[ib][0], c1 = tb.c[ib][1], c2 = tb.c[ib][2];
    double cbu = c0 * ubf[0] + c1 * ubf[1] + c2 * ubf[2];
    double cbF = c0 * uF[0] + c1 * uF[1] + c2 * uF[2];
    double uFsq = uF[0] * uF[0] + uF[1] * uF[1] + uF[2] * uF[2];
    if (p.eq == 0) return tb.w[ib] * (rhoF + p.rho0 * (3.0 * cbu + 4.5 * cbF * cbF - 1.5 * uFsq));
    return tb.w[ib] * rhoF * (1.0 + 3.0 * cbu + 4.5 * cbF * cbF - 1.5 * uFsq);
}

// ==================================================================== fast ==
// FP32, deviation form: d = f - w, drho = rho - 1.

template <class L>
__device__ __forceinline__ void moments_f(const Params &p, const float f[], float &drho, float u[3]) {
    float r = 0.f, j0 = 0.f, j1 = 0.f, j2 = 0.f;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        r += f[i];
        if (L::cx(i) == 1) j0 += f[i];
        if (L::cx(i) == -1) j0 -= f[i];
        if (L::cy(i) == 1) j1 += f[i];
        if (L::cy(i) == -1) j1 -= f[i];
        if (L::cz(i) == 1) j2 += f[i];
        if (L::cz(i) == -1) j2 -= f[i];
    }
    if (p.has_force) {
        j0 = fmaf(0.5f, p.gf[0], j0);
        j1 = fmaf(0.5f, p.gf[1], j1);
        j2 = fmaf(0.5f, p.gf[2], j2);
    }
    const float inv = p.eq == 0 ? p.inv_rho0f : 1.0f / (1.0f + r);
    drho = r;
    u[0] = j0 * inv;
    u[1] = j1 * inv;
    u[2] = j2 * inv;
}

// link mode: the moments (drho, u) of f(t) of a node near a body, one float4
// per cell, for the cut links of the next step and the refill
__device__ __forceinline__ void store_mac(float *mac, long long cell, float drho, const float u[3]) {
    reinterpret_cast<float4 *>(mac)[cell] = make_float4(drho, u[0], u[1], u[2]);
}
__device__ __forceinline__ float4 load_mac(const float *mac, long long cell) {
    return reinterpret_cast<const float4 *>(mac)[cell];
}
__device__ __forceinline__ void store_mac(double *, long long, double, const double *) {}

// c_i . u with the lattice components folded in (adds and subtracts only:
// the library is built without contraction, so products with 0 and +-1 are
// not removed by the compiler)
template <class L> __device__ __forceinline__ float cdot_f(int i, const float u[3]) {
    float s = 0.0f;
    bool any = false;
    const int c[3] = {L::cx(i), L::cy(i), L::cz(i)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (c[k] == 0) continue;
        const float t = c[k] > 0 ? u[k] : -u[k];
        s = any ? s + t : t;
        any = true;
    }
    return s;
}

// deviation of the equilibrium, f^eq_i - w_i
template <class L>
__device__ __forceinline__ float dfeq_f(const Params &p, int i, float drho, const float u[3], float usq15) {
    const float cu = cdot_f<L>(i, u);
    float poly = fmaf(cu, fmaf(4.5f, cu, 3.0f), -usq15); // 3cu + 4.5cu^2 - 1.5u^2
    float rr = p.eq == 0 ? p.rho0f : 1.0f + drho;
    return L::template w<float>(i) * fmaf(rr, poly, drho);
}

// BGK relaxation fhat = (1 - omega) f + omega f^eq in the deviation form:
// omega (f^eq_i - w_i) = (w_i omega rho_u) poly_i + w_i omega drho, with the
// two products formed once per weight class (rest, axis, diagonal)
template <class L>
__device__ __forceinline__ void collide_f(const Params &p, float f[], float drho, const float u[3]) {
    const float om = p.omegaf;
    const float usq15 = 1.5f * fmaf(u[0], u[0], fmaf(u[1], u[1], u[2] * u[2]));
    const float rr = p.eq == 0 ? p.rho0f : 1.0f + drho;
    const float omr = om * rr, omd = om * drho;
    // two copies of the loop behind one uniform branch: unforced domains
    // (nearly all) issue none of the Guo source
    if (!p.has_force) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const float cu = cdot_f<L>(i, u);
            const float poly = fmaf(cu, fmaf(4.5f, cu, 3.0f), -usq15); // 3cu + 4.5cu^2 - 1.5u^2
            const float w = L::template w<float>(i);
            f[i] = fmaf(p.keepf, f[i], fmaf(w * omr, poly, w * omd));
        }
        return;
    }
    const float ug = u[0] * p.gf[0] + u[1] * p.gf[1] + u[2] * p.gf[2];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const float cu = cdot_f<L>(i, u);
        const float poly = fmaf(cu, fmaf(4.5f, cu, 3.0f), -usq15);
        const float w = L::template w<float>(i);
        const float v = fmaf(p.keepf, f[i], fmaf(w * omr, poly, w * omd));
        const float cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const float cg = cx * p.gf[0] + cy * p.gf[1] + cz * p.gf[2];
        f[i] = fmaf((1.0f - 0.5f * om) * w, fmaf(9.0f * cu, cg, 3.0f * (cg - ug)), v);
    }
}

__device__ __forceinline__ float dgeq_f(const Params &p, const LatTab &tb, int ib, float drhoF, const float ubf[3],
                                        const float uF[3]) {
    float c0 = tb.c[ib][0], c1 = tb.c[ib][1], c2 = tb.c[ib][2];
    float cbu = c0 * ubf[0] + c1 * ubf[1] + c2 * ubf[2];
    float cbF = c0 * uF[0] + c1 * uF[1] + c2 * uF[2];
    float uFsq = uF[0] * uF[0] + uF[1] * uF[1] + uF[2] * uF[2];
    float poly = 3.0f * cbu + 4.5f * cbF * cbF - 1.5f * uFsq;
    float rr = p.eq == 0 ? p.rho0f : 1.0f + drhoF;
    return (float)tb.w[ib] * fmaf(rr, poly, drhoF);
}

// ========================================================= fixed point ==
// Reduced-precision modes accumulate the per-body momentum-exchange sums in
// 64-bit fixed point (2^-36 resolution, range +-2^27 per body): integer
// addition is exact and associative, so the sums are exact for the FP32
// per-link terms and independent of summation order (atomics are safe and
// the result is deterministic).
constexpr float FX_SCALE = 68719476736.0f; // 2^36
constexpr double FX_INV = 1.0 / 68719476736.0;

__device__ __forceinline__ unsigned long long to_fx(float v) {
    return (unsigned long long)__float2ll_rn(v * FX_SCALE);
}
__device__ __forceinline__ double from_fx(unsigned long long v) { return (double)(long long)v * FX_INV; }

// moments of the stored post-collision populations (reduced-precision
// modes): BGK conserves rho and rho u, so they are the moments of f(t); with
// the Guo force the collided momentum carries one extra g, removed here.
template <class L, class S>
__device__ __forceinline__ void moments_hat(const Params &p, const S *__restrict__ pop, long long cell, float &drho,
                                            float u[3]) {
    float f[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) f[i] = ldP(pop + (long long)i * p.N + cell);
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (p.has_force) {
        g0 = p.gf[0];
        g1 = p.gf[1];
        g2 = p.gf[2];
    }
    float r = 0.f, j0 = -0.5f * g0, j1 = -0.5f * g1, j2 = -0.5f * g2;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        r += f[i];
        j0 += (float)L::cx(i) * f[i];
        j1 += (float)L::cy(i) * f[i];
        j2 += (float)L::cz(i) * f[i];
    }
    const float inv = 1.0f / (p.eq == 0 ? p.rho0f : 1.0f + r);
    drho = r;
    u[0] = j0 * inv;
    u[1] = j1 * inv;
    u[2] = j2 * inv;
}

// ============================================================== streaming ==

// inlet velocity at the wall point of an edge link (x_B = x_F - c_i / 2)
__device__ __forceinline__ double inlet_u(const Params &p, int y, int cy) {
    if (!p.inlet_parabolic) return p.u_in;
    double ny = (double)p.ny;
    double yb = (double)y - 0.5 * (double)cy;
    return 4.0 * p.u_in * (yb + 0.5) * ((ny - 0.5) - yb) / (ny * ny);
}

// Pull of population i at a node on a non-periodic face.  Out-of-range
// sources: wall / inlet links (Delta = 1/2: chi = 0, so the curved-wall rule
// reduces to moving bounce-back with u_B = 0 / the inlet profile), outlet
// copies the last interior column; a wall wins at corners.
template <class L, class P>
__device__ __noinline__ typename P::C pull_edge(const Params &p, const typename P::S *__restrict__ src,
                                                const typename P::C *__restrict__ mac_t, int x, int y, int z,
                                                long long cell, int i) {
    using C = typename P::C;
    int s[3] = {x - L::cx(i), y - L::cy(i), z - L::cz(i)};
    const int n[3] = {p.nx, p.ny, p.nz};
    bool wall = false, inlet = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int side = s[a] < 0 ? 0 : (s[a] >= n[a] ? 1 : -1);
        if (side < 0) continue;
        int e = p.edge[2 * a + side];
        if (e == 0) s[a] += side == 0 ? n[a] : -n[a];
        else if (e == 1) wall = true;
        else if (e == 2) inlet = true;
        else s[a] = n[a] - 1;
    }
    if (wall || inlet) {
        const int ib = L::opp(i);
        C fb = ldS(src + (long long)ib * p.N + cell);
        double uB0 = inlet && !wall ? inlet_u(p, y, L::cy(i)) : 0.0;
        if constexpr (P::exact) {
            double uB[3] = {uB0, 0.0, 0.0};
            double rhow = p.eq == 0 ? p.rho0 : mac_t[4 * cell];
            double cuB = (double)L::cx(i) * uB[0] + (double)L::cy(i) * uB[1] + (double)L::cz(i) * uB[2];
            return fb + 2.0 * L::template w<double>(i) * rhow * 3.0 * cuB;
        } else {
            float rhow = p.rho0f;
            if (p.eq != 0) {
                float dr, uu[3];
                moments_hat<L>(p, src, cell, dr, uu);
                rhow = 1.0f + dr;
            }
            float cuB = (float)L::cx(i) * (float)uB0;
            return fmaf(6.0f * L::template w<float>(i) * rhow, cuB, fb);
        }
    }
    return ldS(src + (long long)i * p.N + cell_of(p, s[0], s[1], s[2]));
}

// Momentum terms of the wall / inlet links of one node (Delta = 1/2, chi = 0:
// moving bounce-back, u_B = 0 on walls, the inlet profile on inlet links; a
// wall wins at corners) -- the same expressions as pull_edge.
template <class L, class P>
__device__ __forceinline__ void face_terms(const Params &p, const typename P::S *__restrict__ src,
                                        const typename P::C *__restrict__ mac_t, int y, long long cell,
                                        unsigned bounce, unsigned inlet_only, typename P::C *f) {
    if constexpr (P::exact) {
        const double rhow = p.eq == 0 ? p.rho0 : mac_t[4 * cell];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            if (!((bounce >> i) & 1u)) continue;
            const double uB0 = ((inlet_only >> i) & 1u) ? inlet_u(p, y, L::cy(i)) : 0.0;
            const double uB[3] = {uB0, 0.0, 0.0};
            const double cuB = (double)L::cx(i) * uB[0] + (double)L::cy(i) * uB[1] + (double)L::cz(i) * uB[2];
            f[i] = f[i] + 2.0 * L::template w<double>(i) * rhow * 3.0 * cuB;
        }
    } else {
        float rhow = p.rho0f;
        if (p.eq != 0) {
            float dr, uu[3];
            moments_hat<L>(p, src, cell, dr, uu);
            rhow = 1.0f + dr;
        }
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            if (!((bounce >> i) & 1u)) continue;
            const double uB0 = ((inlet_only >> i) & 1u) ? inlet_u(p, y, L::cy(i)) : 0.0;
            const float cuB = (float)L::cx(i) * (float)uB0;
            f[i] = fmaf(6.0f * L::template w<float>(i) * rhow, cuB, (float)f[i]);
        }
    }
}

// true when node (x,y,z) lies on a wall or inlet face (of a Zou-He domain)
__device__ __forceinline__ bool zh_node(const Params &p, int x, int y, int z) {
    auto zf = [](int e) { return e == 1 || e == 2; };
    return (x == 0 && zf(p.edge[0])) || (x == p.nx - 1 && zf(p.edge[1])) || (y == 0 && zf(p.edge[2])) ||
           (y == p.ny - 1 && zf(p.edge[3])) || (z == 0 && zf(p.edge[4])) || (z == p.nz - 1 && zf(p.edge[5]));
}

// Zou-He velocity condition on the wall and inlet faces (LBM_EDGE_RULE_ZOUHE;
// the paper's test section imposes its no-slip walls this way, after its
// cited reference).  The face nodes lie ON the boundary with velocity u_w (0
// on walls; u_in or the on-node parabola 4 u_in y (H - y) / H^2, H = ny - 1,
// on the inlet); `unknown` holds the populations whose pull source lies
// beyond such a face (the bounce bits of pull_core), which are closed here
// from the known ones at the same node:
//   one face, outward normal n along `axis` with sign `sgn`:
//     j = rho_u u_w - g/2 (rho_u = rho0, or rho = (S0 + 2 S+ + g.n/2) /
//     (1 + u_w.n) in the standard model), f_i = f_ib + 6 w_i c_i.j -
//     sum_t c_i,t N_t with N_t = T_t / 2 - j_t / 3 and T_t the c_t-moment of
//     the populations with c.n = 0 -- so that the node's momentum is j;
//   two or three faces (edge, corner): u_w = 0 without the force shift,
//     bounce-back of the unknown populations with a known opposite, along
//     the axis of a 3-D edge a correction that cancels the known pairs'
//     momentum, and the unknown pairs share the rest of the density of the
//     inner diagonal neighbour at t (the sum of its fhat) equally.
// FP64: the oracle's operation order.  Reduced precision: the same formulas
// on the deviations f - w (the weights cancel in each of them).
template <class L, class P>
__device__ __forceinline__ void zouhe_fill(const Params &p, const typename P::S *__restrict__ src, int x, int y, int z,
                                        unsigned unknown, typename P::C *f) {
    using C = typename P::C;
    const int pos[3] = {x, y, z}, nn[3] = {p.nx, p.ny, p.nz};
    int nface = 0, axis = 0, sgn = 0, wall = 0, inward[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        const int elo = p.edge[2 * a], ehi = p.edge[2 * a + 1];
        if (pos[a] == 0 && (elo == 1 || elo == 2)) {
            nface++;
            axis = a;
            sgn = -1;
            inward[a] = 1;
            wall |= elo == 1;
        } else if (pos[a] == nn[a] - 1 && (ehi == 1 || ehi == 2)) {
            nface++;
            axis = a;
            sgn = 1;
            inward[a] = -1;
            wall |= ehi == 1;
        }
    }
    auto cc = [](int i, int a) { return a == 0 ? L::cx(i) : (a == 1 ? L::cy(i) : L::cz(i)); };
    if (nface == 1) {
        C uw[3] = {C(0), C(0), C(0)}, g[3] = {C(0), C(0), C(0)}, j[3], T[3] = {C(0), C(0), C(0)};
        if (!wall) {
            if (!p.inlet_parabolic) {
                uw[0] = (C)p.u_in;
            } else {
                const double H = (double)(p.ny - 1);
                uw[0] = (C)(4.0 * p.u_in * (double)y * (H - (double)y) / (H * H));
            }
        }
        if (p.has_force)
            for (int a = 0; a < 3; ++a) g[a] = (C)p.g[a];
        C S0 = C(0), Sp = C(0);
        for (int i = 0; i < L::Q; ++i) {
            const int cn = cc(i, axis) * sgn;
            if (cn == 0) {
                S0 += f[i];
                for (int a = 0; a < 3; ++a) T[a] += (C)cc(i, a) * f[i];
            } else if (cn > 0) {
                Sp += f[i];
            }
        }
        if (p.eq == 0) {
            for (int a = 0; a < 3; ++a) j[a] = (C)p.rho0 * uw[a] - C(0.5) * g[a];
        } else {
            C rho;
            if constexpr (P::exact) rho = ((S0 + 2.0 * Sp) + (double)sgn * (0.5 * g[axis])) / (1.0 + (double)sgn * uw[axis]);
            else rho = ((1.0f + (S0 + 2.0f * Sp)) + (float)sgn * (0.5f * g[axis])) / (1.0f + (float)sgn * uw[axis]);
            for (int a = 0; a < 3; ++a) j[a] = rho * uw[a] - C(0.5) * g[a];
        }
        C Nt[3] = {C(0), C(0), C(0)};
        for (int a = 0; a < 3; ++a)
            if (a != axis) Nt[a] = C(0.5) * T[a] - j[a] / C(3);
        for (int i = 0; i < L::Q; ++i) {
            if (!((unknown >> i) & 1u)) continue;
            const C cj = ((C)L::cx(i) * j[0] + (C)L::cy(i) * j[1]) + (C)L::cz(i) * j[2];
            C v = f[L::opp(i)] + (C(6) * L::template w<C>(i)) * cj;
            for (int a = 0; a < 3; ++a)
                if (a != axis && cc(i, a) != 0) v = v - (C)cc(i, a) * Nt[a];
            f[i] = v;
        }
        return;
    }
    const long long xin = cell_of(p, x + inward[0], y + inward[1], z + inward[2]);
    C rc = C(0); // density of the inner neighbour at t (its deviation in the reduced modes)
    for (int i = 0; i < L::Q; ++i) rc += (C)ldS(src + (long long)i * p.N + xin);
    unsigned buried = 0u;
    int nbur = 0;
    for (int i = 0; i < L::Q; ++i)
        if (((unknown >> i) & 1u) && ((unknown >> L::opp(i)) & 1u)) {
            buried |= 1u << i;
            nbur++;
        }
    for (int i = 0; i < L::Q; ++i)
        if (((unknown >> i) & 1u) && !((buried >> i) & 1u)) f[i] = f[L::opp(i)];
    for (int a = 0; a < 3; ++a) {
        if (inward[a] != 0) continue;
        C T = C(0);
        int m = 0;
        for (int i = 0; i < L::Q; ++i) {
            if (cc(i, a) == 0) continue;
            if (!((unknown >> i) & 1u) && !((unknown >> L::opp(i)) & 1u)) T += (C)cc(i, a) * f[i];
            if (((unknown >> i) & 1u) && !((buried >> i) & 1u)) m++;
        }
        if (m == 0) continue;
        const C Nt = T / (C)m;
        for (int i = 0; i < L::Q; ++i)
            if (((unknown >> i) & 1u) && !((buried >> i) & 1u) && cc(i, a) != 0) f[i] = f[i] - (C)cc(i, a) * Nt;
    }
    C rest = rc;
    for (int i = 0; i < L::Q; ++i)
        if (!((buried >> i) & 1u)) rest = rest - f[i];
    for (int i = 0; i < L::Q; ++i)
        if ((buried >> i) & 1u) f[i] = rest / (C)nbur;
}

__device__ __forceinline__ bool on_edge(const Params &p, int x, int y, int z) {
    return (!p.per[0] && (x == 0 || x == p.nx - 1)) || (!p.per[1] && (y == 0 || y == p.ny - 1)) ||
           (!p.per[2] && (z == 0 || z == p.nz - 1));
}

// Directions whose component along `axis` equals `sgn` (bit i = direction i).
template <class L> __host__ __device__ constexpr unsigned dir_mask(int axis, int sgn) {
    unsigned m = 0u;
    for (int i = 0; i < L::Q; ++i) {
        const int c = axis == 0 ? L::cx(i) : (axis == 1 ? L::cy(i) : L::cz(i));
        if (c == sgn) m |= 1u << i;
    }
    return m;
}

// Source coordinates along one axis for c = +1 (m) and c = -1 (pp), with the
// face rule of pull_edge: periodic faces wrap, an outlet repeats the last
// column, a wall or inlet face makes the link a bounce link.  fl collects,
// per axis a, bounce bits (2a: c = +1, 2a+1: c = -1), wall bits (8 + ...)
// and inlet bits (16 + ...).
__device__ __forceinline__ void face_axis(int v, int n, int per, int e_lo, int e_hi, int axis, int &m, int &pp,
                                          unsigned &fl) {
    m = v - 1;
    pp = v + 1;
    if (v == 0) {
        if (per || e_lo == 0 || e_lo == 3) m = n - 1;
        else fl |= (1u | (e_lo == 1 ? 1u << 8 : 0u) | (e_lo == 2 ? 1u << 16 : 0u)) << (2 * axis);
    }
    if (v == n - 1) {
        if (per || e_hi == 0) pp = 0;
        else if (e_hi == 3) pp = n - 1;
        else fl |= (2u | (e_hi == 1 ? 2u << 8 : 0u) | (e_hi == 2 ? 2u << 16 : 0u)) << (2 * axis);
    }
}

// the direction mask selected by the six per-axis bits of fl starting at bit `base`
template <class L> __device__ __forceinline__ unsigned face_dirs(unsigned fl, int base) {
    return ((fl >> base) & 1u ? dir_mask<L>(0, 1) : 0u) | ((fl >> (base + 1)) & 1u ? dir_mask<L>(0, -1) : 0u) |
           ((fl >> (base + 2)) & 1u ? dir_mask<L>(1, 1) : 0u) | ((fl >> (base + 3)) & 1u ? dir_mask<L>(1, -1) : 0u) |
           ((fl >> (base + 4)) & 1u ? dir_mask<L>(2, 1) : 0u) | ((fl >> (base + 5)) & 1u ? dir_mask<L>(2, -1) : 0u);
}

// load of a stored population, either converted to the compute type or raw
template <class V, class S> __device__ __forceinline__ V ld_as(const S *ptr) {
    if constexpr (std::is_same<V, S>::value) return __ldg(ptr);
    else return ldS(ptr);
}

// The Q source loads of node (x,y,z) into v[] (compute type, or raw storage
// type).  Fully periodic domains, and warps of a non-periodic domain with no
// node on a y or z face, take the plain path, which applies the x-face rule
// per direction (wall / inlet links bounce, an outlet repeats the last
// column) with a few selects; warps with a node on a y or z face take the
// face path, where every direction applies the full face rule.  Both give
// the sources of pull_edge, and all Q loads are issued before any is used.
// Returns the wall / inlet links of the node (their momentum terms are added
// by face_terms) and, in inlet_only, the inlet links not overridden by a
// wall.
// Face modes of the stream-collide kernels: FM_PERIODIC (every axis
// periodic), FM_XFACES (only x non-periodic: channels with periodic cross
// sections), FM_GENERAL (any edges).
constexpr int FM_PERIODIC = 0, FM_XFACES = 1, FM_GENERAL = 2;

// resident blocks of 128 the reduced-precision stream-collide kernels are
// built for: 10 (<= 48 registers, 62.5 % of the warps) where the face code is
// light (periodic domains, x faces only), 8 (<= 64 registers) for the general
// face code; more blocks spill (measured: 12 blocks lose 5 %)
template <int FM> constexpr int bulk_min_blocks() { return FM == FM_GENERAL ? 8 : 10; }

inline int face_mode(const Params &p) {
    if (!p.nonper) return FM_PERIODIC;
    return (p.per[1] && p.per[2]) ? FM_XFACES : FM_GENERAL;
}

template <class L, class P, int FM, class V>
__device__ __forceinline__ unsigned pull_core(const Params &p, const typename P::S *__restrict__ src, int x, int y,
                                              int z, long long cell, V v[], unsigned &inlet_only) {
    inlet_only = 0u;
    bool plain = true;
    if constexpr (FM == FM_GENERAL) {
        const bool yzface = (!p.per[1] && (y == 0 || y == p.ny - 1)) || (!p.per[2] && (z == 0 || z == p.nz - 1));
        plain = !p.nonper || !__any_sync(__activemask(), yzface);
    }
    if (plain) {
        const int ym = y == 0 ? p.ny - 1 : y - 1, yp = y == p.ny - 1 ? 0 : y + 1;
        const int zm = z == 0 ? p.nz - 1 : z - 1, zp = z == p.nz - 1 ? 0 : z + 1;
        // 32-bit in-plane indices (fewer than 2^32 cells) and one wide
        // multiply-add per plane pointer
        const unsigned nx = (unsigned)p.nx, ny = (unsigned)p.ny, N32 = (unsigned)p.N;
        // warps without a node on a non-periodic x face (all but the first and
        // last warp of a row) take the straight loads, with no per-direction
        // selects
        bool xface = false;
        if constexpr (FM != FM_PERIODIC) xface = !p.per[0] && __any_sync(__activemask(), x == 0 || x == p.nx - 1);
        if (!xface) {
            const int xm = x == 0 ? p.nx - 1 : x - 1, xp = x == p.nx - 1 ? 0 : x + 1;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                const int sx = L::cx(i) == 1 ? xm : (L::cx(i) == -1 ? xp : x);
                const int sy = L::cy(i) == 1 ? ym : (L::cy(i) == -1 ? yp : y);
                const int sz = L::cz(i) == 1 ? zm : (L::cz(i) == -1 ? zp : z);
                const unsigned k = ((unsigned)sz * ny + (unsigned)sy) * nx + (unsigned)sx;
                v[i] = ld_as<V>(src + (size_t)N32 * (unsigned)i + k);
            }
            return 0u;
        }
        unsigned bounce = 0u;
        if constexpr (FM != FM_PERIODIC) {
            // x faces: wall / inlet links bounce, an outlet repeats the last column
            int xm = x == 0 ? p.nx - 1 : x - 1, xp = x == p.nx - 1 ? 0 : x + 1;
            const int e_lo = p.edge[0], e_hi = p.edge[1];
            const bool lo_b = x == 0 && (e_lo == 1 || e_lo == 2);
            const bool hi_b = x == p.nx - 1 && (e_hi == 1 || e_hi == 2);
            const bool lo_in = lo_b && e_lo == 2;
            const bool hi_in = hi_b && e_hi == 2;
            if (x == p.nx - 1) xp = p.nx - 1;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                const int sx = L::cx(i) == 1 ? xm : (L::cx(i) == -1 ? xp : x);
                const int sy = L::cy(i) == 1 ? ym : (L::cy(i) == -1 ? yp : y);
                const int sz = L::cz(i) == 1 ? zm : (L::cz(i) == -1 ? zp : z);
                const unsigned k = ((unsigned)sz * ny + (unsigned)sy) * nx + (unsigned)sx;
                const bool b = (L::cx(i) == 1 && lo_b) || (L::cx(i) == -1 && hi_b);
                const typename P::S *plane = src + (size_t)N32 * (unsigned)(b ? L::opp(i) : i);
                v[i] = ld_as<V>(plane + (b ? (unsigned)cell : k));
                bounce |= (b ? 1u : 0u) << i;
                inlet_only |= ((L::cx(i) == 1 && lo_in) || (L::cx(i) == -1 && hi_in) ? 1u : 0u) << i;
            }
        }
        return bounce;
    }
    unsigned bounce = 0u;
    if constexpr (FM == FM_GENERAL) {
        int xm, xp, ym, yp, zm, zp;
        unsigned fl = 0u;
        face_axis(x, p.nx, p.per[0], p.edge[0], p.edge[1], 0, xm, xp, fl);
        face_axis(y, p.ny, p.per[1], p.edge[2], p.edge[3], 1, ym, yp, fl);
        face_axis(z, p.nz, p.per[2], p.edge[4], p.edge[5], 2, zm, zp, fl);
        bounce = face_dirs<L>(fl, 0);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const int sx = L::cx(i) == 1 ? xm : (L::cx(i) == -1 ? xp : x);
            const int sy = L::cy(i) == 1 ? ym : (L::cy(i) == -1 ? yp : y);
            const int sz = L::cz(i) == 1 ? zm : (L::cz(i) == -1 ? zp : z);
            const long long idx = ((bounce >> i) & 1u) ? (long long)L::opp(i) * p.N + cell
                                                       : (long long)i * p.N + cell_of(p, sx, sy, sz);
            v[i] = ld_as<V>(src + idx);
        }
        if (bounce) inlet_only = face_dirs<L>(fl, 16) & ~face_dirs<L>(fl, 8);
    }
    return bounce;
}

// f_i(x, t+1) for all i at node (x,y,z): the pulls of pull_core plus the
// momentum terms of the node's wall / inlet links
template <class L, class P, int FM = FM_GENERAL>
__device__ __forceinline__ void pull_all(const Params &p, const typename P::S *__restrict__ src,
                                         const typename P::C *__restrict__ mac_t, int x, int y, int z,
                                         long long cell, typename P::C f[]) {
    unsigned inlet_only;
    const unsigned bounce = pull_core<L, P, FM>(p, src, x, y, z, cell, f, inlet_only);
    if constexpr (FM != FM_PERIODIC) {
        if (bounce) face_terms<L, P>(p, src, mac_t, y, cell, bounce, inlet_only, f);
    }
}


// ================================================================== kernels ==

// f(x,0) = f^eq(1, u0); store fhat(x,0) and the moments of f(x,0)
template <class L, class P>
__global__ void __launch_bounds__(BULK_THREADS) k_init(Params p, typename P::S *__restrict__ dst,
                                                       typename P::C *__restrict__ mac,
                                                       const uint8_t *__restrict__ flags, double u0x, double u0y,
                                                       double u0z) {
    using C = typename P::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= p.nx) return;
    const long long cell = cell_of(p, x, y, z);
    const bool mac_here = flags[cell] & FL_MAC;
    C f[L::Q];
    if constexpr (P::exact) {
        double u0[3] = {u0x, u0y, u0z};
        for (int i = 0; i < L::Q; ++i) f[i] = feq_x<L>(p, i, 1.0, u0);
        double rho, u[3];
        moments_x<L>(p, f, rho, u);
        if (mac_here) {
            mac[4 * cell] = rho;
            mac[4 * cell + 1] = u[0];
            mac[4 * cell + 2] = u[1];
            mac[4 * cell + 3] = u[2];
        }
        collide_x<L>(p, f, rho, u);
    } else {
        float u0[3] = {(float)u0x, (float)u0y, (float)u0z};
        const float usq15 = 1.5f * (u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2]);
        for (int i = 0; i < L::Q; ++i) f[i] = dfeq_f<L>(p, i, 0.0f, u0, usq15);
        float drho, u[3];
        moments_f<L>(p, f, drho, u);
        if (p.linkmode && mac_here) store_mac(mac, cell, drho, u);
        collide_f<L>(p, f, drho, u);
    }
    for (int i = 0; i < L::Q; ++i) stS(dst + (long long)i * p.N + cell, f[i]);
}

// f(x, t) given on the host (FP64, staged as [Q][n] for the cells c0 ..
// c0 + n - 1): moments (kept at the FL_MAC nodes in FP64 mode), collision,
// store of fhat(x, t) -- the state the next step starts from, as after k_init
template <class L, class P>
__global__ void __launch_bounds__(BULK_THREADS) k_load(Params p, const double *__restrict__ stage, long long c0,
                                                       long long n, typename P::S *__restrict__ dst,
                                                       typename P::C *__restrict__ mac,
                                                       const uint8_t *__restrict__ flags) {
    using C = typename P::C;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long cell = c0 + k;
    C f[L::Q];
    if constexpr (P::exact) {
        for (int i = 0; i < L::Q; ++i) f[i] = stage[(long long)i * n + k];
        double rho, u[3];
        moments_x<L>(p, f, rho, u);
        if (flags[cell] & FL_MAC) {
            mac[4 * cell] = rho;
            mac[4 * cell + 1] = u[0];
            mac[4 * cell + 2] = u[1];
            mac[4 * cell + 3] = u[2];
        }
        collide_x<L>(p, f, rho, u);
    } else {
        for (int i = 0; i < L::Q; ++i) f[i] = (float)(stage[(long long)i * n + k] - L::template w<double>(i));
        float drho, u[3];
        moments_f<L>(p, f, drho, u);
        if (p.linkmode && (flags[cell] & FL_MAC)) store_mac(mac, cell, drho, u);
        collide_f<L>(p, f, drho, u);
    }
    for (int i = 0; i < L::Q; ++i) stS(dst + (long long)i * p.N + cell, f[i]);
}

// rho(x, t), u(x, t) of the cells c0 .. c0 + n - 1 from the stored fhat(x, t):
// the collision keeps rho and adds the body force g to sum_i c_i f_i, so
// rho_u u = sum_i c_i fhat_i - g/2 (rho_u = rho0, or rho in the standard
// model); out[4][n], zero at solid nodes
template <class L, class P>
__global__ void __launch_bounds__(BULK_THREADS) k_macros(Params p, const typename P::S *__restrict__ src,
                                                         const uint16_t *__restrict__ owner, long long c0,
                                                         long long n, double *__restrict__ out) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long cell = c0 + k;
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    if (owner[cell] == 0) { // fluid at t
        for (int i = 0; i < L::Q; ++i) {
            double v = (double)ldS(src + (long long)i * p.N + cell);
            if constexpr (!P::exact) v += L::template w<double>(i);
            r += v;
            j[0] += (double)L::cx(i) * v;
            j[1] += (double)L::cy(i) * v;
            j[2] += (double)L::cz(i) * v;
        }
        const double den = p.eq == 0 ? p.rho0 : r;
        for (int a = 0; a < 3; ++a) j[a] = (j[a] - 0.5 * p.g[a]) / den;
    }
    out[k] = r;
    for (int a = 0; a < 3; ++a) out[(long long)(a + 1) * n + k] = j[a];
}

// pull-stream + moments + BGK collision of one node (x, y, z)
template <class L, class P, int FM = FM_GENERAL>
__device__ __forceinline__ void bulk_node(const Params &p, const typename P::S *__restrict__ src,
                                          typename P::S *__restrict__ dst, const uint8_t *__restrict__ flags,
                                          const typename P::C *__restrict__ mac_t, typename P::C *__restrict__ mac_t1,
                                          int x, int y, int z) {
    using C = typename P::C;
    if constexpr (FM != FM_PERIODIC) {
        if (p.zouhe && zh_node(p, x, y, z)) return; // Zou-He face nodes: k_zouhe
    }
    const long long cell = cell_of(p, x, y, z);
    const uint8_t fl = __ldg(flags + cell);
    if constexpr (P::exact) {
        if (fl & FL_SOLID) return;
    }
    // reduced precision: the pulls do not wait for the flag (a solid node, or
    // a boundary node left to k_bnd, is stepped and not stored), so the flag
    // load and the population loads are in flight together
    bool store = true;
    if constexpr (!P::exact) store = !(fl & FL_SOLID) && (p.linkmode || !(fl & FL_BND));
    C f[L::Q];
    pull_all<L, P, FM>(p, src, mac_t, x, y, z, cell, f);
    if constexpr (P::exact) {
        double rho, u[3];
        moments_x<L>(p, f, rho, u);
        if (fl & FL_MAC) {
            mac_t1[4 * cell] = rho;
            mac_t1[4 * cell + 1] = u[0];
            mac_t1[4 * cell + 2] = u[1];
            mac_t1[4 * cell + 3] = u[2];
        }
        collide_x<L>(p, f, rho, u);
    } else {
        float drho, u[3];
        moments_f<L>(p, f, drho, u);
        if (store && p.linkmode && (fl & FL_MAC)) store_mac(mac_t1, cell, drho, u);
        collide_f<L>(p, f, drho, u);
    }
    if (!store) return;
    const unsigned N32 = (unsigned)p.N, c32 = (unsigned)cell;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) stS(dst + (size_t)N32 * (unsigned)i + c32, f[i]);
}

// pull-stream + moments + BGK collision over every fluid node
template <class L, class P, int FM>
__global__ void __launch_bounds__(BULK_THREADS, P::exact ? 4 : bulk_min_blocks<FM>()) k_bulk(Params p, const typename P::S *__restrict__ src,
                                                       typename P::S *__restrict__ dst,
                                                       const uint8_t *__restrict__ flags,
                                                       const typename P::C *__restrict__ mac_t,
                                                       typename P::C *__restrict__ mac_t1) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= p.nx) return;
    bulk_node<L, P, FM>(p, src, dst, flags, mac_t, mac_t1, x, y, z);
}

// Zou-He face nodes (the bulk kernel skips them): pull, closure of the
// populations entering from outside (zouhe_fill), moments, BGK collision,
// store.  One thread per node of a face plane, blockIdx.z = face (x-lo, x-hi,
// y-lo, y-hi, z-lo, z-hi); a node on several Zou-He faces is taken by the
// first of them.
template <class L, class P>
__global__ void __launch_bounds__(BULK_THREADS) k_zouhe(Params p, const typename P::S *__restrict__ src,
                                                        typename P::S *__restrict__ dst,
                                                        const uint8_t *__restrict__ flags,
                                                        const typename P::C *__restrict__ mac_t,
                                                        typename P::C *__restrict__ mac_t1) {
    using C = typename P::C;
    const int face = blockIdx.z, a = face >> 1, side = face & 1;
    auto zf = [](int e) { return e == 1 || e == 2; };
    if (!zf(p.edge[face])) return;
    const int nn[3] = {p.nx, p.ny, p.nz};
    const int au = a == 0 ? 1 : 0, av = a == 2 ? 1 : 2;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)nn[au] * nn[av]) return;
    int q[3];
    q[a] = side ? nn[a] - 1 : 0;
    q[au] = (int)(k % nn[au]);
    q[av] = (int)(k / nn[au]);
    for (int f = 0; f < face; ++f)
        if (zf(p.edge[f]) && q[f >> 1] == ((f & 1) ? nn[f >> 1] - 1 : 0)) return;
    const int x = q[0], y = q[1], z = q[2];
    const long long cell = cell_of(p, x, y, z);
    const uint8_t fl = __ldg(flags + cell);
    if (fl & FL_SOLID) return;
    C f[L::Q];
    unsigned inlet_only;
    const unsigned unknown = pull_core<L, P, FM_GENERAL>(p, src, x, y, z, cell, f, inlet_only);
    zouhe_fill<L, P>(p, src, x, y, z, unknown, f);
    if constexpr (P::exact) {
        double rho, u[3];
        moments_x<L>(p, f, rho, u);
        if (fl & FL_MAC) {
            mac_t1[4 * cell] = rho;
            mac_t1[4 * cell + 1] = u[0];
            mac_t1[4 * cell + 2] = u[1];
            mac_t1[4 * cell + 3] = u[2];
        }
        collide_x<L>(p, f, rho, u);
    } else {
        float drho, u[3];
        moments_f<L>(p, f, drho, u);
        if (p.linkmode && (fl & FL_MAC)) store_mac(mac_t1, cell, drho, u);
        collide_f<L>(p, f, drho, u);
    }
    for (int i = 0; i < L::Q; ++i) stS(dst + (long long)i * p.N + cell, f[i]);
}

// Work of one cut link j of body b: the wall value fhat_i(x_A, t) of Eq.
// Fillipova_interpolation is stored in slot i of the solid node x_A (so the
// pull of k_bulk reads it), and the link's momentum-exchange contributions
// are returned in out[12]: static force, static torque (Eqs. flow_force_2,
// flow_torque_2), moving-frame force and torque (Eqs.
// ForceInMovementMovingFrame / TorqueInMovementMovingFrame); by Eq.
// Equalities they need exactly the wall value and fhat_ib(x_F, t).
template <class L, class P>
__device__ __forceinline__ void link_work(const Params &p, const StepBufs &sb, const LatTab &tb,
                                          const BodyDev &B, const double *X, long long j, double out[ME_PER_LINK],
                                          float outf[ME_PER_LINK]) {
    using S = typename P::S;
    using C = typename P::C;
    S *pop = (S *)sb.src;
    const C *mac = (const C *)sb.mac_t;
    (void)mac;
    const long long N = p.N;
    const long long cell = sb.Lcell[j];
    const int i = sb.Ldir[j];
    const double delta = sb.Ldelta[j];
    int x, y, z;
    coords_of(p, cell, x, y, z);
    const int cxi = tb.c[i][0], cyi = tb.c[i][1], czi = tb.c[i][2];
    const int ib = tb.opp[i];
    const long long A =
        cell_of(p, wrap_axis(x - cxi, p.nx), wrap_axis(y - cyi, p.ny), wrap_axis(z - czi, p.nz));
    double d[3], uB[3];
    if constexpr (P::exact) {
        double rB[3];
        disp(p, X, x, y, z, d);
        rB[0] = d[0] - delta * cxi;
        rB[1] = d[1] - delta * cyi;
        rB[2] = d[2] - delta * czi;
        body_velocity(B, rB, uB);
    } else { // FP32 link geometry (reduced-precision modes)
        const double *Pf = X + 9; // floor(Xw), frac(Xw)
        const int c3[3] = {x, y, z};
        float df[3], rb[3];
        for (int a = 0; a < 3; ++a) df[a] = frame_axis(c3[a] - (int)Pf[a], (float)Pf[3 + a], axis_len(p, a), p.per[a]);
        const float dl = (float)delta;
        rb[0] = df[0] - dl * cxi;
        rb[1] = df[1] - dl * cyi;
        rb[2] = df[2] - dl * czi;
        const float W0 = (float)B.W[0], W1 = (float)B.W[1], W2 = (float)B.W[2];
        uB[0] = (float)B.U[0] + (W1 * rb[2] - W2 * rb[1]);
        uB[1] = (float)B.U[1] + (W2 * rb[0] - W0 * rb[2]);
        uB[2] = (float)B.U[2] + (W0 * rb[1] - W1 * rb[0]);
        d[0] = df[0];
        d[1] = df[1];
        d[2] = df[2];
    }
    // u_G = u(x_F + c_i, t) for Delta < 1/2 (Sec. 2.1)
    long long G = -1;
    if (delta < 0.5) {
        int g[3] = {x + cxi, y + cyi, z + czi};
        const int n[3] = {p.nx, p.ny, p.nz};
        bool ok = true;
        for (int a = 0; a < 3; ++a) {
            if (g[a] >= 0 && g[a] < n[a]) continue;
            if (!p.per[a]) ok = false;
            else g[a] += g[a] < 0 ? n[a] : -n[a];
        }
        if (ok) {
            G = cell_of(p, g[0], g[1], g[2]);
            if (sb.owner_t[G] != 0) G = -1;
        }
        if (G < 0) atomicAdd(&sb.counters[0], 1ull);
    }
    double fa, fb, ps[3], pm[3];
    if constexpr (P::exact) {
        fb = ldP(pop + (long long)ib * N + cell);
        const double rhoF = mac[4 * cell];
        const double uF[3] = {mac[4 * cell + 1], mac[4 * cell + 2], mac[4 * cell + 3]};
        double ubf[3], chi;
        if (delta < 0.5) {
            if (G >= 0) {
                for (int a = 0; a < 3; ++a) ubf[a] = mac[4 * G + 1 + a];
                chi = (2.0 * delta - 1.0) / (p.tau - 2.0);
            } else {
                for (int a = 0; a < 3; ++a) ubf[a] = uF[a];
                chi = 0.0;
            }
        } else {
            double k3 = 3.0 / (2.0 * delta);
            for (int a = 0; a < 3; ++a) ubf[a] = uF[a] + k3 * (uB[a] - uF[a]);
            chi = (2.0 * delta - 1.0) / (p.tau + 0.5);
        }
        double g = geq_x(p, tb, ib, rhoF, ubf, uF);
        double rhow = p.eq == 0 ? p.rho0 : rhoF;
        double cuB = (double)cxi * uB[0] + (double)cyi * uB[1] + (double)czi * uB[2];
        double bc = (1.0 - chi) * fb + chi * g + 2.0 * tb.w[i] * rhow * 3.0 * cuB;
        stS(pop + (long long)i * N + A, bc);
        fa = bc;
        double sum = fa + fb;
        ps[0] = -cxi * sum;
        ps[1] = -cyi * sum;
        ps[2] = -czi * sum;
        const int cb[3] = {-cxi, -cyi, -czi};
        const int cc[3] = {cxi, cyi, czi};
        for (int a = 0; a < 3; ++a) pm[a] = -(cc[a] - uB[a]) * fa + (cb[a] - uB[a]) * fb;
    } else {
        const float fbf = ldP(pop + (long long)ib * N + cell);
        // moments of f(t) at x_F (and at x_F + c_i): kept by the previous
        // stream-collide pass (or the refill, or the initial state)
        const float *macf = (const float *)sb.mac_t;
        const float4 mF = load_mac(macf, cell);
        const float drF = mF.x;
        const float uF[3] = {mF.y, mF.z, mF.w};
        // stability check at the fluid end of every cut link: a NaN or
        // |u| > 0.3 marks the solve unstable (counters[5]; LBM_ERR_UNSTABLE)
        if (!(uF[0] * uF[0] + uF[1] * uF[1] + uF[2] * uF[2] < 0.09f)) atomicOr(&sb.counters[5], 1ull);
        float ubf[3], chi;
        const float dl = (float)delta;
        if (delta < 0.5) {
            if (G >= 0) {
                const float4 mG = load_mac(macf, G);
                ubf[0] = mG.y;
                ubf[1] = mG.z;
                ubf[2] = mG.w;
                chi = (2.0f * dl - 1.0f) / ((float)p.tau - 2.0f);
            } else {
                ubf[0] = uF[0];
                ubf[1] = uF[1];
                ubf[2] = uF[2];
                chi = 0.0f;
            }
        } else {
            const float k3 = 3.0f / (2.0f * dl);
            for (int a = 0; a < 3; ++a) ubf[a] = fmaf(k3, (float)uB[a] - uF[a], uF[a]);
            chi = (2.0f * dl - 1.0f) / ((float)p.tau + 0.5f);
        }
        const float g = dgeq_f(p, tb, ib, drF, ubf, uF);
        const float rhow = p.eq == 0 ? p.rho0f : 1.0f + drF;
        const float cuB = cxi * (float)uB[0] + cyi * (float)uB[1] + czi * (float)uB[2];
        const float bc = fmaf(6.0f * (float)tb.w[i] * rhow, cuB, fmaf(chi, g - fbf, fbf));
        stS(pop + (long long)i * N + A, bc);
        fa = (double)roundS(pop, bc);
        fb = (double)fbf;
        // deviation form: the constant parts -2 w_i c_i cancel over the
        // closed link set of a body (N_i = N_ib on every lattice line);
        // per-link products in FP32, the per-body sums in FP64
        const float sum = (float)fa + fbf, dif = (float)fa - fbf;
        const float d0 = (float)d[0], d1 = (float)d[1], d2 = (float)d[2];
        const float s0 = -cxi * sum, s1 = -cyi * sum, s2 = -czi * sum;
        const float m0 = fmaf((float)uB[0], dif, s0), m1 = fmaf((float)uB[1], dif, s1),
                    m2 = fmaf((float)uB[2], dif, s2);
        outf[0] = s0;
        outf[1] = s1;
        outf[2] = s2;
        outf[3] = d1 * s2 - d2 * s1;
        outf[4] = d2 * s0 - d0 * s2;
        outf[5] = d0 * s1 - d1 * s0;
        outf[6] = m0;
        outf[7] = m1;
        outf[8] = m2;
        outf[9] = d1 * m2 - d2 * m1;
        outf[10] = d2 * m0 - d0 * m2;
        outf[11] = d0 * m1 - d1 * m0;
        return;
    }
    double ts[3], tm[3];
    cross3(d, ps, ts);
    cross3(d, pm, tm);
    out[0] = ps[0];
    out[1] = ps[1];
    out[2] = ps[2];
    out[3] = ts[0];
    out[4] = ts[1];
    out[5] = ts[2];
    out[6] = pm[0];
    out[7] = pm[1];
    out[8] = pm[2];
    out[9] = tm[0];
    out[10] = tm[1];
    out[11] = tm[2];
}

// wall values on cut links + per-link momentum-exchange contributions.
// FP64 mode: one thread per link over a global index, contributions stored
// per link and summed by k_finish in link order.  Reduced-precision modes:
// each block iteration takes one tile of LINK_THREADS consecutive links of
// one body and sums the tile in FP64 (fixed order), so k_finish only adds a
// few tile partials per body.
template <class L, class P>
__global__ void __launch_bounds__(LINK_THREADS) k_links(Params p, StepBufs sb) {
    __shared__ LatTab tb;
    if (threadIdx.x == 0) tb = make_tab<L>();
    __syncthreads();
    if constexpr (P::exact) {
        const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        const long long gsz = (long long)gridDim.x * blockDim.x;
        const long long total = sb.link_pre[p.nb];
        for (long long k = gtid; k < total; k += gsz) {
            int b = 0, hi = p.nb;
            while (hi - b > 1) {
                const int mid = (b + hi) >> 1;
                if (sb.link_pre[mid] <= k) b = mid;
                else hi = mid;
            }
            const BodyDev &B = sb.bodies[b];
            const double *X = sb.poses + (long long)b * POSE_STRIDE + 3;
            const long long j = B.link_off + (k - sb.link_pre[b]);
            double out[ME_PER_LINK];
            float outf[ME_PER_LINK];
            link_work<L, P>(p, sb, tb, B, X, j, out, outf);
            const long long st = p.me_stride;
            for (int c = 0; c < ME_PER_LINK; ++c) sb.me[c * st + j] = out[c];
        }
    } else {
        // tile -> body map in shared memory (binary search), global beyond 1024 bodies
        __shared__ long long tp_s[1025];
        __shared__ unsigned long long part[LINK_THREADS / 32][ME_PER_LINK];
        const bool in_smem = p.nb < 1025;
        if (in_smem)
            for (int k = threadIdx.x; k <= p.nb; k += blockDim.x) tp_s[k] = sb.tile_pre[k];
        __syncthreads();
        const long long *tp = in_smem ? tp_s : sb.tile_pre;
        const long long tiles = tp[p.nb];
        const int lane = threadIdx.x & 31;
        for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
            int b = 0, hi = p.nb;
            while (hi - b > 1) {
                const int mid = (b + hi) >> 1;
                if (tp[mid] <= tile) b = mid;
                else hi = mid;
            }
            const BodyDev &B = sb.bodies[b];
            const double *X = sb.poses + (long long)b * POSE_STRIDE + 3;
            const long long k = (tile - tp[b]) * LINK_THREADS + threadIdx.x;
            // appended lists count past a full segment; only its links exist
            const long long cnt = min(sb.link_cnt[b], B.link_cap);
            double out[ME_PER_LINK];
            float outf[ME_PER_LINK];
            for (int c = 0; c < ME_PER_LINK; ++c) outf[c] = 0.0f;
            if (k < cnt) link_work<L, P>(p, sb, tb, B, X, B.link_off + k, out, outf);
            // the tile's sums: warp shuffles, then one atomic per block and
            // component (every tile of a body adds into the same 12 words)
            const int wid = threadIdx.x >> 5;
#pragma unroll
            for (int c = 0; c < ME_PER_LINK; ++c) {
                unsigned long long v = to_fx(outf[c]);
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane == 0) part[wid][c] = v;
            }
            __syncthreads();
            if (threadIdx.x < ME_PER_LINK) {
                unsigned long long v = 0ull;
                for (int w = 0; w < LINK_THREADS / 32; ++w) v += part[w][threadIdx.x];
                const int c = threadIdx.x;
                if (v) atomicAdd(sb.acc + (long long)b * SERIES_ROW + (c < 6 ? c : c + 6), v);
            }
            __syncthreads();
        }
    }
}

// covered (sign +1) and uncovered (sign -1) nodes of one moving body:
// impulsive terms and refill (one CTA per moving body)
// Extrapolation refill (LBM_REFILL_EXTRAP; the extrapolation proposal the
// paper cites in Sec. 3, after Eq. ForceInMovement): the uncovered node A
// takes f_i(A, t+1) = 3 fhat_i(A + c*, t) - 3 fhat_i(A + 2c*, t) + fhat_i(A + 3c*, t)
// along the lattice direction c* closest to the outward normal n of the body
// at t+1 through A (largest n.c / |c|, the first in direction order): n is the
// gradient of the shape function (r for a sphere, (r_x, r_y, 0) for a
// cylinder, the body-axes gradient (xi / R^2, eta / R2^2) turned back for an
// ellipse).  The three cells must lie in the lattice (periodic axes wrap) and
// be fluid at t; returns 0 when they do not (the equilibrium rule then
// applies), else the index of c* with the three cells.
template <class L>
__device__ __forceinline__ int extrap_cells(const Params &p, const BodyDev &B, const double *X1, const uint16_t *owner_t,
                                            int x, int y, int z, long long cells[3]) {
    // every product and sum explicitly rounded (no contraction, whatever the
    // unit's build flags): the choice of c* is the oracle's
    double r1[3], n[3];
    disp(p, X1, x, y, z, r1);
    if (B.shape == 2) {
        const double co = X1[15], si = X1[16]; // orientation at t+1
        const double xi = __dadd_rn(__dmul_rn(co, r1[0]), __dmul_rn(si, r1[1]));
        const double eta = __dsub_rn(__dmul_rn(co, r1[1]), __dmul_rn(si, r1[0]));
        const double gx = __ddiv_rn(xi, __dmul_rn(B.R, B.R)), gy = __ddiv_rn(eta, __dmul_rn(B.R2, B.R2));
        n[0] = __dsub_rn(__dmul_rn(co, gx), __dmul_rn(si, gy));
        n[1] = __dadd_rn(__dmul_rn(si, gx), __dmul_rn(co, gy));
        n[2] = 0.0;
    } else {
        n[0] = r1[0];
        n[1] = r1[1];
        n[2] = B.shape == 1 ? r1[2] : 0.0;
    }
    int best = 0;
    double top = 0.0;
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        const double sdot = __dadd_rn(__dadd_rn(__dmul_rn((double)L::cx(i), n[0]), __dmul_rn((double)L::cy(i), n[1])),
                                      __dmul_rn((double)L::cz(i), n[2]));
        const int len2 = L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i);
        const double score = len2 == 1 ? sdot : __dmul_rn(sdot, 0.70710678118654752440);
        if (best == 0 || score > top) {
            best = i;
            top = score;
        }
    }
    const int c[3] = {L::cx(best), L::cy(best), L::cz(best)};
    const int nn[3] = {p.nx, p.ny, p.nz};
    const int o[3] = {x, y, z};
    for (int k = 1; k <= 3; ++k) {
        int q[3];
        for (int a = 0; a < 3; ++a) {
            q[a] = o[a] + k * c[a];
            if (q[a] >= 0 && q[a] < nn[a]) continue;
            if (!p.per[a]) return 0;
            q[a] = ((q[a] % nn[a]) + nn[a]) % nn[a];
        }
        const long long cq = cell_of(p, q[0], q[1], q[2]);
        if (owner_t[cq] != 0) return 0;
        cells[k - 1] = cq;
    }
    return best;
}

template <class L, class P>
__device__ __forceinline__ void imp_body_exact(const Params &p, const StepBufs &sb, int b) {
    using S = typename P::S;
    using C = typename P::C;
    __shared__ double part[IMP_THREADS][6];
    __shared__ int sgn[IMP_THREADS];
    const BodyDev &B = sb.bodies[b];
    const long long cnt = sb.apm_cnt[b];
    const S *src = (const S *)sb.src;
    S *dst = (S *)sb.dst;
    const C *mac_t = (const C *)sb.mac_t;
    C *mac_t1 = (C *)sb.mac_t1;
    const double *X = sb.poses + (long long)b * POSE_STRIDE + 3;  // wrapped pose at t
    const double *X1 = sb.poses + (long long)b * POSE_STRIDE + 9; // wrapped pose at t+1
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long base = 0; base < cnt; base += IMP_THREADS) {
        const long long e = base + threadIdx.x;
        const long long A0 = e < cnt ? sb.apm_cell[B.apm_off + e] : 0;
        const int s0 = e < cnt ? sb.apm_sign[B.apm_off + e] : 0;
        // PH_FIX: only the nodes uncovered now and not by the prediction
        const bool skip = sb.phase == PH_FIX && (s0 > 0 || pred_uncovered(sb, B, b, A0));
        if (e < cnt && skip) sgn[threadIdx.x] = 0;
        if (e < cnt && !skip) {
            const long long A = A0;
            const int s = s0;
            int x, y, z;
            coords_of(p, A, x, y, z);
            double m[3] = {0.0, 0.0, 0.0};
            if (s > 0) { // covered: the streamed values f_i(A, t+1)
                C f[L::Q];
                pull_all<L, P>(p, (const S *)src, mac_t, x, y, z, A, f);
                for (int i = 0; i < L::Q; ++i) {
                    m[0] += (double)L::cx(i) * (double)f[i];
                    m[1] += (double)L::cy(i) * (double)f[i];
                    m[2] += (double)L::cz(i) * (double)f[i];
                }
                atomicAdd(&sb.counters[1], 1ull);
            } else { // uncovered: refill f(A, t+1) = f^eq(rho_bar, u_B or u_bar)
                double r1[3], uB[3];
                disp(p, X1, x, y, z, r1);
                body_velocity(B, r1, uB);
                double sum = 0.0, us[3] = {0.0, 0.0, 0.0};
                int nn = 0;
                for (int i = 1; i < L::Q; ++i) {
                    int q[3] = {x + L::cx(i), y + L::cy(i), z + L::cz(i)};
                    const int n[3] = {p.nx, p.ny, p.nz};
                    bool ok = true;
                    for (int a = 0; a < 3; ++a) {
                        if (q[a] >= 0 && q[a] < n[a]) continue;
                        if (!p.per[a]) ok = false;
                        else q[a] += q[a] < 0 ? n[a] : -n[a];
                    }
                    if (!ok) continue;
                    const long long nb = cell_of(p, q[0], q[1], q[2]);
                    if (sb.owner_t[nb] != 0) continue;
                    sum += (double)mac_t[4 * nb];
                    for (int a = 0; a < 3; ++a) us[a] += (double)mac_t[4 * nb + 1 + a];
                    nn++;
                }
                C f[L::Q];
                long long ec[3];
                const bool ex = p.refill == 2 && extrap_cells<L>(p, B, X1, sb.owner_t, x, y, z, ec) != 0;
                if (ex) {
                    for (int i = 0; i < L::Q; ++i) {
                        const S *fi = src + (long long)i * p.N;
                        f[i] = ((C)3 * (C)ldP(fi + ec[0]) - (C)3 * (C)ldP(fi + ec[1])) + (C)ldP(fi + ec[2]);
                    }
                }
                if constexpr (P::exact) {
                    double rbar = nn ? sum / (double)nn : p.rho0;
                    double uf[3];
                    for (int a = 0; a < 3; ++a) uf[a] = (p.refill == 1 && nn) ? us[a] / (double)nn : uB[a];
                    if (!ex)
                        for (int i = 0; i < L::Q; ++i) f[i] = feq_x<L>(p, i, rbar, uf);
                    for (int i = 0; i < L::Q; ++i) {
                        m[0] += (double)L::cx(i) * f[i];
                        m[1] += (double)L::cy(i) * f[i];
                        m[2] += (double)L::cz(i) * f[i];
                    }
                    double rho, u[3];
                    moments_x<L>(p, f, rho, u);
                    mac_t1[4 * A] = rho;
                    mac_t1[4 * A + 1] = u[0];
                    mac_t1[4 * A + 2] = u[1];
                    mac_t1[4 * A + 3] = u[2];
                    collide_x<L>(p, f, rho, u);
                } else {
                    float drb = nn ? (float)(sum / (double)nn) : 0.0f;
                    float uf[3];
                    for (int a = 0; a < 3; ++a) uf[a] = (float)((p.refill == 1 && nn) ? us[a] / (double)nn : uB[a]);
                    const float usq15 = 1.5f * (uf[0] * uf[0] + uf[1] * uf[1] + uf[2] * uf[2]);
                    if (!ex)
                        for (int i = 0; i < L::Q; ++i) f[i] = dfeq_f<L>(p, i, drb, uf, usq15);
                    for (int i = 0; i < L::Q; ++i) {
                        m[0] += (double)L::cx(i) * (double)f[i];
                        m[1] += (double)L::cy(i) * (double)f[i];
                        m[2] += (double)L::cz(i) * (double)f[i];
                    }
                    float drho, u[3];
                    moments_f<L>(p, f, drho, u);
                    reinterpret_cast<float4 *>(mac_t1)[A] = make_float4(drho, u[0], u[1], u[2]);
                    collide_f<L>(p, f, drho, u);
                }
                for (int i = 0; i < L::Q; ++i) stS(dst + (long long)i * p.N + A, f[i]);
                atomicAdd(&sb.counters[2], 1ull);
                if (ex) atomicAdd(&sb.counters[8], 1ull);
            }
            double r[3], tq[3];
            disp(p, X, x, y, z, r);
            cross3(r, m, tq);
            // the free-body schemes leave the solid flags to the next prep (the
            // lists it applies are those of the displacement made)
            if (p.free_scheme == 0) sb.flags[A] = (uint8_t)((sb.flags[A] & ~FL_SOLID) | (s > 0 ? FL_SOLID : 0));
            part[threadIdx.x][0] = m[0];
            part[threadIdx.x][1] = m[1];
            part[threadIdx.x][2] = m[2];
            part[threadIdx.x][3] = tq[0];
            part[threadIdx.x][4] = tq[1];
            part[threadIdx.x][5] = tq[2];
            sgn[threadIdx.x] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) { // list order = cell order, as in the oracle
            const long long m_ = cnt - base < IMP_THREADS ? cnt - base : IMP_THREADS;
            for (int e2 = 0; e2 < m_; ++e2) {
                if (sgn[e2] > 0)
                    for (int a = 0; a < 6; ++a) acc[a] += part[e2][a];
                else if (sgn[e2] < 0)
                    for (int a = 0; a < 6; ++a) acc[a] -= part[e2][a];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && sb.phase != PH_FIX) {
        double *row = sb.series + ((sb.t % p.series_cap) * p.nb + b) * SERIES_ROW;
        double *to = (sb.phase == PH_IMP && B.free && p.free_scheme == 1) ? sb.imp_prev + 6 * b : row + 6;
        for (int a = 0; a < 6; ++a) to[a] = acc[a];
    }
}


// reduced-precision modes: same terms, FP32 per node, fixed-point block sum
template <class L, class P>
__device__ __forceinline__ void imp_body_fast(const Params &p, const StepBufs &sb, int b) {
    using S = typename P::S;
    __shared__ unsigned long long acc_s[6];
    if (threadIdx.x < 6) acc_s[threadIdx.x] = 0ull;
    __syncthreads();
    const BodyDev &B = sb.bodies[b];
    const long long cnt = sb.apm_cnt[b];
    const S *src = (const S *)sb.src;
    S *dst = (S *)sb.dst;
    const double *X = sb.poses + (long long)b * POSE_STRIDE + 3;  // wrapped pose at t
    const double *X1 = sb.poses + (long long)b * POSE_STRIDE + 9; // wrapped pose at t+1
    for (long long e = threadIdx.x; e < cnt; e += IMP_THREADS) {
        const long long A = sb.apm_cell[B.apm_off + e];
        const int s = sb.apm_sign[B.apm_off + e];
        // PH_FIX: only the nodes uncovered now and not by the prediction
        if (sb.phase == PH_FIX && (s > 0 || pred_uncovered(sb, B, b, A))) continue;
        int x, y, z;
        coords_of(p, A, x, y, z);
        float m[3] = {0.f, 0.f, 0.f};
        float f[L::Q];
        if (s > 0) { // covered: the streamed values f_i(A, t+1) (cut links read the
                     // wall values that k_links left in the solid nodes' slots)
            pull_all<L, P>(p, src, (const float *)nullptr, x, y, z, A, f);
            atomicAdd(&sb.counters[1], 1ull);
        } else { // uncovered: refill f(A, t+1) = f^eq(rho_bar, u_B or u_bar)
            double r1[3], uBd[3];
            disp(p, X1, x, y, z, r1);
            body_velocity(B, r1, uBd);
            float sum = 0.f, us[3] = {0.f, 0.f, 0.f};
            int nn = 0;
#pragma unroll
            for (int i = 1; i < L::Q; ++i) {
                int q[3] = {x + L::cx(i), y + L::cy(i), z + L::cz(i)};
                const int n[3] = {p.nx, p.ny, p.nz};
                bool ok = true;
                for (int a = 0; a < 3; ++a) {
                    if (q[a] >= 0 && q[a] < n[a]) continue;
                    if (!p.per[a]) ok = false;
                    else q[a] += q[a] < 0 ? n[a] : -n[a];
                }
                if (!ok) continue;
                const long long nb = cell_of(p, q[0], q[1], q[2]);
                if (sb.owner_t[nb] != 0) continue;
                const float4 m = load_mac((const float *)sb.mac_t, nb); // moments of f(t)
                sum += m.x;
                us[0] += m.y;
                us[1] += m.z;
                us[2] += m.w;
                nn++;
            }
            long long ec[3];
            if (p.refill == 2 && extrap_cells<L>(p, B, X1, sb.owner_t, x, y, z, ec) != 0) {
                for (int i = 0; i < L::Q; ++i) {
                    const S *fi = src + (long long)i * p.N;
                    f[i] = (3.0f * ldP(fi + ec[0]) - 3.0f * ldP(fi + ec[1])) + ldP(fi + ec[2]);
                }
                atomicAdd(&sb.counters[8], 1ull);
            } else {
                const float drb = nn ? sum / (float)nn : 0.0f;
                float uf[3];
                for (int a = 0; a < 3; ++a) uf[a] = (p.refill == 1 && nn) ? us[a] / (float)nn : (float)uBd[a];
                const float usq15 = 1.5f * (uf[0] * uf[0] + uf[1] * uf[1] + uf[2] * uf[2]);
                for (int i = 0; i < L::Q; ++i) f[i] = dfeq_f<L>(p, i, drb, uf, usq15);
            }
            atomicAdd(&sb.counters[2], 1ull);
        }
        for (int i = 0; i < L::Q; ++i) {
            m[0] += (float)L::cx(i) * f[i];
            m[1] += (float)L::cy(i) * f[i];
            m[2] += (float)L::cz(i) * f[i];
        }
        if (s < 0) { // the refilled node starts the next step collided
            float drho, u[3];
            moments_f<L>(p, f, drho, u);
            store_mac((float *)sb.mac_t1, A, drho, u);
            collide_f<L>(p, f, drho, u);
            for (int i = 0; i < L::Q; ++i) stS(dst + (long long)i * p.N + A, f[i]);
        }
        double r[3];
        disp(p, X, x, y, z, r);
        const float r0 = (float)r[0], r1_ = (float)r[1], r2 = (float)r[2];
        const float tq[3] = {r1_ * m[2] - r2 * m[1], r2 * m[0] - r0 * m[2], r0 * m[1] - r1_ * m[0]};
        const float sg = s > 0 ? 1.0f : -1.0f;
        for (int a = 0; a < 3; ++a) {
            atomicAdd(&acc_s[a], to_fx(sg * m[a]));
            atomicAdd(&acc_s[3 + a], to_fx(sg * tq[a]));
        }
    }
    __syncthreads();
    if (threadIdx.x < 6 && sb.phase != PH_FIX) {
        double *row = sb.series + ((sb.t % p.series_cap) * p.nb + b) * SERIES_ROW;
        double *to = (sb.phase == PH_IMP && B.free && p.free_scheme == 1) ? sb.imp_prev + 6 * b : row + 6;
        to[threadIdx.x] = from_fx(acc_s[threadIdx.x]);
    }
}

// per-body sum of the link contributions into the series row of step t
template <bool EXACT> __device__ __forceinline__ void reduce_body(const Params &p, const StepBufs &sb, int b) {
    const BodyDev &B = sb.bodies[b];
    double *row = sb.series + ((sb.t % p.series_cap) * p.nb + b) * SERIES_ROW;
    if (threadIdx.x < ME_PER_LINK) {
        const int k = threadIdx.x;
        double acc = 0.0;
        if constexpr (EXACT) { // sequential in link order (= cell, direction order of the oracle)
            const long long cnt = sb.link_cnt[b];
            const double *mk = sb.me + k * p.me_stride + B.link_off;
            for (long long j = 0; j < cnt; ++j) acc += mk[j];
        } else { // exact fixed-point sums accumulated by k_links; cleared for the next step
            unsigned long long *a = sb.acc + (long long)b * SERIES_ROW + (k < 6 ? k : k + 6);
            acc = from_fx(*a);
            *a = 0ull;
        }
        row[k < 6 ? k : k + 6] = acc;
        if (!isfinite(acc)) atomicOr(&sb.counters[5], 1ull); // FP64 mode: a non-finite force marks the solve unstable
    }
    if (!B.moving && threadIdx.x < 6) row[6 + threadIdx.x] = 0.0;
    // scheme 1: a free body's impulsive terms are those of its previous
    // displacement (known before the body moves)
    if (sb.phase == PH_REDUCE && B.free && p.free_scheme == 1 && threadIdx.x < 6)
        row[6 + threadIdx.x] = sb.imp_prev[6 * b + threadIdx.x];
}

// end of step: blocks [0, nb) reduce the link contributions of one body,
// blocks [nb, nb + moving) handle the covered/uncovered nodes of one moving
// body (they write disjoint parts of the series row)
template <class L, class P> __global__ void __launch_bounds__(IMP_THREADS) k_finish(Params p, StepBufs sb) {
    // the step index from the device (kernels replayed from a graph read it
    // there); the next step's index goes into the other parity's word, which
    // no kernel of this step reads
    sb.t = (long long)sb.counters[9 + sb.par];
    const bool reduce = sb.phase == PH_ALL || sb.phase == PH_REDUCE; // once per step
    if (reduce && blockIdx.x == 0 && threadIdx.x == 0) sb.counters[9 + (sb.par ^ 1)] = (unsigned long long)(sb.t + 1);
    if (!P::exact && reduce && blockIdx.x == 0 && threadIdx.x == 0) {
        sb.counters[4] = sb.counters[3];
        sb.counters[3] = 0ull;
    }
    if ((int)blockIdx.x < p.nb) {
        if (reduce) reduce_body<P::exact>(p, sb, blockIdx.x);
        return;
    }
    if (sb.phase == PH_REDUCE) return;
    if constexpr (P::exact) imp_body_exact<L, P>(p, sb, sb.moving_ids[blockIdx.x - p.nb]);
    else imp_body_fast<L, P>(p, sb, sb.moving_ids[blockIdx.x - p.nb]);
}

} // namespace lbm
