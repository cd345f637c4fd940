// lbm_bnd.cuh -- boundary-node kernel of the reduced-precision modes.
//
// A boundary node is a fluid node with at least one solid neighbour at t:
// the node x_F = x_A + c_i of a cut link (Sec. 2.1).  k_bulk skips these nodes
// (flag FL_BND); this kernel runs on the side stream beside k_bulk and does
// their whole step.  One warp per node, one lane per lattice direction i:
//   lane i pulls fhat_i(x - c_i, t) (Eq. streaming) or, if x - c_i is solid,
//   evaluates the wall value of Eq. Fillipova_interpolation (Delta from the
//   body pose, u_bf and chi of Sec. 2.1, u_G from the moments of fhat at
//   x + c_i) and the link's momentum-exchange terms (Eqs. flow_force_2,
//   flow_torque_2, ForceInMovementMovingFrame, TorqueInMovementMovingFrame),
//   summed exactly in fixed point per body;
// moments are warp reductions; the node is collided and stored.  A node that
// a body covers at t+1 keeps its streamed f(x, t+1) for the impulsive terms
// of k_finish.
//
// Node lists: nodes whose solid neighbours all belong to static bodies are
// listed once; nodes next to a moving body are listed per step by k_fgeom2
// (a node next to several moving bodies is listed by the lowest-numbered one).
#pragma once

#include "lbm_internal.h"
#include "lbm_region.cuh"

namespace lbm {

constexpr int BND_THREADS = 256; // 8 nodes per block

__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// the step of boundary node `cell` (one warp; lane = lattice direction)
template <class L, class P>
__device__ __forceinline__ void bnd_node(const Params &p, const BndArgs &a, const StepBufs &sb, long long cell,
                                         bool from_static, unsigned &nlinks) {
    using S = typename P::S;
    const int lane = threadIdx.x & 31;
    const bool act = lane < L::Q;
    const int i = act ? lane : 0; // lattice direction of this lane
    const int cxi = L::cx(i), cyi = L::cy(i), czi = L::cz(i);
    const int ib = L::opp(i);
    const float wi = L::template w<float>(i);
    const S *src = (const S *)sb.src;
    S *dst = (S *)sb.dst;
    const long long N = p.N;
    int x, y, z;
    coords_of(p, cell, x, y, z);
    const long long sc = i == 0 ? cell : nbr<L>(p, x, y, z, i, 1);      // pull source x - c_i
    const long long G = act && i > 0 ? nbr<L>(p, x, y, z, ib, 1) : -1; // x + c_i
    // every load that depends on the node alone is issued here, together:
    // the owners at t (node, pull sources, x + c_i) and t+1, fhat(x, t) and
    // the pulled fhat_i(x - c_i, t) (not used where x - c_i is solid)
    const uint16_t own = a.owner_t[cell], own1 = a.owner_t1[cell];
    const uint16_t o = (act && i > 0 && sc >= 0) ? a.owner_t[sc] : (uint16_t)0;
    const uint16_t oG = G >= 0 ? a.owner_t[G] : (uint16_t)1;
    const float fo = act ? ldP(src + (long long)i * N + cell) : 0.0f;
    const float fp = (act && sc >= 0) ? ldS(src + (long long)i * N + sc) : 0.0f;
    if (own != 0) return; // warp-uniform
    if (from_static) { // a moving body next to it: that body's list has it
        const bool mv = o != 0 && a.bodies[o - 1].moving;
        if (__any_sync(0xffffffffu, mv)) return;
    }
    const unsigned cutmask = __ballot_sync(0xffffffffu, o != 0);
    if (!cutmask) return;
    // moments of the collided populations fhat(x, t) (= those of f(x, t))
    const float drF = warp_sum(fo);
    float uF[3];
    {
        float j0 = warp_sum(cxi * fo), j1 = warp_sum(cyi * fo), j2 = warp_sum(czi * fo);
        if (p.has_force) {
            j0 -= 0.5f * p.gf[0];
            j1 -= 0.5f * p.gf[1];
            j2 -= 0.5f * p.gf[2];
        }
        const float inv = 1.0f / (p.eq == 0 ? p.rho0f : 1.0f + drF);
        uF[0] = j0 * inv;
        uF[1] = j1 * inv;
        uF[2] = j2 * inv;
        // stability check at the boundary nodes: a NaN or |u| > 0.3 marks the
        // solve unstable (counters[5]; the host reports LBM_ERR_UNSTABLE)
        const float usq = uF[0] * uF[0] + uF[1] * uF[1] + uF[2] * uF[2];
        if (lane == 0 && !(usq < 0.09f)) atomicOr(&sb.counters[5], 1ull);
    }
    const float fb = __shfl_sync(0xffffffffu, fo, ib); // fhat_ib(x, t)
    float fi = 0.0f;
    float v[ME_PER_LINK];
#pragma unroll
    for (int c = 0; c < ME_PER_LINK; ++c) v[c] = 0.0f;
    const int bi = (int)o - 1;
    if (o) {
        const BodyDev &Bi = a.bodies[bi];
        const double *Pf = a.poses + (long long)bi * POSE_STRIDE + 12; // floor, frac of the pose at t
        float d[3];
        const int c3[3] = {x, y, z};
        for (int q = 0; q < 3; ++q) d[q] = frame_axis(c3[q] - (int)Pf[q], (float)Pf[3 + q], axis_len(p, q), p.per[q]);
        const double *Po = a.poses + (long long)bi * POSE_STRIDE + 18; // orientation at t
        const float dl = link_delta_f(Bi.halfway, Bi.shape, (float)Bi.R, (float)Bi.R2, (float)Po[0], (float)Po[1],
                                      d, cxi, cyi, czi);
        const float rb[3] = {d[0] - dl * cxi, d[1] - dl * cyi, d[2] - dl * czi};
        const float W0 = (float)Bi.W[0], W1 = (float)Bi.W[1], W2 = (float)Bi.W[2];
        const float uB[3] = {(float)Bi.U[0] + (W1 * rb[2] - W2 * rb[1]),
                             (float)Bi.U[1] + (W2 * rb[0] - W0 * rb[2]),
                             (float)Bi.U[2] + (W0 * rb[1] - W1 * rb[0])};
        float ubf[3], chi;
        if (dl < 0.5f) {
            // u_bf = u_G = u(x_F + c_i, t), chi = (2 Delta - 1)/(tau - 2)
            if (G >= 0 && oG == 0) { // x + c_i fluid at t
                float drG;
                moments_hat<L>(p, src, G, drG, ubf);
                chi = (2.0f * dl - 1.0f) / ((float)p.tau - 2.0f);
            } else {
                ubf[0] = uF[0];
                ubf[1] = uF[1];
                ubf[2] = uF[2];
                chi = 0.0f;
                atomicAdd(&sb.counters[0], 1ull);
            }
        } else {
            // u_bf = u_F + 3/(2 Delta) (u_B - u_F), chi = (2 Delta - 1)/(tau + 1/2)
            const float k3 = 3.0f / (2.0f * dl);
            for (int q = 0; q < 3; ++q) ubf[q] = fmaf(k3, uB[q] - uF[q], uF[q]);
            chi = (2.0f * dl - 1.0f) / ((float)p.tau + 0.5f);
        }
        // fictitious equilibrium g_ib (Eq. Fillipova_equilibrium), deviation form
        const float cbu = -(cxi * ubf[0] + cyi * ubf[1] + czi * ubf[2]);
        const float cbF = -(cxi * uF[0] + cyi * uF[1] + czi * uF[2]);
        const float uFsq = uF[0] * uF[0] + uF[1] * uF[1] + uF[2] * uF[2];
        const float rr = p.eq == 0 ? p.rho0f : 1.0f + drF;
        const float gq = wi * fmaf(rr, 3.0f * cbu + 4.5f * cbF * cbF - 1.5f * uFsq, drF);
        const float cuB = cxi * uB[0] + cyi * uB[1] + czi * uB[2];
        fi = fmaf(6.0f * wi * rr, cuB, fmaf(chi, gq - fb, fb));
        // momentum exchange of this link (deviation form: the -2 w_i c_i
        // parts cancel over the body's closed link set)
        const float sum = fi + fb, dif = fi - fb;
        const float s0 = -cxi * sum, s1 = -cyi * sum, s2 = -czi * sum;
        const float m0 = fmaf(uB[0], dif, s0), m1 = fmaf(uB[1], dif, s1), m2 = fmaf(uB[2], dif, s2);
        v[0] = s0;
        v[1] = s1;
        v[2] = s2;
        v[3] = d[1] * s2 - d[2] * s1;
        v[4] = d[2] * s0 - d[0] * s2;
        v[5] = d[0] * s1 - d[1] * s0;
        v[6] = m0;
        v[7] = m1;
        v[8] = m2;
        v[9] = d[1] * m2 - d[2] * m1;
        v[10] = d[2] * m0 - d[0] * m2;
        v[11] = d[0] * m1 - d[1] * m0;
    } else if (act) {
        fi = sc >= 0 ? fp : pull_edge<L, P>(p, src, (const float *)nullptr, x, y, z, cell, i);
    }
    // collision (or the streamed values of a node covered at t+1)
    float out = fi;
    if (own1 == 0) {
        const float dr = warp_sum(fi);
        float j0 = warp_sum(cxi * fi), j1 = warp_sum(cyi * fi), j2 = warp_sum(czi * fi);
        if (p.has_force) {
            j0 = fmaf(0.5f, p.gf[0], j0);
            j1 = fmaf(0.5f, p.gf[1], j1);
            j2 = fmaf(0.5f, p.gf[2], j2);
        }
        const float inv = 1.0f / (p.eq == 0 ? p.rho0f : 1.0f + dr);
        const float u[3] = {j0 * inv, j1 * inv, j2 * inv};
        const float usq15 = 1.5f * fmaf(u[0], u[0], fmaf(u[1], u[1], u[2] * u[2]));
        const float cu = cxi * u[0] + cyi * u[1] + czi * u[2];
        const float rr = p.eq == 0 ? p.rho0f : 1.0f + dr;
        const float fe = wi * fmaf(rr, fmaf(cu, fmaf(4.5f, cu, 3.0f), -usq15), dr);
        const float om = p.omegaf;
        out = fmaf(-om, fi - fe, fi);
        if (p.has_force) {
            const float cg = cxi * p.gf[0] + cyi * p.gf[1] + czi * p.gf[2];
            const float ug = u[0] * p.gf[0] + u[1] * p.gf[1] + u[2] * p.gf[2];
            out = fmaf((1.0f - 0.5f * om) * wi, fmaf(9.0f * cu, cg, 3.0f * (cg - ug)), out);
        }
    }
    if (act) stS(dst + (long long)i * N + cell, out);
    // per-body fixed-point sums: one atomic per component when all the
    // node's cut links belong to one body (the usual case)
    nlinks += __popc(cutmask);
    const int b0 = __shfl_sync(0xffffffffu, bi, __ffs(cutmask) - 1);
    const bool one_body = __all_sync(0xffffffffu, o == 0 || bi == b0);
    if (one_body) {
        // lane c (< 12) gathers component c of every cut link's lane and
        // sums it in fixed point: as many rounds as cut links
        unsigned long long *acc = sb.acc + (long long)b0 * SERIES_ROW;
        const int myc = lane < ME_PER_LINK ? lane : 0;
        unsigned long long tot = 0ull;
        unsigned m = cutmask;
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            float mine = 0.0f;
#pragma unroll
            for (int c = 0; c < ME_PER_LINK; ++c) {
                const float vc = __shfl_sync(0xffffffffu, v[c], j);
                if (c == myc) mine = vc;
            }
            tot += to_fx(mine);
        }
        if (lane < ME_PER_LINK && tot) atomicAdd(acc + (lane < 6 ? lane : lane + 6), tot);
    } else if (o) {
        unsigned long long *acc = sb.acc + (long long)bi * SERIES_ROW;
        for (int c = 0; c < ME_PER_LINK; ++c) atomicAdd(acc + (c < 6 ? c : c + 6), to_fx(v[c]));
    }
}

template <class L, class P>
__global__ void __launch_bounds__(BND_THREADS) k_bnd(Params p, BndArgs a, StepBufs sb) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long ns = (long long)min((unsigned long long)a.static_cap, *a.static_cnt);
    const long long nm = (long long)min((unsigned long long)a.mov_cap, *a.mov_cnt);
    unsigned nlinks = 0;
    for (long long k = warp; k < ns + nm; k += nwarps) {
        const bool from_static = k < ns;
        const long long cell = from_static ? a.static_cells[k] : a.mov_cells[k - ns];
        bnd_node<L, P>(p, a, sb, cell, from_static, nlinks);
    }
    if (lane == 0 && nlinks) atomicAdd(&sb.counters[3], (unsigned long long)nlinks);
}

template <class L, class P>
cudaError_t bnd_t(const Params &p, const BndArgs &a, const StepBufs &sb, int grid, cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    k_bnd<L, P><<<grid, BND_THREADS, 0, s>>>(p, a, sb);
    return cudaGetLastError();
}

} // namespace lbm
