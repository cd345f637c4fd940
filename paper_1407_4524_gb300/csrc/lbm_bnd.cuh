// lbm_bnd.cuh -- boundary-node kernel of the reduced-precision modes.
//
// A boundary node is a fluid node with at least one solid neighbour at t:
// node x_F = x_A + c_i of a cut link (Sec. 2.1).  k_bulk skips these nodes
// (flag FL_BND); this kernel, which runs on the side stream beside k_bulk,
// does their whole step: for every direction it either pulls fhat_i(x - c_i,
// t) (Eq. streaming) or, on a cut link, evaluates the wall value of Eq.
// Fillipova_interpolation (Delta from the body pose, u_bf / chi of Sec. 2.1);
// it adds the link's momentum-exchange terms (Eqs. flow_force_2,
// flow_torque_2 and the moving-frame Eqs. ForceInMovementMovingFrame /
// TorqueInMovementMovingFrame) to exact fixed-point per-body sums; then it
// collides and stores fhat(x, t+1).  A node covered by a body at t+1 keeps
// its streamed f(x, t+1) instead (read by the impulsive terms of k_finish).
//
// Nodes are found by scanning the shell R - 1/2 .. R + 3/2 around each body
// (boundary nodes lie within R + sqrt(2)); a node next to several bodies is
// handled in the scan of the lowest-numbered one.
#pragma once

#include "lbm_internal.h"
#include "lbm_region.cuh"

namespace lbm {

template <class L, class P>
__global__ void __launch_bounds__(GEOM_THREADS) k_bnd(Params p, GeomArgs g, StepBufs sb) {
    using S = typename P::S;
    const int2 cm = g.chunk_map[blockIdx.x];
    const int b = cm.x;
    const BodyDev &B = g.bodies[b];
    const double *P0 = g.poses + (long long)b * POSE_STRIDE;
    __shared__ Frame F;
    __shared__ LatTab tb;
    if (threadIdx.x == 0) {
        make_frame(P0 + 3, F);
        tb = make_tab<L>();
    }
    __syncthreads();
    int lo[3];
    region_lo(p, B, P0, REGION_MARGIN, lo);
    const S *src = (const S *)sb.src;
    S *dst = (S *)sb.dst;
    const long long N = p.N;
    const uint16_t me = (uint16_t)(b + 1);
    const float R = (float)B.R;
    unsigned nlinks = 0;
    unsigned long long accb[ME_PER_LINK]; // exact fixed-point sums of this thread's links
#pragma unroll
    for (int c = 0; c < ME_PER_LINK; ++c) accb[c] = 0ull;

    for (int j = 0; j < GEOM_CELLS; ++j) {
        RegionCell rc = region_cell(p, B, lo, cm.y, j);
        if (!rc.valid) continue;
        const float dist = frame_dist(p, B, F, rc);
        if (dist < R - 0.5f || dist > R + 1.5f) continue;
        const long long cell = rc.cell;
        if (g.owner_t[cell] != 0) continue;
        const int x = rc.x, y = rc.y, z = rc.z;
        // sources x - c_i: owners and cell indices (bodies never touch
        // non-periodic faces, so sources wrap periodically)
        uint16_t ob[L::Q];
        long long sc[L::Q];
        unsigned cut = 0;
        int minb = 1 << 20;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            sc[i] = i == 0 ? cell : nbr<L>(p, x, y, z, i, 1);
            ob[i] = (i > 0 && sc[i] >= 0) ? g.owner_t[sc[i]] : (uint16_t)0;
            if (ob[i]) {
                cut |= 1u << i;
                minb = min(minb, (int)ob[i]);
            }
        }
        if (!cut || minb != me) continue;
        nlinks += __popc(cut);
        // own collided populations fhat(x, t): moments rho_F, u_F and fhat_ib
        float fo[L::Q];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) fo[i] = ldP(src + (long long)i * N + cell);
        float drF, uF[3];
        {
            float r = 0.f, j0 = 0.f, j1 = 0.f, j2 = 0.f;
            if (p.has_force) {
                j0 = -0.5f * p.gf[0];
                j1 = -0.5f * p.gf[1];
                j2 = -0.5f * p.gf[2];
            }
#pragma unroll
            for (int i = 0; i < L::Q; ++i) {
                r += fo[i];
                j0 += (float)L::cx(i) * fo[i];
                j1 += (float)L::cy(i) * fo[i];
                j2 += (float)L::cz(i) * fo[i];
            }
            const float inv = 1.0f / (p.eq == 0 ? p.rho0f : 1.0f + r);
            drF = r;
            uF[0] = j0 * inv;
            uF[1] = j1 * inv;
            uF[2] = j2 * inv;
        }
        float f[L::Q];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            if (!(cut & (1u << i))) {
                f[i] = sc[i] >= 0 ? ldS(src + (long long)i * N + sc[i])
                                  : pull_edge<L, P>(p, src, (const float *)nullptr, x, y, z, cell, i);
                continue;
            }
            const int bi = ob[i] - 1;
            const BodyDev &Bi = g.bodies[bi];
            Frame Fo;
            const Frame *Fi = &F;
            if (bi != b) {
                make_frame(g.poses + (long long)bi * POSE_STRIDE + 3, Fo);
                Fi = &Fo;
            }
            float d[3];
            frame_disp_f(p, *Fi, x, y, z, d);
            const int cxi = L::cx(i), cyi = L::cy(i), czi = L::cz(i);
            const int ib = L::opp(i);
            const float dl = link_delta_f(Bi, d, cxi, cyi, czi);
            const float rb[3] = {d[0] - dl * cxi, d[1] - dl * cyi, d[2] - dl * czi};
            const float W0 = (float)Bi.W[0], W1 = (float)Bi.W[1], W2 = (float)Bi.W[2];
            const float uB[3] = {(float)Bi.U[0] + (W1 * rb[2] - W2 * rb[1]),
                                 (float)Bi.U[1] + (W2 * rb[0] - W0 * rb[2]),
                                 (float)Bi.U[2] + (W0 * rb[1] - W1 * rb[0])};
            float ubf[3], chi;
            if (dl < 0.5f) {
                // u_bf = u_G = u(x_F + c_i, t), chi = (2 Delta - 1)/(tau - 2)
                const long long G = nbr<L>(p, x, y, z, ib, 1); // x - c_ib = x + c_i
                if (G >= 0 && g.owner_t[G] == 0) {
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
                for (int a = 0; a < 3; ++a) ubf[a] = fmaf(k3, uB[a] - uF[a], uF[a]);
                chi = (2.0f * dl - 1.0f) / ((float)p.tau + 0.5f);
            }
            const float fb = fo[ib];
            const float gq = dgeq_f(p, tb, ib, drF, ubf, uF);
            const float rhow = p.eq == 0 ? p.rho0f : 1.0f + drF;
            const float cuB = cxi * uB[0] + cyi * uB[1] + czi * uB[2];
            const float fa = fmaf(6.0f * L::template w<float>(i) * rhow, cuB, fmaf(chi, gq - fb, fb));
            f[i] = fa;
            // momentum exchange of this link (deviation form: the -2 w_i c_i
            // parts cancel over the body's closed link set)
            const float sum = fa + fb, dif = fa - fb;
            const float s0 = -cxi * sum, s1 = -cyi * sum, s2 = -czi * sum;
            const float m0 = fmaf(uB[0], dif, s0), m1 = fmaf(uB[1], dif, s1), m2 = fmaf(uB[2], dif, s2);
            const float v[ME_PER_LINK] = {s0, s1, s2, d[1] * s2 - d[2] * s1, d[2] * s0 - d[0] * s2,
                                          d[0] * s1 - d[1] * s0, m0, m1, m2, d[1] * m2 - d[2] * m1,
                                          d[2] * m0 - d[0] * m2, d[0] * m1 - d[1] * m0};
            if (bi == b) {
#pragma unroll
                for (int c = 0; c < ME_PER_LINK; ++c) accb[c] += to_fx(v[c]);
            } else {
                unsigned long long *ao = sb.acc + (long long)bi * SERIES_ROW;
                for (int c = 0; c < ME_PER_LINK; ++c) atomicAdd(ao + (c < 6 ? c : c + 6), to_fx(v[c]));
            }
        }
        if (g.owner_t1[cell] != 0) {
            // covered at t+1: keep the streamed values for the impulsive terms
#pragma unroll
            for (int i = 0; i < L::Q; ++i) stS(dst + (long long)i * N + cell, f[i]);
        } else {
            float drho, u[3];
            moments_f<L>(p, f, drho, u);
            collide_f<L>(p, f, drho, u);
#pragma unroll
            for (int i = 0; i < L::Q; ++i) stS(dst + (long long)i * N + cell, f[i]);
        }
    }
    // warp sums in exact fixed point, one atomic per warp and component
    const int lane = threadIdx.x & 31;
    for (int o = 16; o > 0; o >>= 1) nlinks += __shfl_down_sync(0xffffffffu, nlinks, o);
    if (lane == 0 && nlinks) atomicAdd(&sb.counters[3], (unsigned long long)nlinks);
    unsigned long long *acc = sb.acc + (long long)b * SERIES_ROW;
#pragma unroll
    for (int c = 0; c < ME_PER_LINK; ++c) {
        unsigned long long v = accb[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0 && v) atomicAdd(acc + (c < 6 ? c : c + 6), v);
    }
}

template <class L, class P>
cudaError_t bnd_t(const Params &p, const GeomArgs &g, const StepBufs &sb, cudaStream_t s) {
    if (g.nchunks == 0) return cudaSuccess;
    k_bnd<L, P><<<g.nchunks, GEOM_THREADS, 0, s>>>(p, g, sb);
    return cudaGetLastError();
}

} // namespace lbm
