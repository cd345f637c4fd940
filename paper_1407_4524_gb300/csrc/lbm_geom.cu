// lbm_geom.cu -- body geometry on the device (FP64, identical in every
// precision mode): solid owner of each node, covered / uncovered node lists
// A+ / A- between t and t+1 (Sec. 3.2.2), node flags, and the cut-link lists
// (fluid node x_F, direction i with x_F - c_i inside the body, fractional
// distance Delta of Sec. 2.1).
//
// Work is split into chunks of GEOM_THREADS consecutive cells of each body's
// region (a box covering the body at t and t+1 plus a margin), enumerated in
// ascending cell order even across periodic seams.  Lists are compacted with
// block scans and per-chunk offsets, so every list is in cell order (then
// direction order) whatever the launch configuration: the FP64 mode can then
// sum link contributions in exactly the oracle's order.
#include "lbm_internal.h"
#include "lbm_region.cuh"

namespace lbm {

namespace {

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
    for (int o = 1; o < 32; o <<= 1) {
        int n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// exclusive block scan of v over GEOM_THREADS threads; *total gets the sum
__device__ __forceinline__ int block_excl_scan(int v, int *total) {
    __shared__ int wsum[GEOM_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int s = lane < GEOM_THREADS / 32 ? wsum[lane] : 0;
        s = warp_incl_scan(s);
        if (lane < GEOM_THREADS / 32) wsum[lane] = s;
    }
    __syncthreads();
    int base = wid ? wsum[wid - 1] : 0;
    *total = wsum[GEOM_THREADS / 32 - 1];
    __syncthreads();
    return base + inc - v;
}

// sum of the counts of the chunks [first, first + n) (block-wide)
__device__ __forceinline__ long long block_sum_range(const int *cnt, int first, int n) {
    __shared__ long long red[GEOM_THREADS];
    long long s = 0;
    for (int k = threadIdx.x; k < n; k += GEOM_THREADS) s += cnt[first + k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = GEOM_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    long long r = red[0];
    __syncthreads();
    return r;
}

template <class L>
__device__ __forceinline__ uint8_t node_flags(const Params &p, const uint16_t *owner_t, const uint16_t *owner_m,
                                              int x, int y, int z, long long cell) {
    const uint8_t f = owner_t[cell] ? FL_SOLID : 0;
    if (owner_m[cell]) return f;
    // all neighbour loads are independent (no early exit), so they overlap
    unsigned one = 0, two = 0;
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        const long long a = nbr<L>(p, x, y, z, i, 1);
        const long long b = nbr<L>(p, x, y, z, i, 2);
        one |= (a >= 0 ? owner_m[a] : 0u);
        two |= (b >= 0 ? owner_m[b] : 0u);
    }
    uint8_t r = f;
    if (one | two || edge_node(p, x, y, z)) r |= FL_MAC;
    if (one && !owner_t[cell]) r |= FL_BND;
    return r;
}

// exclusive prefix over bodies of v(b) = link_cnt[b] (tiles = 0) or of the
// number of LINK_THREADS-link tiles of each body (tiles = 1); one block of
// 1024 threads, out has nb + 1 entries
__device__ void prefix_over_bodies(const Params &p, const long long *link_cnt, long long *out, int tiles) {
    __shared__ long long ws[32];
    __shared__ long long carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < p.nb; base += 1024) {
        const int b = base + threadIdx.x;
        long long v = b < p.nb ? link_cnt[b] : 0;
        if (tiles) v = (v + LINK_THREADS - 1) / LINK_THREADS;
        long long inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            long long n = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += n;
        }
        if (lane == 31) ws[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            long long s = ws[lane];
            for (int o = 1; o < 32; o <<= 1) {
                long long n = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += n;
            }
            ws[lane] = s;
        }
        __syncthreads();
        const long long before = carry + (wid ? ws[wid - 1] : 0);
        if (b < p.nb) out[b] = before + inc - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += ws[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[p.nb] = carry;
    __syncthreads();
}

// wrapped poses at t and t+1, prefixes of link counts and link tiles, and
// the solid flags of the nodes that the previous step covered (A+) or
// uncovered (A-), so that the flags describe the solid set of step t
__global__ void __launch_bounds__(1024) k_prep(Params p, const BodyDev *bodies, const long long *link_cnt,
                                               long long *link_pre, long long *tile_pre, double *poses, long long t_arg,
                                               const unsigned long long *tdev, uint8_t *flags,
                                               const long long *apm_cnt, const uint32_t *apm_cell,
                                               const int8_t *apm_sign) {
    const long long t = tdev ? (long long)*tdev : t_arg; // the device step counter, when given
    if (flags) {
        for (int b = 0; b < p.nb; ++b) {
            const BodyDev &B = bodies[b];
            const long long n = apm_cnt[b];
            for (long long e = threadIdx.x; e < n; e += 1024) {
                const long long c = apm_cell[B.apm_off + e];
                flags[c] = (uint8_t)((flags[c] & ~FL_SOLID) | (apm_sign[B.apm_off + e] > 0 ? FL_SOLID : 0));
            }
        }
        __syncthreads();
    }
    prefix_over_bodies(p, link_cnt, link_pre, 0);
    prefix_over_bodies(p, link_cnt, tile_pre, 1);
    for (int b = threadIdx.x; b < p.nb; b += 1024) {
        double *P = poses + (long long)b * POSE_STRIDE;
        pose(bodies[b], t, P);
        wrap_pose(p, P, P + 3);
        pose(bodies[b], t + 1, P + 6);
        wrap_pose(p, P + 6, P + 9);
        if (bodies[b].shape == 2) {
            sincos_cw(orient(bodies[b], t), P[19], P[18]);
            sincos_cw(orient(bodies[b], t + 1), P[25], P[24]);
        } else {
            P[18] = P[24] = 1.0;
            P[19] = P[25] = 0.0;
        }
        for (int a = 0; a < 3; ++a) {
            P[12 + a] = floor(P[3 + a]);
            P[15 + a] = P[3 + a] - P[12 + a];
        }
    }
}

__global__ void __launch_bounds__(GEOM_THREADS) k_raster(Params p, GeomArgs g, uint16_t *owner, long long) {
    const int2 cm = g.chunk_map[blockIdx.x];
    const BodyDev &B = g.bodies[cm.x];
    const double *P = g.poses + (long long)cm.x * POSE_STRIDE;
    __shared__ Frame F;
    if (threadIdx.x == 0) make_frame(P + 3, F);
    __syncthreads();
    int lo[3];
    region_lo(p, B, P, REGION_MARGIN, lo);
    for (int j = 0; j < GEOM_CELLS; ++j) {
        RegionCell rc = region_cell(p, B, lo, cm.y, j);
        if (rc.valid && inside_screened(p, B, F, rc.x, rc.y, rc.z)) owner[rc.cell] = (uint16_t)(cm.x + 1);
    }
}

// moving step, part a: owner at t+1 for this body's region; count A+/A-.
// Only the shell R-2 <= |x - X(t+1)| <= R+2 can change owner (the surface
// moves less than half a cell per step).
__global__ void __launch_bounds__(GEOM_THREADS) k_geom_a(Params p, GeomArgs g) {
    const int2 cm = g.chunk_map[blockIdx.x];
    const int b = cm.x;
    const BodyDev &B = g.bodies[b];
    const double *P = g.poses + (long long)b * POSE_STRIDE;
    __shared__ Frame F;
    if (threadIdx.x == 0) make_frame(P + 9, F);
    __syncthreads();
    int lo[3];
    region_lo(p, B, P, REGION_MARGIN, lo);
    const uint16_t me = (uint16_t)(b + 1);
    const float Rin = body_rin(B), Rout = body_rout(B);
    int flags = 0;
    for (int j = 0; j < GEOM_CELLS; ++j) {
        RegionCell rc = region_cell(p, B, lo, cm.y, j);
        if (!rc.valid) continue;
        const float dist = frame_dist(p, B, F, rc);
        if (dist < Rin - 2.0f || dist > Rout + 2.0f) continue;
        const bool in_t = g.owner_t[rc.cell] == me;
        const bool in1 = inside_screened(p, B, F, rc.x, rc.y, rc.z);
        if (in1) g.owner_t1[rc.cell] = me;
        else if (in_t || g.owner_t1[rc.cell] == me) g.owner_t1[rc.cell] = 0;
        flags += in_t != in1;
    }
    int total;
    block_excl_scan(flags, &total);
    if (threadIdx.x == 0) g.chunk_cnt_apm[blockIdx.x] = total;
}

// part b: A+/A- lists (moving step), node flags (FP64 mode), link counts
template <class L>
__global__ void __launch_bounds__(GEOM_THREADS) k_geom_b(Params p, GeomArgs g) {
    const int2 cm = g.chunk_map[blockIdx.x];
    const int b = cm.x;
    const BodyDev &B = g.bodies[b];
    const uint16_t me = (uint16_t)(b + 1);
    const uint16_t *owner_L = g.owner_t1; // geometry of the links being built
    const double *P = g.poses + (long long)b * POSE_STRIDE;
    const double *XL = P + (g.t_link == g.t ? 3 : 9);
    __shared__ Frame F;
    if (threadIdx.x == 0) make_frame(XL, F);
    __syncthreads();
    int lo[3];
    region_lo(p, B, P, REGION_MARGIN, lo);
    const int first = blockIdx.x - cm.y; // first chunk of this body
    const float Rin = body_rin(B), Rout = body_rout(B);
    unsigned apm_mask = 0, apm_sign = 0;
    int nl = 0;
    for (int j = 0; j < GEOM_CELLS; ++j) {
        RegionCell rc = region_cell(p, B, lo, cm.y, j);
        if (!rc.valid) continue;
        const float dist = frame_dist(p, B, F, rc);
        if (g.do_apm && dist >= Rin - 2.0f && dist <= Rout + 2.0f) {
            const bool in_t = g.owner_t[rc.cell] == me, in1 = g.owner_t1[rc.cell] == me;
            if (in_t != in1) {
                apm_mask |= 1u << j;
                if (in1) apm_sign |= 1u << j;
            }
        }
        // node flags (FP64 mode: the moment-store flag follows the geometry of t+1;
        // under the semi-implicit schemes a free body's pose of t+1 is known only
        // after the step's force, so its moments are kept on the band within
        // R + MAC_BAND of the pose the flags are built from, which holds the
        // nodes within two links of the body at t+1 and t+2 whatever the update)
        if (g.do_flags && dist >= Rin - 2.0f && dist <= Rout + 5.5f) {
            uint8_t nf = node_flags<L>(p, g.owner_t, owner_L, rc.x, rc.y, rc.z, rc.cell);
            if (p.free_scheme && B.free && dist <= Rout + MAC_BAND) nf |= FL_MAC;
            g.flags[rc.cell] = nf;
        }
        if (dist >= Rin - 0.5f && dist <= Rout + 2.0f && owner_L[rc.cell] == 0) {
#pragma unroll
            for (int i = 1; i < L::Q; ++i) {
                const long long a = nbr<L>(p, rc.x, rc.y, rc.z, i, 1);
                nl += (a >= 0 ? owner_L[a] : (uint16_t)0) == me;
            }
        }
    }
    if (g.do_apm) {
        const long long before = block_sum_range(g.chunk_cnt_apm, first, cm.y);
        int total;
        long long at = before + block_excl_scan(__popc(apm_mask), &total);
        for (int j = 0; j < GEOM_CELLS; ++j) {
            if (!(apm_mask & (1u << j))) continue;
            if (at < B.apm_cap) {
                RegionCell rc = region_cell(p, B, lo, cm.y, j);
                g.apm_cell[B.apm_off + at] = (uint32_t)rc.cell;
                g.apm_sign[B.apm_off + at] = (int8_t)((apm_sign & (1u << j)) ? 1 : -1);
            }
            at++;
        }
        if (cm.y == B.nchunks - 1 && threadIdx.x == 0) {
            long long n = before + total;
            g.apm_cnt[b] = n < B.apm_cap ? n : B.apm_cap;
        }
    }
    int total;
    block_excl_scan(nl, &total);
    if (threadIdx.x == 0) g.chunk_cnt_link[blockIdx.x] = total;
}

// part c: fill the cut-link list of the body (cell order, then direction)
template <class L>
__global__ void __launch_bounds__(GEOM_THREADS) k_geom_c(Params p, GeomArgs g) {
    const int2 cm = g.chunk_map[blockIdx.x];
    const int b = cm.x;
    const BodyDev &B = g.bodies[b];
    const uint16_t me = (uint16_t)(b + 1);
    const uint16_t *owner_L = g.owner_t1;
    const double *P = g.poses + (long long)b * POSE_STRIDE;
    const double *XL = P + (g.t_link == g.t ? 3 : 9);
    __shared__ Frame F;
    if (threadIdx.x == 0) make_frame(XL, F);
    __syncthreads();
    int lo[3];
    region_lo(p, B, P, REGION_MARGIN, lo);
    const int first = blockIdx.x - cm.y;
    const float Rin = body_rin(B), Rout = body_rout(B);
    unsigned mask[GEOM_CELLS];
    int nl = 0;
#pragma unroll
    for (int j = 0; j < GEOM_CELLS; ++j) {
        mask[j] = 0;
        RegionCell rc = region_cell(p, B, lo, cm.y, j);
        if (!rc.valid) continue;
        const float dist = frame_dist(p, B, F, rc);
        if (dist >= Rin - 0.5f && dist <= Rout + 2.0f && owner_L[rc.cell] == 0) {
#pragma unroll
            for (int i = 1; i < L::Q; ++i) {
                const long long a = nbr<L>(p, rc.x, rc.y, rc.z, i, 1);
                if ((a >= 0 ? owner_L[a] : (uint16_t)0) == me) mask[j] |= 1u << i;
            }
            nl += __popc(mask[j]);
        }
    }
    const long long before = block_sum_range(g.chunk_cnt_link, first, cm.y);
    int total;
    long long at = before + block_excl_scan(nl, &total);
#pragma unroll
    for (int j = 0; j < GEOM_CELLS; ++j) {
        if (!mask[j]) continue;
        RegionCell rc = region_cell(p, B, lo, cm.y, j);
        double d[3];
        float df[3];
        if (p.exact) disp(p, XL, rc.x, rc.y, rc.z, d);
        else frame_disp_f(p, F, rc.x, rc.y, rc.z, df);
        for (int i = 1; i < L::Q; ++i) {
            if (!(mask[j] & (1u << i))) continue;
            if (at < B.link_cap) {
                const long long jj = B.link_off + at;
                g.Lcell[jj] = (uint32_t)rc.cell;
                g.Ldir[jj] = (uint8_t)i;
                g.Ldelta[jj] = p.exact ? link_delta(B, d, L::cx(i), L::cy(i), L::cz(i), F.co, F.si)
                                       : (double)link_delta_f(B.halfway, B.shape, (float)B.R, (float)B.R2, F.cof,
                                                              F.sif, df, L::cx(i), L::cy(i), L::cz(i));
            }
            at++;
        }
    }
    if (cm.y == B.nchunks - 1 && threadIdx.x == 0) {
        long long n = before + total;
        g.link_cnt[b] = n < B.link_cap ? n : B.link_cap;
    }
}

template <class L>
__global__ void k_flags_full(Params p, const uint16_t *owner, uint8_t *flags) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= p.nx) return;
    const long long cell = cell_of(p, x, y, z);
    flags[cell] = node_flags<L>(p, owner, owner, x, y, z, cell);
}

template <class L, class P>
__global__ void k_export(Params p, const typename P::S *pop, double *out) {
    const long long n = (long long)L::Q * p.N;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k / p.N);
        double v = (double)ldP(pop + k);
        if constexpr (!P::exact) v += L::template w<double>(i);
        out[k] = v;
    }
}

template <class L, class P>
__global__ void k_import(Params p, const double *in, typename P::S *pop) {
    const long long n = (long long)L::Q * p.N;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k / p.N);
        double v = in[k];
        if constexpr (!P::exact) v -= L::template w<double>(i);
        stS(pop + k, (typename P::C)v);
    }
}


// ----------------------------------------------------------------------------
// Reduced-precision modes.  Momentum-exchange sums are order independent
// there (exact fixed point), so lists are appended with atomics.

// Three independent parts, one block each, so that their memory latencies
// overlap instead of adding up: block 0 the link tiles of t (and the empty
// lists of t+1), block 1 the solid flags of t+1 queued by the previous step's
// geometry, block 2 the poses of t and t+1.
__global__ void __launch_bounds__(1024) k_fprep(Params p, const BodyDev *bodies, double *poses, long long t_arg,
                                                const unsigned long long *tdev, uint8_t *flags,
                                                unsigned long long *chg_cnt, const uint32_t *chg_cell,
                                                const uint8_t *chg_val, long long chg_cap, long long *apm_cnt,
                                                unsigned long long *bn_mov_next_cnt, const long long *link_cnt_t,
                                                long long *link_cnt_t1, long long *tile_pre) {
    if (blockIdx.x == 0) {
        if (p.linkmode && link_cnt_t) {
            // link mode: the cut links of t are complete (static bodies: from
            // their placement; moving ones: appended by the previous step's
            // geometry); the tiles of the link kernel follow them, and the
            // moving bodies' lists of t+1 start empty
            prefix_over_bodies(p, link_cnt_t, tile_pre, 1);
            for (int b = threadIdx.x; b < p.nb; b += blockDim.x)
                if (bodies[b].moving) link_cnt_t1[b] = 0;
        }
        return;
    }
    if (blockIdx.x == 1) {
        const long long n = (long long)min((unsigned long long)chg_cap, *chg_cnt);
        for (long long e = threadIdx.x; e < n; e += blockDim.x) {
            const long long c = chg_cell[e];
            flags[c] = (uint8_t)((flags[c] & ~(FL_SOLID | FL_BND)) | chg_val[e]);
        }
        __syncthreads(); // every thread has read the count
        if (threadIdx.x == 0) {
            *chg_cnt = 0ull;
            *bn_mov_next_cnt = 0ull;
        }
        return;
    }
    const long long t = tdev ? (long long)*tdev : t_arg; // the device step counter, when given
    for (int b = threadIdx.x; b < p.nb; b += blockDim.x) {
        apm_cnt[b] = 0;
        double *P = poses + (long long)b * POSE_STRIDE;
        pose(bodies[b], t, P);
        wrap_pose(p, P, P + 3);
        pose(bodies[b], t + 1, P + 6);
        wrap_pose(p, P + 6, P + 9);
        if (bodies[b].shape == 2) {
            sincos_cw(orient(bodies[b], t), P[19], P[18]);
            sincos_cw(orient(bodies[b], t + 1), P[25], P[24]);
        } else {
            P[18] = P[24] = 1.0;
            P[19] = P[25] = 0.0;
        }
        for (int a = 0; a < 3; ++a) {
            P[12 + a] = floor(P[3 + a]);
            P[15 + a] = P[3 + a] - P[12 + a];
        }
    }
}

// owner at t+1 in the shell R-2 <= |x - X(t+1)| <= R+2, A+/A- appended
__global__ void __launch_bounds__(GEOM_THREADS) k_fgeom1(Params p, GeomArgs g) {
    __shared__ Frame F;
    for (int ch = blockIdx.x; ch < g.nchunks; ch += gridDim.x) {
        const int2 cm = g.chunk_map[ch];
        const int b = cm.x;
        const BodyDev &B = g.bodies[b];
        const double *P = g.poses + (long long)b * POSE_STRIDE;
        __syncthreads();
        if (threadIdx.x == 0) make_frame(P + 9, F);
        __syncthreads();
        int lo[3];
        region_lo(p, B, P, REGION_MARGIN, lo);
        const uint16_t me = (uint16_t)(b + 1);
        const float Rin = body_rin(B), Rout = body_rout(B);
        RegionWalk w;
        walk_start(w, p, B, lo, cm.y);
        for (int j = 0; j < GEOM_CELLS; ++j, walk_next(w)) {
            RegionCell rc = walk_cell(w, p, lo);
            if (!rc.valid) continue;
            const float dist = frame_dist(p, B, F, rc);
            // link mode: the nodes whose moments the cut links of the next
            // steps read (within R + 4 of the body at t+1; never cleared)
            if (p.linkmode && dist <= Rout + MAC_BAND && !(g.flags[rc.cell] & FL_MAC)) g.flags[rc.cell] |= FL_MAC;
            if (dist < Rin - 2.0f || dist > Rout + 2.0f) continue;
            const bool in_t = g.owner_t[rc.cell] == me;
            const bool in1 = inside_screened(p, B, F, rc.x, rc.y, rc.z);
            if (in1) g.owner_t1[rc.cell] = me;
            else if (in_t || g.owner_t1[rc.cell] == me) g.owner_t1[rc.cell] = 0;
            if (in_t != in1) {
                const unsigned long long at = atomicAdd((unsigned long long *)&g.apm_cnt[b], 1ull);
                if ((long long)at < B.apm_cap) {
                    g.apm_cell[B.apm_off + at] = (uint32_t)rc.cell;
                    g.apm_sign[B.apm_off + at] = (int8_t)(in1 ? 1 : -1);
                }
            }
        }
    }
}

// flags of t+1 (solid, boundary node) in the shell R-2 .. R+3; changes appended
template <class L>
__global__ void __launch_bounds__(GEOM_THREADS) k_fgeom2(Params p, GeomArgs g) {
    __shared__ Frame F;
    for (int ch = blockIdx.x; ch < g.nchunks; ch += gridDim.x) {
        const int2 cm = g.chunk_map[ch];
        const int b = cm.x;
        const BodyDev &B = g.bodies[b];
        const double *P = g.poses + (long long)b * POSE_STRIDE;
        __syncthreads();
        if (threadIdx.x == 0) make_frame(P + 9, F);
        __syncthreads();
        int lo[3];
        region_lo(p, B, P, REGION_MARGIN, lo);
        const float Rin = body_rin(B), Rout = body_rout(B);
        for (int j = 0; j < GEOM_CELLS; ++j) {
            RegionCell rc = region_cell_i(p, B, lo, cm.y, j);
            if (!rc.valid) continue;
            const float dist = frame_dist(p, B, F, rc);
            if (dist < Rin - 2.0f || dist > Rout + 3.0f) continue;
            uint8_t nf;
            if (g.owner_t1[rc.cell]) {
                nf = FL_SOLID;
            } else {
                unsigned one = 0, lowest = 0xffffu;
                bool mine = false;
#pragma unroll
                for (int i = 1; i < L::Q; ++i) {
                    const long long a = nbr<L>(p, rc.x, rc.y, rc.z, i, 1);
                    const unsigned o = a >= 0 ? g.owner_t1[a] : 0u;
                    one |= o;
                    mine |= o == (unsigned)(b + 1);
                    if (o && o < lowest) lowest = o;
                }
                nf = one ? FL_BND : 0;
                // boundary node of t+1 next to a moving body: listed by the
                // lowest-numbered moving one (this body is moving; a
                // lower-numbered neighbour body is looked up only if present)
                bool list = mine && dist <= Rout + 1.5f;
                if (list && lowest < (unsigned)(b + 1)) {
#pragma unroll
                    for (int i = 1; i < L::Q; ++i) {
                        const long long a = nbr<L>(p, rc.x, rc.y, rc.z, i, 1);
                        const unsigned o = a >= 0 ? g.owner_t1[a] : 0u;
                        if (o && o < (unsigned)(b + 1) && g.bodies[o - 1].moving) list = false;
                    }
                }
                if (list) {
                    const unsigned long long at = atomicAdd(g.bn_mov_cnt, 1ull);
                    if ((long long)at < g.bn_mov_cap) g.bn_mov[at] = (uint32_t)rc.cell;
                }
            }
            if ((g.flags[rc.cell] & (FL_SOLID | FL_BND)) != nf) {
                const unsigned long long at = atomicAdd(g.chg_cnt, 1ull);
                if ((long long)at < g.chg_cap) {
                    g.chg_cell[at] = (uint32_t)rc.cell;
                    g.chg_val[at] = nf;
                }
            }
        }
    }
}

// link mode: the solid flags of t+1 in the shell R-2 .. R+3 (changes
// appended; link mode reads no boundary-node flag), and the cut links of t+1
// to this body (fluid node at t+1 within R + 1.5, direction i with x - c_i
// inside the body at t+1, Delta in FP32 from the pose of t+1), appended to the
// body's segment of the other list buffer: a thread first finds the links of
// its GEOM_CELLS cells, then one block scan and one atomic per chunk place them
// (their order does not matter: exact fixed-point sums)
template <class L>
__global__ void __launch_bounds__(GEOM_THREADS) k_fgeom2l(Params p, GeomArgs g) {
    __shared__ Frame F;
    for (int ch = blockIdx.x; ch < g.nchunks; ch += gridDim.x) {
        const int2 cm = g.chunk_map[ch];
        const int b = cm.x;
        const BodyDev &B = g.bodies[b];
        const double *P = g.poses + (long long)b * POSE_STRIDE;
        __syncthreads();
        if (threadIdx.x == 0) make_frame(P + 9, F);
        __syncthreads();
        int lo[3];
        region_lo(p, B, P, REGION_MARGIN, lo);
        const float Rin = body_rin(B), Rout = body_rout(B);
        const uint16_t me = (uint16_t)(b + 1);
        unsigned mj[GEOM_CELLS]; // directions of each cell's cut links to the body
        int nl = 0;
        const long long sy = p.nx, sz = (long long)p.nx * p.ny;
        RegionWalk w;
        walk_start(w, p, B, lo, cm.y);
#pragma unroll
        for (int j = 0; j < GEOM_CELLS; ++j, walk_next(w)) {
            mj[j] = 0u;
            const RegionCell rc = walk_cell(w, p, lo);
            if (!rc.valid) continue;
            const float dist = frame_dist(p, B, F, rc);
            if (dist < Rin - 2.0f || dist > Rout + 3.0f) continue;
            const bool solid1 = g.owner_t1[rc.cell] != 0;
            const uint8_t nf = solid1 ? FL_SOLID : 0;
            if ((g.flags[rc.cell] & FL_SOLID) != nf) {
                const unsigned long long at = atomicAdd(g.chg_cnt, 1ull);
                if ((long long)at < g.chg_cap) {
                    g.chg_cell[at] = (uint32_t)rc.cell;
                    g.chg_val[at] = nf;
                }
            }
            if (solid1 || dist > Rout + 1.5f) continue;
            unsigned m = 0u;
            if (inner1(p, rc.x, rc.y, rc.z)) {
#pragma unroll
                for (int i = 1; i < L::Q; ++i)
                    m |= (g.owner_t1[nbr1_inner<L>(rc.cell, sy, sz, i)] == me ? 1u : 0u) << i;
            } else {
#pragma unroll
                for (int i = 1; i < L::Q; ++i) {
                    const long long a = nbr<L>(p, rc.x, rc.y, rc.z, i, 1);
                    m |= ((a >= 0 && g.owner_t1[a] == me) ? 1u : 0u) << i;
                }
            }
            mj[j] = m;
            nl += __popc(m);
        }
        int total;
        const long long first = block_excl_scan(nl, &total); // (syncs the block)
        __shared__ unsigned long long base_s;
        if (threadIdx.x == 0)
            base_s = total ? atomicAdd((unsigned long long *)&g.link_cnt[b], (unsigned long long)total) : 0ull;
        __syncthreads();
        long long at = (long long)base_s + first;
        if (!nl) continue;
        walk_start(w, p, B, lo, cm.y);
#pragma unroll
        for (int j = 0; j < GEOM_CELLS; ++j, walk_next(w)) {
            const unsigned m = mj[j];
            if (!m) continue;
            const RegionCell rc = walk_cell(w, p, lo);
            float df[3];
            frame_disp_f(p, F, rc.x, rc.y, rc.z, df);
            for (int i = 1; i < L::Q; ++i) {
                if (!((m >> i) & 1u)) continue;
                if (at < B.link_cap) {
                    const long long jj = B.link_off + at;
                    g.Lcell[jj] = (uint32_t)rc.cell;
                    g.Ldir[jj] = (uint8_t)i;
                    g.Ldelta[jj] = (double)link_delta_f(B.halfway, B.shape, (float)B.R, (float)B.R2, F.cof, F.sif,
                                                        df, L::cx(i), L::cy(i), L::cz(i));
                }
                ++at;
            }
        }
    }
}

// boundary-node lists of step t from scratch: nodes next only to static
// bodies go to the static list, nodes next to a moving body to the moving
// list of step t (each node once: by the lowest-numbered neighbour body)
template <class L>
__global__ void __launch_bounds__(GEOM_THREADS) k_bnd_lists(Params p, GeomArgs g) {
    const int2 cm = g.chunk_map[blockIdx.x];
    const int b = cm.x;
    const BodyDev &B = g.bodies[b];
    const double *P = g.poses + (long long)b * POSE_STRIDE;
    __shared__ Frame F;
    if (threadIdx.x == 0) make_frame(P + 3, F);
    __syncthreads();
    int lo[3];
    region_lo(p, B, P, REGION_MARGIN, lo);
    const float Rin = body_rin(B), Rout = body_rout(B);
    for (int j = 0; j < GEOM_CELLS; ++j) {
        RegionCell rc = region_cell(p, B, lo, cm.y, j);
        if (!rc.valid) continue;
        const float dist = frame_dist(p, B, F, rc);
        if (dist < Rin - 0.5f || dist > Rout + 1.5f || g.owner_t[rc.cell] != 0) continue;
        int minall = 1 << 20, minmov = 1 << 20;
#pragma unroll
        for (int i = 1; i < L::Q; ++i) {
            const long long a = nbr<L>(p, rc.x, rc.y, rc.z, i, 1);
            const unsigned o = a >= 0 ? g.owner_t[a] : 0u;
            if (!o) continue;
            minall = min(minall, (int)o);
            if (g.bodies[o - 1].moving) minmov = min(minmov, (int)o);
        }
        if (minmov < (1 << 20)) {
            if (minmov == b + 1) {
                const unsigned long long at = atomicAdd(g.bn_mov_cnt, 1ull);
                if ((long long)at < g.bn_mov_cap) g.bn_mov[at] = (uint32_t)rc.cell;
            }
        } else if (minall == b + 1) {
            const unsigned long long at = atomicAdd(g.bn_static_cnt, 1ull);
            if ((long long)at < g.bn_static_cap) g.bn_static[at] = (uint32_t)rc.cell;
        }
    }
}

// link mode, at body placement: the nodes within R + 4 of every body at t
__global__ void __launch_bounds__(GEOM_THREADS) k_macband(Params p, GeomArgs g) {
    const int2 cm = g.chunk_map[blockIdx.x];
    const int b = cm.x;
    const BodyDev &B = g.bodies[b];
    const double *P = g.poses + (long long)b * POSE_STRIDE;
    __shared__ Frame F;
    if (threadIdx.x == 0) make_frame(P + 3, F);
    __syncthreads();
    int lo[3];
    region_lo(p, B, P, REGION_MARGIN, lo);
    const float Rout = body_rout(B);
    RegionWalk w;
    walk_start(w, p, B, lo, cm.y);
    for (int j = 0; j < GEOM_CELLS; ++j, walk_next(w)) {
        RegionCell rc = walk_cell(w, p, lo);
        if (!rc.valid) continue;
        if (frame_dist(p, B, F, rc) <= Rout + MAC_BAND) g.flags[rc.cell] |= FL_MAC;
    }
}

} // namespace

cudaError_t launch_macband(const Params &p, const GeomArgs &g, cudaStream_t s) {
    if (g.nchunks == 0) return cudaSuccess;
    k_macband<<<g.nchunks, GEOM_THREADS, 0, s>>>(p, g);
    return cudaGetLastError();
}

cudaError_t launch_prep(const Params &p, const BodyDev *bodies, const long long *link_cnt, long long *link_pre,
                        long long *tile_pre, double *poses, long long t, const unsigned long long *tdev,
                        uint8_t *flags, const long long *apm_cnt, const uint32_t *apm_cell, const int8_t *apm_sign,
                        cudaStream_t s) {
    k_prep<<<1, 1024, 0, s>>>(p, bodies, link_cnt, link_pre, tile_pre, poses, t, tdev, flags, apm_cnt, apm_cell,
                              apm_sign);
    return cudaGetLastError();
}

cudaError_t launch_fprep(const Params &p, const BodyDev *bodies, double *poses, long long t,
                         const unsigned long long *tdev, uint8_t *flags, unsigned long long *chg_cnt,
                         const uint32_t *chg_cell, const uint8_t *chg_val, long long chg_cap, long long *apm_cnt,
                         unsigned long long *bn_mov_next_cnt, const long long *link_cnt_t, long long *link_cnt_t1,
                         long long *tile_pre, cudaStream_t s) {
    k_fprep<<<3, 1024, 0, s>>>(p, bodies, poses, t, tdev, flags, chg_cnt, chg_cell, chg_val, chg_cap, apm_cnt,
                               bn_mov_next_cnt, link_cnt_t, link_cnt_t1, tile_pre);
    return cudaGetLastError();
}


cudaError_t launch_bnd_lists(int Q, const Params &p, const GeomArgs &g, cudaStream_t s) {
    if (g.nchunks == 0) return cudaSuccess;
    if (Q == 9) k_bnd_lists<Lat<9>><<<g.nchunks, GEOM_THREADS, 0, s>>>(p, g);
    else k_bnd_lists<Lat<19>><<<g.nchunks, GEOM_THREADS, 0, s>>>(p, g);
    return cudaGetLastError();
}

cudaError_t launch_fgeom1(int, const Params &p, const GeomArgs &g, cudaStream_t s) {
    if (g.nchunks == 0) return cudaSuccess;
    k_fgeom1<<<g.grid_cap > 0 ? min(g.nchunks, g.grid_cap) : g.nchunks, GEOM_THREADS, 0, s>>>(p, g);
    return cudaGetLastError();
}

cudaError_t launch_fgeom2(int Q, const Params &p, const GeomArgs &g, cudaStream_t s) {
    if (g.nchunks == 0) return cudaSuccess;
    const int grid = g.grid_cap > 0 ? min(g.nchunks, g.grid_cap) : g.nchunks;
    if (p.linkmode) {
        if (Q == 9) k_fgeom2l<Lat<9>><<<grid, GEOM_THREADS, 0, s>>>(p, g);
        else k_fgeom2l<Lat<19>><<<grid, GEOM_THREADS, 0, s>>>(p, g);
    } else if (Q == 9) {
        k_fgeom2<Lat<9>><<<grid, GEOM_THREADS, 0, s>>>(p, g);
    } else {
        k_fgeom2<Lat<19>><<<grid, GEOM_THREADS, 0, s>>>(p, g);
    }
    return cudaGetLastError();
}

cudaError_t launch_raster(int, const Params &p, const GeomArgs &g, uint16_t *owner, long long t_pose,
                          cudaStream_t s) {
    if (g.nchunks == 0) return cudaSuccess;
    k_raster<<<g.nchunks, GEOM_THREADS, 0, s>>>(p, g, owner, t_pose);
    return cudaGetLastError();
}

cudaError_t launch_geom_a(int, const Params &p, const GeomArgs &g, cudaStream_t s) {
    if (g.nchunks == 0) return cudaSuccess;
    k_geom_a<<<g.nchunks, GEOM_THREADS, 0, s>>>(p, g);
    return cudaGetLastError();
}

cudaError_t launch_geom_b(int Q, const Params &p, const GeomArgs &g, cudaStream_t s) {
    if (g.nchunks == 0) return cudaSuccess;
    if (Q == 9) k_geom_b<Lat<9>><<<g.nchunks, GEOM_THREADS, 0, s>>>(p, g);
    else k_geom_b<Lat<19>><<<g.nchunks, GEOM_THREADS, 0, s>>>(p, g);
    return cudaGetLastError();
}

cudaError_t launch_geom_c(int Q, const Params &p, const GeomArgs &g, cudaStream_t s) {
    if (g.nchunks == 0) return cudaSuccess;
    if (Q == 9) k_geom_c<Lat<9>><<<g.nchunks, GEOM_THREADS, 0, s>>>(p, g);
    else k_geom_c<Lat<19>><<<g.nchunks, GEOM_THREADS, 0, s>>>(p, g);
    return cudaGetLastError();
}

cudaError_t launch_flags_full(int Q, const Params &p, const uint16_t *owner, uint8_t *flags, cudaStream_t s) {
    const int bx = p.nx >= 128 ? 128 : 32;
    dim3 grid((p.nx + bx - 1) / bx, p.ny, p.nz);
    if (Q == 9) k_flags_full<Lat<9>><<<grid, bx, 0, s>>>(p, owner, flags);
    else k_flags_full<Lat<19>><<<grid, bx, 0, s>>>(p, owner, flags);
    return cudaGetLastError();
}

template <class L>
static cudaError_t export_t(int prec, const Params &p, const void *pop, double *out, cudaStream_t s) {
    const int grid = 4 * 152;
    if (prec == 0) k_export<L, PF64><<<grid, 256, 0, s>>>(p, (const double *)pop, out);
    else if (prec == 1) k_export<L, PF32><<<grid, 256, 0, s>>>(p, (const float *)pop, out);
    else k_export<L, PF16><<<grid, 256, 0, s>>>(p, (const __half *)pop, out);
    return cudaGetLastError();
}

template <class L>
static cudaError_t import_t(int prec, const Params &p, const double *in, void *pop, cudaStream_t s) {
    const int grid = 4 * 152;
    if (prec == 0) k_import<L, PF64><<<grid, 256, 0, s>>>(p, in, (double *)pop);
    else if (prec == 1) k_import<L, PF32><<<grid, 256, 0, s>>>(p, in, (float *)pop);
    else k_import<L, PF16><<<grid, 256, 0, s>>>(p, in, (__half *)pop);
    return cudaGetLastError();
}

// Free bodies (one thread per body), after the force/torque row of step t is
// complete.  Explicit scheme: the pose advances with U(t) -- the motion the
// step's A+/A- sets were built from.  Semi-implicit schemes (the row holds the
// impulsive terms of the previous displacement or of a predicted one): the
// pose advances with U(t+1), and the step's A+/A- sets are built afterwards.
// Forward Euler gives U(t+1) and W(t+1) from the
// lattice-frame force and torque (Eqs. ForceInMovement, TorqueInMovement:
// static plus impulsive terms), weight less buoyancy (rho_b - rho0) V g and
// M = rho_b V, I = M R^2/2 (cylinder, about z), M (R^2 + R2^2)/4 (ellipse,
// V = pi R R2 nz) or 2/5 M R^2 (sphere).  The body record keeps X0 = X(t+1),
// theta0 = theta(t+1), t0 = t+1, so pose(t+1), pose(t+2) follow.
// A body within 2 cells of a non-periodic face, or faster than 0.25 at its
// surface, sets counters[7].
__global__ void k_free(Params p, BodyDev *bodies, const double *series, unsigned long long *counters,
                       const unsigned long long *tdev) {
    const long long t = (long long)*tdev; // the device step index
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= p.nb) return;
    BodyDev &B = bodies[b];
    if (!B.free) return;
    const double *Rw = series + ((t % p.series_cap) * p.nb + b) * SERIES_ROW;
    const double PI = 3.14159265358979323846;
    double V, I;
    if (B.shape == 1) V = 4.0 / 3.0 * PI * B.R * B.R * B.R;
    else if (B.shape == 2) V = PI * B.R * B.R2 * (double)p.nz;
    else V = PI * B.R * B.R * (double)p.nz;
    const double M = B.density_ratio * p.rho0 * V;
    if (B.shape == 1) I = 0.4 * M * B.R * B.R;
    else if (B.shape == 2) I = 0.25 * M * (B.R * B.R + B.R2 * B.R2);
    else I = 0.5 * M * B.R * B.R;
    double X1[3], X0[3];
    pose(B, t + 1, X1);
    pose(B, t, X0);
    double th1 = orient(B, t + 1);
    const double th0 = orient(B, t);
    for (int a = 0; a < 3; ++a) {
        const double F = Rw[a] + Rw[6 + a];
        B.U[a] = B.U[a] + (F + (B.density_ratio - 1.0) * p.rho0 * V * p.gravity[a]) / M;
    }
    if (B.shape == 1) {
        for (int a = 0; a < 3; ++a) B.W[a] = B.W[a] + (Rw[3 + a] + Rw[9 + a]) / I;
    } else {
        B.W[2] = B.W[2] + (Rw[5] + Rw[11]) / I;
    }
    if (p.free_scheme) { // semi-implicit: the step's displacement is made with U(t+1)
        for (int a = 0; a < 3; ++a) X1[a] = X0[a] + B.U[a];
        th1 = th0 + B.W[2];
    }
    for (int a = 0; a < 3; ++a) B.X0[a] = X1[a];
    B.theta0 = th1;
    B.t0 = t + 1;
    bool bad = false;
    for (int a = 0; a < 3; ++a) {
        if (p.per[a] || (a == 2 && along_z(B.shape))) continue;
        const double n = (double)axis_len(p, a);
        if (X1[a] - B.R < 2.0 || X1[a] + B.R > n - 3.0) bad = true;
    }
    const double us = sqrt(B.U[0] * B.U[0] + B.U[1] * B.U[1] + B.U[2] * B.U[2]) +
                      B.R * sqrt(B.W[0] * B.W[0] + B.W[1] * B.W[1] + B.W[2] * B.W[2]);
    if (!(us <= 0.25)) bad = true;
    if (bad) atomicOr(&counters[7], 1ull);
}

cudaError_t launch_free(const Params &p, BodyDev *bodies, const double *series, unsigned long long *counters,
                        const unsigned long long *tdev, cudaStream_t s) {
    if (p.nb == 0) return cudaSuccess;
    k_free<<<(p.nb + 127) / 128, 128, 0, s>>>(p, bodies, series, counters, tdev);
    return cudaGetLastError();
}

// semi-implicit schemes, after k_free: the poses of t+1 of the free bodies
// from their new records (wrapped pose and orientation of t+1; those of t stay)
__global__ void k_pose1(Params p, const BodyDev *bodies, double *poses, const unsigned long long *tdev) {
    const long long t = (long long)*tdev;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= p.nb || !bodies[b].free) return;
    double *P = poses + (long long)b * POSE_STRIDE;
    pose(bodies[b], t + 1, P + 6);
    wrap_pose(p, P + 6, P + 9);
    if (bodies[b].shape == 2) sincos_cw(orient(bodies[b], t + 1), P[25], P[24]);
}

cudaError_t launch_pose1(const Params &p, const BodyDev *bodies, double *poses, const unsigned long long *tdev,
                         cudaStream_t s) {
    if (p.nb == 0) return cudaSuccess;
    k_pose1<<<(p.nb + 127) / 128, 128, 0, s>>>(p, bodies, poses, tdev);
    return cudaGetLastError();
}

cudaError_t launch_export(int Q, int prec, const Params &p, const void *pop, double *out, cudaStream_t s) {
    return Q == 9 ? export_t<Lat<9>>(prec, p, pop, out, s) : export_t<Lat<19>>(prec, p, pop, out, s);
}

cudaError_t launch_import(int Q, int prec, const Params &p, const double *in, void *pop, cudaStream_t s) {
    return Q == 9 ? import_t<Lat<9>>(prec, p, in, pop, s) : import_t<Lat<19>>(prec, p, in, pop, s);
}

} // namespace lbm
