// lbm_region.cuh -- enumeration of the node region around a body and
// lattice-neighbour helpers shared by the geometry and boundary-node kernels.
#pragma once

#include "lbm_dev.cuh"

namespace lbm {

struct RegionCell {
    bool valid;
    int x, y, z;
    long long cell;
};

// the j-th (0..GEOM_CELLS-1) region cell of this thread in chunk `chunk`:
// a thread owns GEOM_CELLS consecutive cells, so per-thread counts followed
// by a block scan keep every list in cell order
__device__ __forceinline__ RegionCell region_cell(const Params &p, const BodyDev &B, const int lo[3], int chunk,
                                                  int j) {
    RegionCell rc{false, 0, 0, 0, 0};
    const int e0 = B.ext[0], e1 = B.ext[1];
    const int vol = e0 * e1 * B.ext[2];
    const int k = chunk * GEOM_CHUNK + (int)threadIdx.x * GEOM_CELLS + j;
    if (k >= vol) return rc;
    const int kz = k / (e0 * e1);
    const int rem = k - kz * e0 * e1;
    const int ky = rem / e0;
    const int kx = rem - ky * e0;
    rc.x = region_axis(kx, lo[0], e0, p.nx, p.per[0]);
    rc.y = region_axis(ky, lo[1], e1, p.ny, p.per[1]);
    rc.z = region_axis(kz, lo[2], B.ext[2], p.nz, p.per[2]);
    if (rc.x < 0 || rc.y < 0 || rc.z < 0) return rc;
    rc.valid = true;
    rc.cell = cell_of(p, rc.x, rc.y, rc.z);
    return rc;
}

// the same cells as region_cell, interleaved: pass j of a chunk takes cells
// j * GEOM_THREADS + threadIdx.x, so a warp reads consecutive cells (for the
// kernels whose lists do not depend on the order, appended with atomics)
__device__ __forceinline__ RegionCell region_cell_i(const Params &p, const BodyDev &B, const int lo[3], int chunk,
                                                    int j) {
    RegionCell rc{false, 0, 0, 0, 0};
    const int e0 = B.ext[0], e1 = B.ext[1];
    const int vol = e0 * e1 * B.ext[2];
    const int k = chunk * GEOM_CHUNK + j * GEOM_THREADS + (int)threadIdx.x;
    if (k >= vol) return rc;
    const int kz = k / (e0 * e1);
    const int rem = k - kz * e0 * e1;
    const int ky = rem / e0;
    const int kx = rem - ky * e0;
    rc.x = region_axis(kx, lo[0], e0, p.nx, p.per[0]);
    rc.y = region_axis(ky, lo[1], e1, p.ny, p.per[1]);
    rc.z = region_axis(kz, lo[2], B.ext[2], p.nz, p.per[2]);
    if (rc.x < 0 || rc.y < 0 || rc.z < 0) return rc;
    rc.valid = true;
    rc.cell = cell_of(p, rc.x, rc.y, rc.z);
    return rc;
}

// The cells of region_cell_i for j = 0, 1, ... of one chunk, walked with
// the divisions done once: the thread's first cell is split into region
// coordinates, each step adds GEOM_THREADS cells in the same mixed radix, and
// the periodic wrap of each axis uses the start s0 and split wr that
// region_axis recomputes per call.
struct RegionWalk {
    int k, vol, kx, ky, kz, e0, e1, e2, dx, dy, dz;
    int s0[3], wr[3], full[3];
};

__device__ __forceinline__ void walk_start(RegionWalk &w, const Params &p, const BodyDev &B, const int lo[3],
                                           int chunk) {
    w.e0 = B.ext[0];
    w.e1 = B.ext[1];
    w.e2 = B.ext[2];
    w.vol = w.e0 * w.e1 * w.e2;
    w.k = chunk * GEOM_CHUNK + (int)threadIdx.x;
    const int plane = w.e0 * w.e1;
    w.kz = w.k / plane;
    const int rem = w.k - w.kz * plane;
    w.ky = rem / w.e0;
    w.kx = rem - w.ky * w.e0;
    w.dz = GEOM_THREADS / plane;
    const int r2 = GEOM_THREADS - w.dz * plane;
    w.dy = r2 / w.e0;
    w.dx = r2 - w.dy * w.e0;
    const int n[3] = {p.nx, p.ny, p.nz}, len[3] = {w.e0, w.e1, w.e2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        w.full[a] = len[a] >= n[a];
        w.s0[a] = ((lo[a] % n[a]) + n[a]) % n[a];
        w.wr[a] = w.s0[a] + len[a] - n[a];
    }
}

__device__ __forceinline__ void walk_next(RegionWalk &w) {
    w.k += GEOM_THREADS;
    w.kx += w.dx;
    if (w.kx >= w.e0) {
        w.kx -= w.e0;
        ++w.ky;
    }
    w.ky += w.dy;
    if (w.ky >= w.e1) {
        w.ky -= w.e1;
        ++w.kz;
    }
    w.kz += w.dz;
}

// region_axis with the walk's per-axis constants
__device__ __forceinline__ int walk_axis(const RegionWalk &w, int a, int k, int lo, int n, int periodic) {
    if (!periodic) {
        const int v = lo + k;
        return (v < 0 || v >= n) ? -1 : v;
    }
    if (w.full[a]) return k < n ? k : -1;
    if (w.wr[a] > 0) return k < w.wr[a] ? k : w.s0[a] + (k - w.wr[a]);
    return w.s0[a] + k;
}

__device__ __forceinline__ RegionCell walk_cell(const RegionWalk &w, const Params &p, const int lo[3]) {
    RegionCell rc{false, 0, 0, 0, 0};
    if (w.k >= w.vol) return rc;
    rc.x = walk_axis(w, 0, w.kx, lo[0], p.nx, p.per[0]);
    rc.y = walk_axis(w, 1, w.ky, lo[1], p.ny, p.per[1]);
    rc.z = walk_axis(w, 2, w.kz, lo[2], p.nz, p.per[2]);
    if (rc.x < 0 || rc.y < 0 || rc.z < 0) return rc;
    rc.valid = true;
    rc.cell = cell_of(p, rc.x, rc.y, rc.z);
    return rc;
}

// neighbour x - k c_i; -1 if it falls outside a non-periodic axis
template <class L>
__device__ __forceinline__ long long nbr(const Params &p, int x, int y, int z, int i, int k) {
    int q[3] = {x - k * L::cx(i), y - k * L::cy(i), z - k * L::cz(i)};
    const int n[3] = {p.nx, p.ny, p.nz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (q[a] >= 0 && q[a] < n[a]) continue;
        if (!p.per[a]) return -1;
        while (q[a] < 0) q[a] += n[a]; // |k c_i| <= 2: at most two turns
        while (q[a] >= n[a]) q[a] -= n[a];
    }
    return cell_of(p, q[0], q[1], q[2]);
}

// nbr<L>(p, x, y, z, i, 1) for a node one cell or more inside every face of
// the lattice (no wrap): the cell index minus c_i's offset
template <class L>
__device__ __forceinline__ long long nbr1_inner(long long cell, long long sy, long long sz, int i) {
    return cell - ((long long)L::cx(i) + (L::cy(i) == 0 ? 0ll : (L::cy(i) > 0 ? sy : -sy)) +
                   (L::cz(i) == 0 ? 0ll : (L::cz(i) > 0 ? sz : -sz)));
}

__device__ __forceinline__ bool inner1(const Params &p, int x, int y, int z) {
    return x >= 1 && x <= p.nx - 2 && y >= 1 && y <= p.ny - 2 && (p.nz == 1 || (z >= 1 && z <= p.nz - 2));
}

__device__ __forceinline__ bool edge_node(const Params &p, int x, int y, int z) {
    return (!p.per[0] && (x == 0 || x == p.nx - 1)) || (!p.per[1] && (y == 0 || y == p.ny - 1)) ||
           (!p.per[2] && (z == 0 || z == p.nz - 1));
}

// store macros at x if x is fluid and within two hops of a solid node (the
// fluid end of a cut link, or its u_G node), or on a non-periodic face
__device__ __forceinline__ float frame_dist(const Params &p, const BodyDev &B, const Frame &F, const RegionCell &rc) {
    float d[3];
    frame_disp_f(p, F, rc.x, rc.y, rc.z, d);
    return sqrtf(d[0] * d[0] + d[1] * d[1] + (B.shape == 1 ? d[2] * d[2] : 0.0f));
}

} // namespace lbm
