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
