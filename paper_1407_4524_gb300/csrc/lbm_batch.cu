// lbm_batch.cu -- batched kernels of the serving mode.
//
// A serving batch keeps many independent solves resident (reduced-precision
// modes, static bodies) and advances all of them by one step per tick: the
// stream-collide pass of each solve (the standalone kernel, one launch per
// solve on parallel graph branches while few are resident; with many, the
// batched kernel below over a block table covering every solve's rows), the
// boundary-node kernel of each lattice over the concatenated node lists, and
// one end-of-step kernel (series rows, step counters).  Every solve runs the
// same per-node arithmetic as a standalone domain, and its force/torque sums
// are exact fixed point, so a solve's results do not depend on what else is
// in the batch.
#include "lbm_bnd.cuh"
#include "lbm_launch.cuh"

namespace lbm {

namespace {

// work[k] = (slot, row, x0): block k does the BBULK_THREADS nodes x0 .. of one
// row (y, z) of one solve, row = y + ny * z.  Row-aligned blocks keep a warp
// on one row (so only the blocks at the row ends take the face path) and
// need no 64-bit division per node.
template <class L, class P, int FM>
__global__ void __launch_bounds__(BBULK_THREADS, FM == FM_GENERAL ? 16 : 20) k_bbulk(const SolveDev *__restrict__ solves,
                                                         const int4 *__restrict__ work) {
    // the solve's record in shared memory: its parameters are read many times
    __shared__ SolveDev sv;
    const int4 w = work[blockIdx.x];
    {
        static_assert(sizeof(SolveDev) % 4 == 0, "SolveDev is copied as 32-bit words");
        const int *from = (const int *)(solves + w.x);
        int *to = (int *)&sv;
        for (int k = threadIdx.x; k < (int)(sizeof(SolveDev) / 4); k += blockDim.x) to[k] = from[k];
    }
    __syncthreads();
    if (!sv.active) return;
    const int x = w.z + threadIdx.x;
    if (x >= sv.p.nx) return;
    const int z = w.y / sv.p.ny, y = w.y - z * sv.p.ny;
    const int cur = (int)(sv.t & 1);
    bulk_node<L, P, FM>(sv.p, (const typename P::S *)sv.pop[cur], (typename P::S *)sv.pop[cur ^ 1], sv.flags,
                        (const typename P::C *)nullptr, (typename P::C *)nullptr, x, y, z);
}

// warp per boundary node over the node lists of the slots of one lattice
template <class L, class P>
__global__ void __launch_bounds__(BND_THREADS) k_bbnd(const SolveDev *__restrict__ solves,
                                                      const int *__restrict__ slots,
                                                      const long long *__restrict__ node_pre, int nslots) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long total = node_pre[nslots];
    int k_slot = 0;
    for (long long k = warp; k < total; k += nwarps) {
        while (k_slot + 1 < nslots && node_pre[k_slot + 1] <= k) ++k_slot; // k grows: forward scan
        const SolveDev &sv = solves[slots[k_slot]];
        if (!sv.active) continue;
        const int cur = (int)(sv.t & 1);
        BndArgs a{};
        a.static_cells = sv.bn_static;
        a.static_cnt = sv.bn_cnt;
        a.static_cap = sv.bn_cap;
        a.owner_t = sv.owner;
        a.owner_t1 = sv.owner;
        a.bodies = sv.bodies;
        a.poses = sv.poses;
        StepBufs sb{};
        sb.src = sv.pop[cur];
        sb.dst = sv.pop[cur ^ 1];
        sb.counters = sv.counters;
        sb.acc = sv.acc;
        unsigned nl = 0;
        bnd_node<L, P>(sv.p, a, sb, sv.bn_static[k - node_pre[k_slot]], true, nl);
        if (lane == 0 && nl) atomicAdd(&sv.counters[3], (unsigned long long)nl);
    }
}

// end of step of every solve: series rows from the fixed-point sums, t + 1;
// runs after both the bulk and the boundary-node kernels of the tick (they
// read t)
__global__ void __launch_bounds__(128) k_bfinish(SolveDev *solves, const int *slots) {
    SolveDev &sv = solves[slots[blockIdx.x]];
    if (!sv.active) return;
    const Params &p = sv.p;
    for (int b = 0; b < p.nb; ++b) {
        double *row = sv.series + ((sv.t % p.series_cap) * p.nb + b) * SERIES_ROW;
        unsigned long long *acc = sv.acc + (long long)b * SERIES_ROW;
        if (threadIdx.x < SERIES_ROW) {
            const int k = threadIdx.x;
            if (k >= 6 && k < 12) {
                row[k] = 0.0; // static bodies: no impulsive terms
            } else {
                row[k] = from_fx(acc[k]);
                acc[k] = 0ull;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sv.counters[4] = sv.counters[3];
        sv.counters[3] = 0ull;
        sv.t += 1;
        if (sv.t >= sv.t_end) sv.active = 0;
    }
}

template <class L, class P>
cudaError_t bbulk_fm(int fm, const SolveDev *solves, const int4 *work, int nwork, cudaStream_t s) {
    if (fm == FM_PERIODIC) k_bbulk<L, P, FM_PERIODIC><<<nwork, BBULK_THREADS, 0, s>>>(solves, work);
    else if (fm == FM_XFACES) k_bbulk<L, P, FM_XFACES><<<nwork, BBULK_THREADS, 0, s>>>(solves, work);
    else k_bbulk<L, P, FM_GENERAL><<<nwork, BBULK_THREADS, 0, s>>>(solves, work);
    return cudaGetLastError();
}

template <class L>
cudaError_t bbulk_t(int kind, int fm, const SolveDev *solves, const int4 *work, int nwork, cudaStream_t s) {
    if (nwork == 0) return cudaSuccess;
    return kind == BK_FP16 ? bbulk_fm<L, PF16>(fm, solves, work, nwork, s) : bbulk_fm<L, PF32>(fm, solves, work, nwork, s);
}

template <class L, class P>
cudaError_t bbnd_t(const SolveDev *solves, const int *slots, const long long *node_pre, int nslots, int grid,
                   cudaStream_t s) {
    if (nslots == 0 || grid <= 0) return cudaSuccess;
    k_bbnd<L, P><<<grid, BND_THREADS, 0, s>>>(solves, slots, node_pre, nslots);
    return cudaGetLastError();
}

} // namespace

cudaError_t launch_bbulk(int Q, int kind, int fm, const SolveDev *solves, const int4 *work, int nwork,
                         cudaStream_t s) {
    return Q == 9 ? bbulk_t<Lat<9>>(kind, fm, solves, work, nwork, s) : bbulk_t<Lat<19>>(kind, fm, solves, work, nwork, s);
}

cudaError_t launch_bbnd(int Q, int prec, const SolveDev *solves, const int *slots, const long long *node_pre,
                        int nslots, int grid, cudaStream_t s) {
    if (prec == 1)
        return Q == 9 ? bbnd_t<Lat<9>, PF32>(solves, slots, node_pre, nslots, grid, s)
                      : bbnd_t<Lat<19>, PF32>(solves, slots, node_pre, nslots, grid, s);
    return Q == 9 ? bbnd_t<Lat<9>, PF16>(solves, slots, node_pre, nslots, grid, s)
                  : bbnd_t<Lat<19>, PF16>(solves, slots, node_pre, nslots, grid, s);
}

cudaError_t launch_bfinish(SolveDev *solves, const int *slots, int nslots, cudaStream_t s) {
    if (nslots == 0) return cudaSuccess;
    k_bfinish<<<nslots, 128, 0, s>>>(solves, slots);
    return cudaGetLastError();
}

} // namespace lbm
