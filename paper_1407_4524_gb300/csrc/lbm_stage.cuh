// lbm_stage.cuh -- stream-collide with the source rows staged in shared memory
// by bulk asynchronous copies (reduced-precision modes).
//
// A block handles segments of SEG = min(256, nx) consecutive nodes of one row
// (y, z), one node per thread, in a loop over segments with two shared-memory
// stages: while the nodes of segment k are computed from stage k & 1, the
// copies of segment k + 1 fill the other stage.  For each direction i one
// 1-D bulk copy (cp.async.bulk, completion counted in bytes on the stage's
// mbarrier) brings the source row of plane i -- row (y - c_iy, z - c_iz)
// after the periodic wrap, or, on a y / z wall row, the node row of plane
// opp(i) (bounce-back) -- over the window x0 - PAD .. x0 + SEG + PAD, PAD
// being 16 bytes of elements.  Periodic x adds the wrapped 16-byte end
// chunks of the row.  A thread then takes population i from slot i at its
// own x - c_ix: the memory parallelism comes from the copies in flight, not
// from registers.  The face rule is the one of pull_edge; the wall / inlet
// links on the x faces (one node per row end) read their own opposite
// population from global memory.  Each node runs exactly the arithmetic of
// bulk_node, so the results are those of k_bulk bit for bit.
//
// Requirements (checked by the launcher): nx * sizeof(S) a multiple of 16
// bytes (so every row and every window edge is 16-byte aligned), reduced
// precision.  Every wait on an mbarrier is bounded (one second); on expiry
// the block records LBM_TIMEOUT_FLAG in counters[6], waits (bounded) for its
// own copies and returns.
#pragma once

#include "lbm_step.cuh"

namespace lbm {

constexpr int STAGE_SEG = 256;        // nodes per segment (threads per block) at most
constexpr int STAGE_BLOCKS_PER_SM = 4;
constexpr unsigned long long LBM_TIMEOUT_FLAG = 1ull;
constexpr unsigned long long STAGE_WAIT_NS = 1000000000ull; // a wait gives up after one second
constexpr long long STAGE_WAIT_ROUNDS = 1ll << 24;             // and after this many poll rounds at most

__device__ __forceinline__ unsigned smem_u32(const void *ptr) {
    return (unsigned)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\t"
                 "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0u;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait for the phase of the given parity (one second, and a round
// count); false if it never completed
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long long r = 0; r < STAGE_WAIT_ROUNDS; ++r) {
        for (int k = 0; k < 64; ++k)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > STAGE_WAIT_NS) return false;
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(void *sdst, const void *gsrc, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(sdst)),
                 "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// geometry of segment s: row (y, z) and first node x0
struct Seg {
    int x0, y, z;
};
__device__ __forceinline__ Seg seg_of(const Params &p, int seg, long long s) {
    const int spr = (p.nx + seg - 1) / seg;
    const long long r = s / spr;
    Seg g;
    g.x0 = (int)(s - r * spr) * seg;
    g.y = (int)(r % p.ny);
    g.z = (int)(r / p.ny);
    return g;
}

// Issue the copies of segment g into stage buffer `buf` (Q slots of W
// elements) on barrier `bar`.  Called by warp 0 (a full warp): lane 0
// registers the byte count, then lane i copies slot i.
template <class L, class S>
__device__ __forceinline__ void stage_issue(const Params &p, const S *__restrict__ src, S *buf, int W, int seg,
                                            const Seg &g, unsigned long long *bar) {
    constexpr int PAD = 16 / (int)sizeof(S);
    const int lane = threadIdx.x & 31;
    const int xs = g.x0 > 0 ? g.x0 - PAD : 0;
    const int xe = min(p.nx, g.x0 + seg + PAD);
    const bool wrap_lo = g.x0 == 0 && p.per[0], wrap_hi = g.x0 + seg >= p.nx && p.per[0];
    const unsigned row_bytes = (unsigned)((xe - xs) * (int)sizeof(S));
    const unsigned chunk = 16u;
    const unsigned total = (unsigned)L::Q * (row_bytes + (wrap_lo ? chunk : 0u) + (wrap_hi ? chunk : 0u));
    if (lane == 0) mbar_arrive_expect_tx(bar, total);
    __syncwarp();
    // test hook: register the bytes but issue no copy, so that the wait on
    // this stage expires (the timeout path is exercised without a fault)
    if (p.stage_expire_test) return;
    if (lane < L::Q) {
        const int i = lane;
        int ym, yp, zm, zp;
        unsigned fl = 0u;
        face_axis(g.y, p.ny, p.per[1], p.edge[2], p.edge[3], 1, ym, yp, fl);
        face_axis(g.z, p.nz, p.per[2], p.edge[4], p.edge[5], 2, zm, zp, fl);
        const int cy = L::cy(i), cz = L::cz(i);
        // y / z bounce of direction i: its c_y (c_z) points out of a wall row
        const bool ybz = (cy == 1 && (fl & 4u)) || (cy == -1 && (fl & 8u)) || (cz == 1 && (fl & 16u)) ||
                         (cz == -1 && (fl & 32u));
        const int sy = cy == 1 ? ym : (cy == -1 ? yp : g.y);
        const int sz = cz == 1 ? zm : (cz == -1 ? zp : g.z);
        const S *row = ybz ? src + (long long)L::opp(i) * p.N + cell_of(p, 0, g.y, g.z)
                           : src + (long long)i * p.N + cell_of(p, 0, sy, sz);
        S *slot = buf + (long long)i * W;
        // window element e holds x = x0 - PAD + e
        bulk_g2s(slot + (xs - (g.x0 - PAD)), row + xs, row_bytes, bar);
        if (wrap_lo) bulk_g2s(slot, row + p.nx - PAD, chunk, bar);
        if (wrap_hi) bulk_g2s(slot + (p.nx - g.x0) + PAD, row, chunk, bar);
    }
}

template <class L, class P>
__global__ void __launch_bounds__(STAGE_SEG, STAGE_BLOCKS_PER_SM)
    k_bulk_staged(Params p, const typename P::S *__restrict__ src, typename P::S *__restrict__ dst,
                  const uint8_t *__restrict__ flags, unsigned long long *counters, float *__restrict__ mac_t1) {
    using S = typename P::S;
    constexpr int PAD = 16 / (int)sizeof(S);
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned long long *bar = (unsigned long long *)smem; // two stage barriers
    const int seg = blockDim.x;
    const int W = seg + 2 * PAD;
    S *stage0 = (S *)(smem + 128);
    S *stage1 = stage0 + (long long)L::Q * W;
    const long long nseg = (long long)((p.nx + seg - 1) / seg) * p.ny * p.nz;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int t = threadIdx.x;
    long long s = blockIdx.x;
    if (s < nseg && t < 32) stage_issue<L, S>(p, src, stage0, W, seg, seg_of(p, seg, s), &bar[0]);
    bool timed_out = false;
    int k = 0;
    for (; s < nseg; s += gridDim.x, ++k) {
        const int b = k & 1;
        const long long s_next = s + gridDim.x;
        if (s_next < nseg && t < 32) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            stage_issue<L, S>(p, src, b ? stage0 : stage1, W, seg, seg_of(p, seg, s_next), &bar[b ^ 1]);
        }
        const bool ok = mbar_wait_bounded(&bar[b], (unsigned)((k >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        const Seg g = seg_of(p, seg, s);
        const int x = g.x0 + t;
        const S *buf = b ? stage1 : stage0;
        if (x < p.nx) {
            const long long cell = cell_of(p, x, g.y, g.z);
            const uint8_t fl = __ldg(flags + cell);
            if (!(fl & FL_SOLID) && (p.linkmode || !(fl & FL_BND))) {
                // y / z wall bounces of the row (same for every node of the segment)
                int ym, yp, zm, zp;
                unsigned ffl = 0u;
                face_axis(g.y, p.ny, p.per[1], p.edge[2], p.edge[3], 1, ym, yp, ffl);
                face_axis(g.z, p.nz, p.per[2], p.edge[4], p.edge[5], 2, zm, zp, ffl);
                const unsigned yzb = face_dirs<L>(ffl, 0);
                const bool lo_face = x == 0 && !p.per[0], hi_face = x == p.nx - 1 && !p.per[0];
                const int e_lo = p.edge[0], e_hi = p.edge[1];
                unsigned bounce = yzb, inlet_only = 0u;
                float f[L::Q];
#pragma unroll
                for (int i = 0; i < L::Q; ++i) {
                    const int cx = L::cx(i);
                    const bool ybz = (yzb >> i) & 1u;
                    const int e = ybz ? PAD + t : PAD + t - cx;
                    float v = ldP(buf + (long long)i * W + e);
                    if (!ybz && cx == 1 && lo_face) { // x - 1 is outside: wall / inlet link
                        v = ldS(src + (long long)L::opp(i) * p.N + cell);
                        bounce |= 1u << i;
                        if (e_lo == 2) inlet_only |= 1u << i;
                    } else if (!ybz && cx == -1 && hi_face) {
                        if (e_hi == 3) v = ldP(buf + (long long)i * W + PAD + t); // outlet: own column
                        else {
                            v = ldS(src + (long long)L::opp(i) * p.N + cell);
                            bounce |= 1u << i;
                            if (e_hi == 2) inlet_only |= 1u << i;
                        }
                    }
                    f[i] = v;
                }
                if (bounce) face_terms<L, P>(p, src, (const float *)nullptr, g.y, cell, bounce, inlet_only, f);
                float drho, u[3];
                moments_f<L>(p, f, drho, u);
                if (p.linkmode && (fl & FL_MAC)) store_mac(mac_t1, cell, drho, u);
                collide_f<L>(p, f, drho, u);
#pragma unroll
                for (int i = 0; i < L::Q; ++i) stS(dst + (long long)i * p.N + cell, f[i]);
            }
        }
        __syncthreads(); // stage b is free again
    }
    if (timed_out) {
        if (t == 0) atomicOr(&counters[6], LBM_TIMEOUT_FLAG);
        // let the copies of this block finish before its shared memory goes away
        if (t == 0) {
            mbar_wait_bounded(&bar[k & 1], (unsigned)((k >> 1) & 1));
            mbar_wait_bounded(&bar[(k + 1) & 1], (unsigned)(((k + 1) >> 1) & 1));
        }
        __syncthreads();
    }
}

// shared memory of one block: barriers + two stages
template <class L, class S> inline size_t stage_smem(int seg) {
    const int W = seg + 2 * (16 / (int)sizeof(S));
    return 128 + 2 * (size_t)L::Q * W * sizeof(S);
}

// rows 16-byte aligned, and at least one full warp per block (warp 0 issues
// the copies)
template <class L, class P> inline bool staged_ok(const Params &p) {
    using S = typename P::S;
    return !P::exact && !p.zouhe && ((size_t)p.nx * sizeof(S)) % 16 == 0 && p.nx >= 32;
}

} // namespace lbm
