// lbm_launch.cuh -- typed launchers of the step kernels; included by the
// precision translation units (lbm_fp64.cu, lbm_fp32.cu).
#pragma once

#include <algorithm>

#include "lbm_internal.h"
#include "lbm_pair.cuh"
#include "lbm_stage.cuh"

namespace lbm {

inline dim3 bulk_block(const Params &p) {
    int bx = BULK_THREADS;
    while (bx > 32 && bx / 2 >= p.nx) bx /= 2;
    return dim3(bx, 1, 1);
}

inline dim3 bulk_grid(const Params &p) {
    dim3 b = bulk_block(p);
    return dim3((p.nx + b.x - 1) / b.x, p.ny, p.nz);
}

template <class L, class P>
cudaError_t init_t(const Params &p, void *dst, void *mac, const uint8_t *flags, const double u0[3], cudaStream_t s) {
    k_init<L, P><<<bulk_grid(p), bulk_block(p), 0, s>>>(p, (typename P::S *)dst, (typename P::C *)mac, flags, u0[0],
                                                         u0[1], u0[2]);
    return cudaGetLastError();
}

template <class L, class P>
cudaError_t load_t(const Params &p, const double *stage, long long c0, long long n, void *dst, void *mac,
                   const uint8_t *flags, cudaStream_t s) {
    const unsigned grid = (unsigned)((n + BULK_THREADS - 1) / BULK_THREADS);
    k_load<L, P><<<grid, BULK_THREADS, 0, s>>>(p, stage, c0, n, (typename P::S *)dst, (typename P::C *)mac, flags);
    return cudaGetLastError();
}

template <class L, class P>
cudaError_t macros_t(const Params &p, const void *src, const uint16_t *owner, long long c0, long long n, double *out,
                     cudaStream_t s) {
    const unsigned grid = (unsigned)((n + BULK_THREADS - 1) / BULK_THREADS);
    k_macros<L, P><<<grid, BULK_THREADS, 0, s>>>(p, (const typename P::S *)src, owner, c0, n, out);
    return cudaGetLastError();
}

template <class L, class P> cudaError_t links_t(const Params &p, const StepBufs &sb, int grid, cudaStream_t s) {
    if (p.nb == 0 || grid <= 0) return cudaSuccess;
    k_links<L, P><<<grid, LINK_THREADS, 0, s>>>(p, sb);
    return cudaGetLastError();
}

// reduced precision with 16-byte aligned rows: rows staged by bulk copies
template <class L, class P> void staged_launch(const Params &p, const StepBufs &sb, cudaStream_t s) {
    using S = typename P::S;
    const int seg = std::min(STAGE_SEG, p.nx);
    const long long nseg = (long long)((p.nx + seg - 1) / seg) * p.ny * p.nz;
    const int grid = (int)std::min<long long>(nseg, (long long)std::max(1, p.nsm) * STAGE_BLOCKS_PER_SM);
    k_bulk_staged<L, P><<<grid, seg, stage_smem<L, S>(seg), s>>>(p, (const S *)sb.src, (S *)sb.dst, sb.flags,
                                                                  sb.counters, (float *)sb.mac_t1);
}

// one kernel per face mode: the fewer faces, the less code in the loop
template <class L, class P> cudaError_t bulk_t(const Params &p, const StepBufs &sb, cudaStream_t s) {
    if constexpr (!P::exact) {
        if (p.staged && staged_ok<L, P>(p)) {
            staged_launch<L, P>(p, sb, s);
            return cudaGetLastError();
        }
    }
    const int fm = face_mode(p);
    const typename P::S *src = (const typename P::S *)sb.src;
    typename P::S *dst = (typename P::S *)sb.dst;
    const typename P::C *mt = (const typename P::C *)sb.mac_t;
    typename P::C *mt1 = (typename P::C *)sb.mac_t1;
    bool pair = false;
    if constexpr (!P::exact) pair = p.pair && pair_ok(p, fm);
    if (pair) {
        if constexpr (!P::exact) k_bulk_pair<L, P><<<pair_grid(p), pair_block(p), 0, s>>>(p, src, dst, sb.flags, mt1);
    } else if (fm == FM_PERIODIC)
        k_bulk<L, P, FM_PERIODIC><<<bulk_grid(p), bulk_block(p), 0, s>>>(p, src, dst, sb.flags, mt, mt1);
    else if (fm == FM_XFACES)
        k_bulk<L, P, FM_XFACES><<<bulk_grid(p), bulk_block(p), 0, s>>>(p, src, dst, sb.flags, mt, mt1);
    else
        k_bulk<L, P, FM_GENERAL><<<bulk_grid(p), bulk_block(p), 0, s>>>(p, src, dst, sb.flags, mt, mt1);
    if (p.zouhe) { // the Zou-He face nodes, which the bulk kernel skipped
        long long plane = 0;
        const long long n[3] = {p.nx, p.ny, p.nz};
        for (int a = 0; a < 3; ++a) plane = std::max(plane, n[(a + 1) % 3] * n[(a + 2) % 3]);
        const dim3 grid((unsigned)((plane + BULK_THREADS - 1) / BULK_THREADS), 1, 6);
        k_zouhe<L, P><<<grid, BULK_THREADS, 0, s>>>(p, src, dst, sb.flags, mt, mt1);
    }
    return cudaGetLastError();
}

template <class L, class P> cudaError_t finish_t(const Params &p, const StepBufs &sb, cudaStream_t s) {
    const int grid = p.nb + sb.n_moving;
    if (grid == 0) return cudaSuccess;
    k_finish<L, P><<<grid, IMP_THREADS, 0, s>>>(p, sb);
    return cudaGetLastError();
}

} // namespace lbm
