// lbm_pair.cuh -- reduced-precision stream-collide with two nodes per thread.
//
// A thread takes the nodes (x, y, z) and (x + 1, y, z), x even.  Per
// direction the two populations travel as one pair (half2 or float2): one
// address, one load and one store serve both nodes.  The pull of a direction
// with c_x = +-1 needs the pair shifted by one node; the missing element comes
// from the neighbouring lane's pair (a warp shuffle), the lanes at the ends of
// the warp load it.  The arithmetic runs on Blackwell's paired FP32
// instructions (add / sub / mul / fma .f32x2, round to nearest), one pair
// operation per operation of moments_f / collide_f; every lane follows the
// single-node code's operation sequence, so both kernels give the same values.
// The opposite direction o = opp(i) of a pair (i, o) uses c_o . u = -c_i . u
// exactly (round to nearest is odd-symmetric), so its polynomial
// 3 cu + 4.5 cu^2 - 1.5 u^2 at -cu is the negated fma chain
// -(cu (3 - 4.5 cu) + 1.5 u^2), also exact.
//
// Used for fully periodic domains without a body force whose x extent is
// even.
#pragma once

#include "lbm_step.cuh"

namespace lbm {

constexpr int PAIR_THREADS = 128;

// two FP32 lanes in one 64-bit register pair
struct F2 {
    unsigned long long v;
};

// lane 0 in the low 32 bits (plain integer packing: the compiler pairs the
// registers itself)
__device__ __forceinline__ F2 f2(float a, float b) {
    F2 r;
    r.v = ((unsigned long long)__float_as_uint(b) << 32) | (unsigned long long)__float_as_uint(a);
    return r;
}
__device__ __forceinline__ F2 f2s(float a) { return f2(a, a); }
__device__ __forceinline__ float2 unf2(F2 x) {
    return make_float2(__uint_as_float((unsigned)(x.v & 0xffffffffull)), __uint_as_float((unsigned)(x.v >> 32)));
}
__device__ __forceinline__ F2 vadd(F2 a, F2 b) {
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 vsub(F2 a, F2 b) {
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 vmul(F2 a, F2 b) {
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) {
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

// moments_f (no body force) lane by lane
template <class L>
__device__ __forceinline__ void moments_pair(const Params &p, const F2 f[], F2 &drho, F2 u[3]) {
    const F2 zero = f2s(0.0f);
    F2 r = zero, j0 = zero, j1 = zero, j2 = zero;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const F2 fi = f[i];
        r = vadd(r, fi);
        if (L::cx(i) == 1) j0 = vadd(j0, fi);
        if (L::cx(i) == -1) j0 = vsub(j0, fi);
        if (L::cy(i) == 1) j1 = vadd(j1, fi);
        if (L::cy(i) == -1) j1 = vsub(j1, fi);
        if (L::cz(i) == 1) j2 = vadd(j2, fi);
        if (L::cz(i) == -1) j2 = vsub(j2, fi);
    }
    F2 inv;
    if (p.eq == 0) {
        inv = f2s(p.inv_rho0f);
    } else {
        const float2 rr = unf2(r);
        inv = f2(1.0f / (1.0f + rr.x), 1.0f / (1.0f + rr.y));
    }
    drho = r;
    u[0] = vmul(j0, inv);
    u[1] = vmul(j1, inv);
    u[2] = vmul(j2, inv);
}

// c_i . u of a direction whose first non-zero component is +1, or (D2Q9's
// (-1, 1)) -1 followed by +1: the value cdot_f gives
template <class L> __device__ __forceinline__ F2 cdot_pair(int i, const F2 u[3]) {
    const int c[3] = {L::cx(i), L::cy(i), L::cz(i)};
    int a = -1, b = -1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (c[k] == 0) continue;
        if (a < 0) a = k;
        else b = k;
    }
    if (b < 0) return c[a] > 0 ? u[a] : vsub(f2s(0.0f), u[a]); // (the second form is not reached)
    if (c[a] > 0) return c[b] > 0 ? vadd(u[a], u[b]) : vsub(u[a], u[b]);
    return vsub(u[b], u[a]); // -u_a + u_b
}

// collide_f (no body force) lane by lane
template <class L> __device__ __forceinline__ void collide_pair(const Params &p, F2 f[], F2 drho, const F2 u[3]) {
    const F2 om = f2s(p.omegaf);
    const F2 s = vfma(u[0], u[0], vfma(u[1], u[1], vmul(u[2], u[2])));
    const F2 usq15 = vmul(f2s(1.5f), s), nusq15 = vmul(f2s(-1.5f), s);
    const F2 rr = p.eq == 0 ? f2s(p.rho0f) : vadd(f2s(1.0f), drho);
    const F2 omr = vmul(om, rr), omd = vmul(om, drho);
    const F2 keep = f2s(p.keepf);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int o = L::opp(i);
        if (o < i) continue; // relaxed with its partner
        const float w = L::template w<float>(i);
        const F2 wr = vmul(f2s(w), omr), wd = vmul(f2s(w), omd);
        if (i == 0) { // rest: c . u = 0
            const F2 poly = vfma(f2s(0.0f), f2s(3.0f), nusq15);
            f[0] = vfma(keep, f[0], vfma(wr, poly, wd));
            continue;
        }
        const F2 cu = cdot_pair<L>(i, u);
        const F2 poly = vfma(cu, vfma(f2s(4.5f), cu, f2s(3.0f)), nusq15);
        f[i] = vfma(keep, f[i], vfma(wr, poly, wd));
        const F2 nwr = vmul(f2s(-w), omr);
        const F2 pn = vfma(cu, vfma(f2s(-4.5f), cu, f2s(3.0f)), usq15); // -(poly at -cu)
        f[o] = vfma(keep, f[o], vfma(nwr, pn, wd));
    }
}

// storage pairs: 32 bits of two halves, or a float2
template <class S> struct Pair;
template <> struct Pair<__half> {
    using T = unsigned;
    static __device__ __forceinline__ T ld(const __half *p) { return __ldg(reinterpret_cast<const unsigned *>(p)); }
    static __device__ __forceinline__ F2 cvt(T v) {
        __half2 h;
        memcpy(&h, &v, sizeof(h));
        const float2 f = __half22float2(h);
        return f2(f.x, f.y);
    }
    // (element 1 of a, element 0 of b)
    static __device__ __forceinline__ T mid(T a, T b) { return __byte_perm(a, b, 0x5432); }
    // the pair of the lane below / above (the element mid() uses)
    static __device__ __forceinline__ T from_below(T own) { return __shfl_up_sync(0xffffffffu, own, 1); }
    static __device__ __forceinline__ T from_above(T own) { return __shfl_down_sync(0xffffffffu, own, 1); }
    static __device__ __forceinline__ void st(__half *p, F2 v) {
        const float2 f = unf2(v);
        const __half2 h = __floats2half2_rn(f.x, f.y);
        unsigned u;
        memcpy(&u, &h, sizeof(u));
        *reinterpret_cast<unsigned *>(p) = u;
    }
};
template <> struct Pair<float> {
    using T = float2;
    static __device__ __forceinline__ T ld(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
    static __device__ __forceinline__ F2 cvt(T v) { return f2(v.x, v.y); }
    static __device__ __forceinline__ T mid(T a, T b) { return make_float2(a.y, b.x); }
    static __device__ __forceinline__ T from_below(T own) {
        return make_float2(0.0f, __shfl_up_sync(0xffffffffu, own.y, 1));
    }
    static __device__ __forceinline__ T from_above(T own) {
        return make_float2(__shfl_down_sync(0xffffffffu, own.x, 1), 0.0f);
    }
    static __device__ __forceinline__ void st(float *p, F2 v) {
        const float2 f = unf2(v);
        *reinterpret_cast<float2 *>(p) = f;
    }
};

// The nodes (x0, y, z) and (x0 + 1, y, z) of the calling thread (x0 even, nx
// even, every axis periodic); all 32 lanes of the warp call it for the same
// row, lanes past the row with x0 >= nx.
template <class L, class P>
__device__ __forceinline__ void pair_nodes(const Params &p, const typename P::S *__restrict__ src,
                                           typename P::S *__restrict__ dst, const uint8_t *__restrict__ flags,
                                           typename P::C *__restrict__ mac_t1, int x0, int y, int z) {
    using S = typename P::S;
    using PT = Pair<S>;
    using T = typename PT::T;
    const int lane = threadIdx.x & 31;
    const int nx = p.nx;
    const bool valid = x0 < nx;
    const int xc = valid ? x0 : nx - 2; // lanes past the row load in bounds, store nothing
    const unsigned ny = (unsigned)p.ny, N32 = (unsigned)p.N;
    const unsigned cell0 = ((unsigned)z * ny + (unsigned)y) * (unsigned)nx + (unsigned)xc;
    const unsigned fl2 = __ldg(reinterpret_cast<const unsigned short *>(flags + cell0));
    const unsigned fl0 = fl2 & 0xffu, fl1 = fl2 >> 8;
    const uint8_t skip = FL_SOLID | (p.linkmode ? 0 : FL_BND);
    // (the pulls do not wait for the flags: a pair with no node to store is
    // stepped all the same, so the flag load overlaps the population loads)
    const bool act0 = valid && !(fl0 & skip), act1 = valid && !(fl1 & skip);
    const int ym = y == 0 ? p.ny - 1 : y - 1, yp = y == p.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? p.nz - 1 : z - 1, zp = z == p.nz - 1 ? 0 : z + 1;
    // the element left of x0 (lane 0) and the pair right of x0 + 1 (lane 31,
    // or the row's last pair): periodic along x where these are used
    const int xl = (x0 == 0 ? nx : x0) - 2; // pair holding x0 - 1 as element 1
    const int xr = x0 + 2 >= nx ? 0 : x0 + 2;
    const bool ld_l = lane == 0, ld_r = lane == 31 || x0 + 2 >= nx;
    F2 f[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int sy = L::cy(i) == 1 ? ym : (L::cy(i) == -1 ? yp : y);
        const int sz = L::cz(i) == 1 ? zm : (L::cz(i) == -1 ? zp : z);
        const S *row = src + (size_t)N32 * (unsigned)i + ((unsigned)sz * ny + (unsigned)sy) * (unsigned)nx;
        const T own = PT::ld(row + xc);
        T v = own;
        if (L::cx(i) == 1) { // sources x0 - 1, x0
            T left = PT::from_below(own);
            if (ld_l) left = PT::ld(row + xl);
            v = PT::mid(left, own);
        } else if (L::cx(i) == -1) { // sources x0 + 1, x0 + 2
            T right = PT::from_above(own);
            if (ld_r) right = PT::ld(row + xr);
            v = PT::mid(own, right);
        }
        f[i] = PT::cvt(v);
    }
    F2 drho, u[3];
    moments_pair<L>(p, f, drho, u);
    if (p.linkmode && ((act0 && (fl0 & FL_MAC)) || (act1 && (fl1 & FL_MAC)))) {
        const float2 d = unf2(drho), u0 = unf2(u[0]), u1 = unf2(u[1]), u2 = unf2(u[2]);
        if (act0 && (fl0 & FL_MAC)) {
            const float uu[3] = {u0.x, u1.x, u2.x};
            store_mac((float *)mac_t1, cell0, d.x, uu);
        }
        if (act1 && (fl1 & FL_MAC)) {
            const float uu[3] = {u0.y, u1.y, u2.y};
            store_mac((float *)mac_t1, cell0 + 1, d.y, uu);
        }
    }
    collide_pair<L>(p, f, drho, u);
    if (act0 && act1) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) PT::st(dst + (size_t)N32 * (unsigned)i + cell0, f[i]);
    } else if (act0 || act1) { // one node of the pair is solid (or a boundary node): store the other
        const unsigned c = act0 ? cell0 : cell0 + 1;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const float2 e = unf2(f[i]);
            stS(dst + (size_t)N32 * (unsigned)i + c, act0 ? e.x : e.y);
        }
    }
}

// resident blocks of PAIR_THREADS the two-node kernel is built for: 8 (64
// registers) with FP16 storage, 7 with FP32 (its float2 pairs need 68
// registers to run without spills)
template <class P> constexpr int pair_min_blocks() { return sizeof(typename P::S) == 2 ? 8 : 7; }

// every thread a pair of one row: blockIdx.y = y, blockIdx.z = z
template <class L, class P>
__global__ void __launch_bounds__(PAIR_THREADS, pair_min_blocks<P>()) k_bulk_pair(Params p, const typename P::S *__restrict__ src,
                                                            typename P::S *__restrict__ dst,
                                                            const uint8_t *__restrict__ flags,
                                                            typename P::C *__restrict__ mac_t1) {
    pair_nodes<L, P>(p, src, dst, flags, mac_t1, 2 * (blockIdx.x * blockDim.x + threadIdx.x), blockIdx.y, blockIdx.z);
}

// the pair kernel's conditions: no body force, nx even, every axis periodic,
// reduced precision.  (Where faces cut the rows, the face rules of the
// single-node kernel measured faster than two-node rows with face lanes.)
inline bool pair_ok(const Params &p, int fm) { return !p.has_force && p.nx % 2 == 0 && p.nx >= 4 && fm == FM_PERIODIC; }

inline dim3 pair_block(const Params &p) {
    int bx = PAIR_THREADS;
    while (bx > 32 && bx / 2 >= p.nx / 2) bx /= 2;
    return dim3(bx, 1, 1);
}

inline dim3 pair_grid(const Params &p) {
    const dim3 b = pair_block(p);
    return dim3((p.nx / 2 + b.x - 1) / b.x, p.ny, p.nz);
}

} // namespace lbm
