// lbm_dev.cuh -- device-side definitions shared by the kernels of liblbm.
//
// Lattice traits (D2Q9 / D3Q19 in the library's direction order), precision
// policies, the POD parameter blocks passed to every kernel, and the FP64
// geometry helpers (pose, minimum image, rigid-body velocity, fractional link
// distance Delta of Sec. 2.1).
//
// Every translation unit of the library is compiled with --fmad=false: the
// FP64 mode must reproduce the fixed operation order of each formula exactly,
// so no multiply-add may be contracted behind our back.  The FP32 path asks
// for fused multiply-adds explicitly with fmaf().
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace lbm {

constexpr uint8_t FL_SOLID = 1; // node inside a body at time t
constexpr uint8_t FL_MAC = 2;   // store rho,u of f(t+1) at this node (FP64 mode)
constexpr uint8_t FL_BND = 4;   // fluid node with a solid neighbour at t (handled by
                                // the boundary-node kernel in the reduced-precision modes)

constexpr int SERIES_ROW = 18;  // Fs Ts Fi Ti Fm Tm
constexpr int ME_PER_LINK = 12; // Fs Ts Fm Tm contributions of one link
constexpr int GEOM_THREADS = 512;
constexpr int GEOM_CELLS = 8; // consecutive region cells per thread
constexpr int GEOM_CHUNK = GEOM_THREADS * GEOM_CELLS;
constexpr int REGION_MARGIN = 4;
// link mode: moments are kept at fluid nodes within R + MAC_BAND of a body
// (a cut link's fluid end and its x_F + c_i lie within 2 sqrt(2) of the
// surface; a body moves less than a quarter cell per step; the region of a
// body reaches R + REGION_MARGIN)
constexpr float MAC_BAND = 4.0f;

// ---------------------------------------------------------------- lattices --
template <int Q_> struct Lat;

template <> struct Lat<9> {
    static constexpr int Q = 9, D = 2;
    __host__ __device__ static constexpr int cx(int i) {
        return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cy(int i) {
        return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
    }
    template <class T> __host__ __device__ static constexpr T w(int i) {
        return i == 0 ? T(4) / T(9) : (i <= 4 ? T(1) / T(9) : T(1) / T(36));
    }
};

template <> struct Lat<19> {
    static constexpr int Q = 19, D = 3;
    // 0 rest; 1..6 +-x +-y +-z; 7..18 face diagonals in opposite pairs
    __host__ __device__ static constexpr int cx(int i) {
        return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
             : ((i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cy(int i) {
        return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
             : ((i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cz(int i) {
        return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
             : ((i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0);
    }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : ((i % 2) == 1 ? i + 1 : i - 1);
    }
    template <class T> __host__ __device__ static constexpr T w(int i) {
        return i == 0 ? T(1) / T(3) : (i <= 6 ? T(1) / T(18) : T(1) / T(36));
    }
};

// run-time indexed copies of the tables (for kernels that walk link lists)
struct LatTab {
    int8_t c[19][3];
    int8_t opp[19];
    double w[19];
};

template <class L> __host__ __device__ inline LatTab make_tab() {
    LatTab t{};
    for (int i = 0; i < L::Q; ++i) {
        t.c[i][0] = (int8_t)L::cx(i);
        t.c[i][1] = (int8_t)L::cy(i);
        t.c[i][2] = (int8_t)L::cz(i);
        t.opp[i] = (int8_t)L::opp(i);
        t.w[i] = L::template w<double>(i);
    }
    return t;
}

// ------------------------------------------------------- precision policies --
struct PF64 { // FP64 arithmetic, FP64 storage of f (no shift)
    using S = double;
    using C = double;
    static constexpr bool exact = true;
};
struct PF32 { // FP32 arithmetic, storage of f - w in FP32
    using S = float;
    using C = float;
    static constexpr bool exact = false;
};
struct PF16 { // FP32 arithmetic, storage of f - w in FP16
    using S = __half;
    using C = float;
    static constexpr bool exact = false;
};

__device__ __forceinline__ double ldS(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ldS(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ldS(const __half *p) { return __half2float(__ldg(p)); }
// plain loads for buffers written earlier in the same kernel's lifetime
__device__ __forceinline__ double ldP(const double *p) { return *p; }
__device__ __forceinline__ float ldP(const float *p) { return *p; }
__device__ __forceinline__ float ldP(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ void stS(double *p, double v) { *p = v; }
__device__ __forceinline__ void stS(float *p, float v) { *p = v; }
__device__ __forceinline__ void stS(__half *p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ float roundS(const __half *, float v) { return __half2float(__float2half_rn(v)); }
__device__ __forceinline__ float roundS(const float *, float v) { return v; }
__device__ __forceinline__ double roundS(const double *, double v) { return v; }

// ------------------------------------------------------------ kernel params --
struct Params {
    int nx, ny, nz;
    int per[3];  // periodic axes
    int edge[6]; // x-lo x-hi y-lo y-hi z-lo z-hi
    long long N; // nx*ny*nz
    int eq;      // 0 quasi-incompressible, 1 standard
    int inlet_parabolic;
    int has_force;
    int refill;
    int nb;      // bodies
    int nonper;  // 1 if any axis is non-periodic
    int exact;   // FP64 mode: link geometry in FP64 (else FP32)
    int staged;  // reduced precision: stream-collide from rows staged in shared memory
    int pair;    // reduced precision: two nodes per thread where that kernel applies
    int stage_expire_test; // test hook: the staged kernel issues no copy, so its waits expire
    int nsm;     // multiprocessors of the device
    int zouhe;   // wall / inlet faces are Zou-He nodes (else half-way links)
    int free_scheme; // covered / uncovered sets of free bodies: 0 explicit, 1 backward sets
                     // of the previous displacement, 2 predictor-corrector
    int linkmode; // reduced precision, single domain: wall values on cut links are written
                  // into the solid nodes' slots before the stream-collide pass (which then
                  // steps the boundary nodes too); the moments (drho, u) of the nodes near
                  // bodies are kept as float4 per cell (FL_MAC).  0: the boundary-node kernel
                  // steps the boundary nodes (serving batches)
    long long series_cap;
    long long me_stride; // ME contribution arrays are [ME_PER_LINK][me_stride]
    double tau, omega, rho0, u_in;
    double g[3];
    double gravity[3]; // acceleration of the free bodies
    float omegaf, rho0f, u_inf;
    float inv_rho0f;  // 1 / rho0f (correctly rounded, as the device division)
    float keepf;      // 1 - omegaf
    float gf[3];
};

struct BodyDev {
    int shape;   // 0 cylinder (x-y disc), 1 sphere
    int halfway; // Delta = 1/2 on every link
    int moving;  // U or W non-zero
    int nchunks; // geometry chunks of its region
    double R;
    double X0[3], U[3], W[3];
    long long t0;
    long long link_off, link_cap; // segment in the link arrays
    long long apm_off, apm_cap;   // segment in the covered/uncovered list
    int ext[3];                   // region extents (cells) per axis
    int chunk_base;               // first geometry chunk of this body
    int free;                     // moved by the flow force and torque (Newton-Euler)
    double density_ratio;         // free bodies: body density / rho0
    double R2;                    // ellipse: second semi-axis (R is the first, R >= R2)
    double theta0;                // ellipse: orientation about z at step t0
};

// shape codes: 0 cylinder (x-y disc, along z), 1 sphere, 2 ellipse (x-y, along z)
__host__ __device__ inline bool along_z(int shape) { return shape != 1; }

// orientation about z at step t: theta(t) = theta0 + (t - t0) W_z
__device__ __forceinline__ double orient(const BodyDev &b, long long t) {
    double dt = (double)(t - b.t0);
    return b.theta0 + dt * b.W[2];
}

// sin and cos by the Cody-Waite reduction (Cody & Waite, "Software Manual for
// the Elementary Functions", 1980): k = nearest integer to x 2/pi, r = x - k pi/2
// with pi/2 in three parts (the first two of 33 significant bits, so k P1 and
// k P2 are exact for |k| < 2^20), Taylor series of sin and cos on |r| <= pi/4
// to r^19 / r^18 in Horner form, then the quadrant.  The same formula is
// evaluated everywhere so that orientations agree bit for bit.
__device__ __forceinline__ void sincos_cw(double x, double &s_out, double &c_out) {
    const double P1 = 0x1.921fb544p+0;
    const double P2 = 0x1.0b4611a6p-34;
    const double P3 = 0x1.3198a2e037073p-69;
    const double kf = nearbyint(x * 0.6366197723675814);
    const double r = ((x - kf * P1) - kf * P2) - kf * P3;
    const double r2 = r * r;
    double ps = 8.22063524662433e-18;
    ps = ps * r2 - 2.8114572543455206e-15;
    ps = ps * r2 + 7.647163731819816e-13;
    ps = ps * r2 - 1.6059043836821613e-10;
    ps = ps * r2 + 2.505210838544172e-08;
    ps = ps * r2 - 2.7557319223985893e-06;
    ps = ps * r2 + 0.0001984126984126984;
    ps = ps * r2 - 0.008333333333333333;
    ps = ps * r2 + 0.16666666666666666;
    const double sr = r - r * r2 * ps;
    double pc = 1.5619206968586225e-16;
    pc = pc * r2 - 4.779477332387385e-14;
    pc = pc * r2 + 1.1470745597729725e-11;
    pc = pc * r2 - 2.08767569878681e-09;
    pc = pc * r2 + 2.755731922398589e-07;
    pc = pc * r2 - 2.48015873015873e-05;
    pc = pc * r2 + 0.001388888888888889;
    pc = pc * r2 - 0.041666666666666664;
    pc = pc * r2 + 0.5;
    const double cr = 1.0 - r2 * pc;
    const long long q = (long long)kf & 3;
    if (q == 0) {
        s_out = sr;
        c_out = cr;
    } else if (q == 1) {
        s_out = cr;
        c_out = -sr;
    } else if (q == 2) {
        s_out = -sr;
        c_out = -cr;
    } else {
        s_out = -cr;
        c_out = sr;
    }
}

// ------------------------------------------------------- FP64 geometry ------
// These follow one fixed expression each; they are shared by all precision
// modes so the solid set and link distances never depend on the mode.
__device__ __forceinline__ void pose(const BodyDev &b, long long t, double X[3]) {
    double dt = (double)(t - b.t0);
    for (int k = 0; k < 3; ++k) X[k] = b.X0[k] + dt * b.U[k];
}

__device__ __forceinline__ int axis_len(const Params &p, int a) { return a == 0 ? p.nx : (a == 1 ? p.ny : p.nz); }

// pose brought into [0, L) on periodic axes (one division per body and step)
__device__ __forceinline__ void wrap_pose(const Params &p, const double X[3], double Xw[3]) {
    for (int a = 0; a < 3; ++a) {
        if (!p.per[a]) {
            Xw[a] = X[a];
            continue;
        }
        double L = (double)axis_len(p, a);
        Xw[a] = X[a] - L * floor(X[a] / L);
    }
}

// minimum-image displacement along one axis from the unwrapped pose X
// (reading of the torque reference, Eq. H of Sec. 3): v = x - X, then on a
// periodic axis v - L floor(v / L + 1/2) -- the oracle's expression, each
// operation rounded explicitly so that no unit's contraction flags change it
__device__ __forceinline__ double axis_disp(const Params &p, int a, double x, double X) {
    const double v = __dsub_rn(x, X);
    if (!p.per[a]) return v;
    const double L = (double)axis_len(p, a);
    return __dsub_rn(v, __dmul_rn(L, floor(__dadd_rn(__ddiv_rn(v, L), 0.5))));
}

// displacement of node (x, y, z) from the unwrapped pose X
__device__ __forceinline__ void disp_from(const Params &p, const double X[3], int x, int y, int z, double r[3]) {
    r[0] = axis_disp(p, 0, (double)x, X[0]);
    r[1] = axis_disp(p, 1, (double)y, X[1]);
    r[2] = axis_disp(p, 2, (double)z, X[2]);
}

// the same from Pw, the wrapped pose of t or t+1 inside a pose record: the
// unwrapped pose of that time sits three entries before it (POSE_STRIDE
// layout below)
__device__ __forceinline__ void disp(const Params &p, const double *Pw, int x, int y, int z, double r[3]) {
    disp_from(p, Pw - 3, x, y, z, r);
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ void body_velocity(const BodyDev &b, const double r[3], double v[3]) {
    double wr[3];
    cross3(b.W, r, wr);
    for (int k = 0; k < 3; ++k) v[k] = b.U[k] + wr[k];
}

// coordinates of an offset in an ellipse's own axes (orientation co, si)
__device__ __forceinline__ void body_axes(double co, double si, double v0, double v1, double &xi, double &eta) {
    xi = co * v0 + si * v1;
    eta = co * v1 - si * v0;
}

// r: offset from the centre; co, si: cos and sin of the orientation (ellipse)
__device__ __forceinline__ bool inside(const BodyDev &b, const double r[3], double co, double si) {
    if (b.shape == 2) {
        double xi, eta;
        body_axes(co, si, r[0], r[1], xi, eta);
        const double qx = xi / b.R, qy = eta / b.R2;
        return qx * qx + qy * qy <= 1.0;
    }
    double s = r[0] * r[0] + r[1] * r[1];
    if (b.shape == 1) s = s + r[2] * r[2];
    return s <= b.R * b.R;
}

// Delta of Sec. 2.1: root s in (0,1] of |d - s c|^2 = R^2 (x_F outside); for
// an ellipse the same quadratic in the scaled body axes
__device__ __forceinline__ double link_delta(const BodyDev &b, const double d[3], int cxi, int cyi, int czi,
                                             double co, double si) {
    if (b.halfway) return 0.5;
    double cx = cxi, cy = cyi, cz = czi;
    double a, bb, cc;
    if (b.shape == 2) {
        double dx, dy, kx, ky;
        body_axes(co, si, d[0], d[1], dx, dy);
        body_axes(co, si, cx, cy, kx, ky);
        dx = dx / b.R;
        dy = dy / b.R2;
        kx = kx / b.R;
        ky = ky / b.R2;
        a = kx * kx + ky * ky;
        bb = dx * kx + dy * ky;
        cc = (dx * dx + dy * dy) - 1.0;
    } else if (b.shape == 1) {
        a = cx * cx + cy * cy + cz * cz;
        bb = d[0] * cx + d[1] * cy + d[2] * cz;
        cc = (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - b.R * b.R;
    } else {
        a = cx * cx + cy * cy;
        bb = d[0] * cx + d[1] * cy;
        cc = (d[0] * d[0] + d[1] * d[1]) - b.R * b.R;
    }
    (void)a;
    double disc = bb * bb - a * cc;
    if (disc < 0.0) disc = 0.0;
    double s = cc / (bb + sqrt(disc));
    if (s > 1.0) s = 1.0;
    if (s < 0.0) s = 0.0;
    return s;
}

// FP32 link distance (reduced-precision modes): same formula as link_delta
__device__ __forceinline__ float link_delta_f(int halfway, int shape, float R, float R2, float co, float si,
                                              const float d[3], int cxi, int cyi, int czi) {
    if (halfway) return 0.5f;
    float cx = cxi, cy = cyi, cz = czi;
    float a, bb, cc;
    if (shape == 2) {
        float dx = (co * d[0] + si * d[1]) / R, dy = (co * d[1] - si * d[0]) / R2;
        float kx = (co * cx + si * cy) / R, ky = (co * cy - si * cx) / R2;
        a = kx * kx + ky * ky;
        bb = dx * kx + dy * ky;
        cc = (dx * dx + dy * dy) - 1.0f;
    } else if (shape == 1) {
        a = cx * cx + cy * cy + cz * cz;
        bb = d[0] * cx + d[1] * cy + d[2] * cz;
        cc = (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - R * R;
    } else {
        a = cx * cx + cy * cy;
        bb = d[0] * cx + d[1] * cy;
        cc = (d[0] * d[0] + d[1] * d[1]) - R * R;
    }
    float disc = bb * bb - a * cc;
    if (disc < 0.0f) disc = 0.0f;
    float sres = cc / (bb + sqrtf(disc));
    return fminf(fmaxf(sres, 0.0f), 1.0f);
}

// Body frame of one step for fast node classification: integer part and FP32
// fraction of the wrapped pose.  Node displacements are k - fr with k an
// integer (minimum image taken on k), accurate to ~1e-6 cells.
struct Frame {
    int xi[3];
    float fr[3];
    double X[3]; // unwrapped pose (the displacement of the FP64 decision)
    double co, si;   // orientation (ellipse)
    float cof, sif;
};

// Xw points at the wrapped pose of t or t+1 in a poses record; the matching
// orientation (cos, sin) sits 15 entries further, the unwrapped pose three
// entries before it (see POSE_STRIDE)
__device__ __forceinline__ void make_frame(const double Xw[3], Frame &f) {
    for (int a = 0; a < 3; ++a) {
        double fl = floor(Xw[a]);
        f.xi[a] = (int)fl;
        f.fr[a] = (float)(Xw[a] - fl);
        f.X[a] = Xw[a - 3];
    }
    f.co = Xw[15];
    f.si = Xw[16];
    f.cof = (float)f.co;
    f.sif = (float)f.si;
}

// FP32 displacement k - fr of a node from a body frame along one axis (k =
// node - floor(pose), fr = pose - floor(pose) in [0, 1)).  On a periodic axis
// of n nodes it is the minimum image in [-n/2, n/2), with the tie at exactly
// n/2 taken as -n/2: the FP64 minimum image v - n floor(v / n + 1/2) of
// axis_disp, decided from the integer k and fr so that the choice is exact.
__device__ __forceinline__ float frame_axis(int k, float fr, int n, int per) {
    if (per) {
        if (2 * k > n) k -= n;
        else if (2 * k < -n) k += n;
        // k - fr now lies in [-n/2 - 1, n/2]: bring its ends into [-n/2, n/2)
        if ((float)(2 * k - n) >= 2.0f * fr) k -= n;
        else if ((float)(2 * k + n) < 2.0f * fr) k += n;
    }
    return (float)k - fr;
}

__device__ __forceinline__ void frame_disp_f(const Params &p, const Frame &f, int x, int y, int z, float d[3]) {
    const int c[3] = {x, y, z};
    for (int a = 0; a < 3; ++a) {
        const int n = a == 0 ? p.nx : (a == 1 ? p.ny : p.nz);
        d[a] = frame_axis(c[a] - f.xi[a], f.fr[a], n, p.per[a]);
    }
}

// Inside test with the exact FP64 decision: FP32 decides unless the node is
// within a thin band around the surface, where the FP64 test of `inside`
// (the one the oracle uses) is evaluated.
__device__ __forceinline__ bool inside_screened(const Params &p, const BodyDev &B, const Frame &f, int x, int y,
                                                int z) {
    float d[3];
    frame_disp_f(p, f, x, y, z, d);
    float s, R2;
    if (B.shape == 2) { // scaled to the first semi-axis: the unit ellipse times R^2
        const float xi = f.cof * d[0] + f.sif * d[1], eta = f.cof * d[1] - f.sif * d[0];
        const float k = (float)(B.R / B.R2);
        s = xi * xi + (k * eta) * (k * eta);
        R2 = (float)(B.R * B.R);
        const float band = (1e-4f * R2 + 0.05f) * k * k;
        if (s < R2 - band) return true;
        if (s > R2 + band) return false;
    } else {
        s = d[0] * d[0] + d[1] * d[1];
        if (B.shape == 1) s += d[2] * d[2];
        R2 = (float)(B.R * B.R);
        const float band = 1e-4f * R2 + 0.05f;
        if (s < R2 - band) return true;
        if (s > R2 + band) return false;
    }
    double r[3];
    disp_from(p, f.X, x, y, z, r);
    return inside(B, r, f.co, f.si);
}

// radial band of the surface: inner and outer radius (the semi-axes of an ellipse)
__device__ __forceinline__ float body_rin(const BodyDev &B) { return (float)(B.shape == 2 ? B.R2 : B.R); }
__device__ __forceinline__ float body_rout(const BodyDev &B) { return (float)B.R; }

__device__ __forceinline__ int wrap_axis(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ long long cell_of(const Params &p, int x, int y, int z) {
    return ((long long)z * p.ny + y) * p.nx + x;
}

// node coordinates of a cell index (domains hold fewer than 2^32 cells, so
// 32-bit unsigned division is exact)
__device__ __forceinline__ void coords_of(const Params &p, long long c, int &x, int &y, int &z) {
    const unsigned cu = (unsigned)c, nx = (unsigned)p.nx, ny = (unsigned)p.ny;
    const unsigned row = cu / nx;
    x = (int)(cu - row * nx);
    const unsigned zz = row / ny;
    z = (int)zz;
    y = (int)(row - zz * ny);
}

// i-th coordinate of a region axis in ascending wrapped order: the region
// covers `len` consecutive (unwrapped) coordinates starting at lo.
// Returns -1 for a coordinate outside a non-periodic axis.
__device__ __forceinline__ int region_axis(int k, int lo, int len, int n, int periodic) {
    if (!periodic) {
        int v = lo + k;
        return (v < 0 || v >= n) ? -1 : v;
    }
    if (len >= n) return k < n ? k : -1;
    int s0 = ((lo % n) + n) % n;
    int wr = s0 + len - n;
    if (wr > 0) return k < wr ? k : s0 + (k - wr);
    return s0 + k;
}

// per body and step: X(t) [0], Xw(t) [3], X(t+1) [6], Xw(t+1) [9] (Xw
// wrapped into [0, L)), floor(Xw(t)) [12] and Xw(t) - floor(Xw(t)) [15],
// cos, sin of the orientation at t [18] and at t+1 [24] (15 after Xw)
constexpr int POSE_STRIDE = 26;

// region of a body covering its poses at t and t+1, dilated by `margin`
__device__ __forceinline__ void region_lo(const Params &p, const BodyDev &b, const double *P, int margin, int lo[3]) {
    for (int a = 0; a < 3; ++a) {
        int n = axis_len(p, a);
        bool full = (a == 2 && along_z(b.shape)) || b.ext[a] >= n;
        if (full) {
            lo[a] = 0;
            continue;
        }
        double m = P[a] < P[6 + a] ? P[a] : P[6 + a];
        lo[a] = (int)floor(m - b.R) - margin;
    }
}

} // namespace lbm
