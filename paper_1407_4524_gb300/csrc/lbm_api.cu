// lbm_api.cu -- host implementation of the C ABI declared in include/lbm.h.
//
// A domain owns: two population buffers (fhat at t and t+1), two moment
// buffers (rho,u at the nodes flagged FL_MAC), the node flags, two owner
// arrays (solid owner at t and t+1), two cut-link buffers (t and t+1), the
// per-link momentum-exchange contributions, the covered/uncovered lists and
// the force/torque ring.  lbm_step enqueues, per step, in FP64 mode:
//   moving bodies only: k_prep (poses, link prefixes),
//                       k_geom_a, k_geom_b, k_geom_c  (geometry of t+1)
//   k_links (wall values + ME per link), k_bulk (stream-collide; then
//   k_zouhe for the Zou-He face nodes), k_finish (per-body series row;
//   A+/A- impulsive terms and refill), k_free (free bodies);
// in the reduced-precision modes (do_step_overlapped): k_fprep on the main
// stream, then the surface kernels (k_fgeom1/2, k_bnd, k_finish, k_free) on
// a high-priority side stream beside k_bulk (+ k_zouhe) on the main stream.
// Each lbm_step call ends with a step event that the series reads wait on.
// The serving batch (lbm_batch_*) keeps solves of this kind in slots and
// replays a CUDA graph of batched ticks (lbm_batch.cu).  Every persistent
// device buffer is recorded with its size at allocation, in order: that list
// is the device part of a state snapshot (lbm_save_state / lbm_load_state).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace lbm {
cudaError_t launch_init_p0(int Q, const Params &p, void *dst, void *mac, const uint8_t *flags, const double u0[3],
                           cudaStream_t s);
cudaError_t launch_links_p0(int Q, const Params &p, const StepBufs &sb, int grid, cudaStream_t s);
cudaError_t launch_bulk_p0(int Q, const Params &p, const StepBufs &sb, cudaStream_t s);
cudaError_t launch_finish_p0(int Q, const Params &p, const StepBufs &sb, cudaStream_t s);
cudaError_t launch_init_p12(int Q, int prec, const Params &p, void *dst, void *mac, const uint8_t *flags,
                            const double u0[3], cudaStream_t s);
cudaError_t launch_links_p12(int Q, int prec, const Params &p, const StepBufs &sb, int grid, cudaStream_t s);
cudaError_t launch_bulk_p12(int Q, int prec, const Params &p, const StepBufs &sb, cudaStream_t s);
cudaError_t launch_finish_p12(int Q, int prec, const Params &p, const StepBufs &sb, cudaStream_t s);

cudaError_t launch_load_p0(int Q, const Params &p, const double *stage, long long c0, long long n, void *dst,
                           void *mac, const uint8_t *flags, cudaStream_t s);
cudaError_t launch_macros_p0(int Q, const Params &p, const void *src, const uint16_t *owner, long long c0,
                             long long n, double *out, cudaStream_t s);
cudaError_t launch_load_p12(int Q, int prec, const Params &p, const double *stage, long long c0, long long n,
                            void *dst, void *mac, const uint8_t *flags, cudaStream_t s);
cudaError_t launch_macros_p12(int Q, int prec, const Params &p, const void *src, const uint16_t *owner, long long c0,
                              long long n, double *out, cudaStream_t s);

cudaError_t launch_load(int Q, int prec, const Params &p, const double *stage, long long c0, long long n, void *dst,
                        void *mac, const uint8_t *flags, cudaStream_t s) {
    return prec == 0 ? launch_load_p0(Q, p, stage, c0, n, dst, mac, flags, s)
                     : launch_load_p12(Q, prec, p, stage, c0, n, dst, mac, flags, s);
}
cudaError_t launch_macros(int Q, int prec, const Params &p, const void *src, const uint16_t *owner, long long c0,
                          long long n, double *out, cudaStream_t s) {
    return prec == 0 ? launch_macros_p0(Q, p, src, owner, c0, n, out, s)
                     : launch_macros_p12(Q, prec, p, src, owner, c0, n, out, s);
}
cudaError_t launch_init(int Q, int prec, const Params &p, void *dst, void *mac, const uint8_t *flags,
                        const double u0[3], cudaStream_t s) {
    return prec == 0 ? launch_init_p0(Q, p, dst, mac, flags, u0, s) : launch_init_p12(Q, prec, p, dst, mac, flags, u0, s);
}
cudaError_t launch_links(int Q, int prec, const Params &p, const StepBufs &sb, int grid, cudaStream_t s) {
    return prec == 0 ? launch_links_p0(Q, p, sb, grid, s) : launch_links_p12(Q, prec, p, sb, grid, s);
}
cudaError_t launch_bulk(int Q, int prec, const Params &p, const StepBufs &sb, cudaStream_t s) {
    return prec == 0 ? launch_bulk_p0(Q, p, sb, s) : launch_bulk_p12(Q, prec, p, sb, s);
}
cudaError_t launch_finish(int Q, int prec, const Params &p, const StepBufs &sb, cudaStream_t s) {
    return prec == 0 ? launch_finish_p0(Q, p, sb, s) : launch_finish_p12(Q, prec, p, sb, s);
}
} // namespace lbm

using namespace lbm;

void noalloc_scratch_setup(int dev);

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define CK(x)                                                                                                   \
    do {                                                                                                        \
        cudaError_t e_ = (x);                                                                                   \
        if (e_ != cudaSuccess) return fail(LBM_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_));    \
    } while (0)

constexpr double PI = 3.14159265358979323846;

// Makes `dev` the calling thread's current device for the guard's lifetime
// and gives the caller's own current device back afterwards: no entry point
// leaves the calling thread's current device changed.
struct DevGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DevGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) err = cudaSetDevice(dev);
    }
    ~DevGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
    DevGuard(const DevGuard &) = delete;
    DevGuard &operator=(const DevGuard &) = delete;
};

// the device of a domain / batch current for the rest of the entry point
#define DEVICE_SCOPE(dev)                                                                                       \
    DevGuard dev_guard_(dev);                                                                                   \
    if (dev_guard_.err != cudaSuccess)                                                                          \
        return fail(LBM_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(dev_guard_.err))

} // namespace

struct lbm_domain {
    lbm_domain_desc d{};
    Params p{};
    int Q = 0, prec = 0;
    size_t Ssize = 0, Csize = 0;
    cudaStream_t s = nullptr;
    size_t bytes = 0;
    long long h2d = 0, d2h = 0;
    // lattice state
    void *pop[2] = {nullptr, nullptr};
    void *mac[2] = {nullptr, nullptr};
    uint8_t *flags = nullptr;
    uint16_t *owner[2] = {nullptr, nullptr};
    unsigned long long *counters = nullptr;
    // bodies
    int nb = 0, n_moving = 0, n_free = 0;
    std::vector<lbm_body> hb;
    std::vector<BodyDev> hbd;
    std::vector<void *> body_allocs;
    // every persistent device buffer with its size, in allocation order: the
    // device part of a state snapshot (lbm_save_state / lbm_load_state)
    std::vector<std::pair<void *, size_t>> state_bufs;
    BodyDev *dbodies = nullptr;
    int *dmoving = nullptr;
    int2 *chunk_all = nullptr, *chunk_mov = nullptr;
    int nchunk_all = 0, nchunk_mov = 0;
    int *chunk_cnt_apm = nullptr, *chunk_cnt_link = nullptr;
    uint32_t *Lcell[2] = {nullptr, nullptr};
    uint8_t *Ldir[2] = {nullptr, nullptr};
    double *Ldelta[2] = {nullptr, nullptr};
    long long *link_cnt[2] = {nullptr, nullptr};
    long long link_cap_total = 0;
    double *me = nullptr;
    uint32_t *apm_cell = nullptr;
    int8_t *apm_sign = nullptr;
    long long *apm_cnt = nullptr;
    long long apm_cap_total = 0;
    // semi-implicit free-body schemes: impulsive terms of the previous
    // displacement (scheme 1) and the covered / uncovered lists of the
    // predicted displacement (scheme 2)
    double *imp_prev = nullptr;
    uint32_t *apm_pred_cell = nullptr;
    int8_t *apm_pred_sign = nullptr;
    long long *apm_pred_cnt = nullptr;
    double *series = nullptr;
    long long series_cap = 0;
    double *poses = nullptr;
    long long *link_pre = nullptr;
    long long *tile_pre = nullptr;
    unsigned long long *acc = nullptr;
    unsigned long long *chg_cnt = nullptr;
    uint32_t *chg_cell = nullptr;
    uint8_t *chg_val = nullptr;
    long long chg_cap = 0;
    uint32_t *bn_static = nullptr;
    uint32_t *bn_mov[2] = {nullptr, nullptr};
    unsigned long long *bn_cnt = nullptr; // [0] static, [1], [2] moving lists of even / odd steps
    long long bn_static_cap = 0, bn_mov_cap = 0;
    bool lists_dirty = true;
    int bnd_grid = 0, bnd_grid_full = 0;
    int side_blocks = 0; // block cap of the side-stream kernels
    bool side_serial = false; // run the surface kernels before k_bulk on one stream, uncapped
    bool batch = false;       // a serving batch's solve: boundary-node kernel instead of link mode
    bool prep_dirty = true;
    int links_grid = 0;
    int64_t t = 0;
    // side stream: in the reduced-precision modes the geometry of t+1 and the
    // end-of-step kernel run on it, concurrently with the bulk kernel
    cudaStream_t s2 = nullptr;
    cudaEvent_t ev_prep = nullptr, ev_links = nullptr, ev_side = nullptr;
    // timing of the bulk kernel
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    // reads of the force series wait for the step that wrote the rows (an
    // event recorded at the end of each lbm_step call, with the step count
    // reached) on their own non-blocking stream, not for the whole stream:
    // the caller may enqueue step t+1 before reading the row of step t
    static constexpr int N_STEP_EV = 8;
    cudaStream_t sio = nullptr;
    cudaEvent_t step_ev[N_STEP_EV] = {};
    int64_t step_ev_t[N_STEP_EV] = {};
    int step_ev_next = 0;
    // CUDA-graph replay: lbm_step runs GRAPH_STEPS consecutive steps (from an
    // even step, so that the buffer parities match) as one captured graph; the
    // step kernels read their step index from the device counter, so the same
    // graph serves every replay.  Kernel timing inside it uses its own events.
    static constexpr int GRAPH_STEPS = 16;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t scap = nullptr; // capture stream (the domain's stream may be the legacy default stream)
    bool graph_dirty = true;   // capture again before the next replay
    bool graph_failed = false; // capture not possible: plain launches only
    bool capturing = false;
    int cap_k = 0;             // step index within the graph being captured
    cudaEvent_t gev[2 * GRAPH_STEPS] = {};
    bool g_timed = false;      // a timed replay ran since the timings were last read
    // body records staged in pinned memory for lbm_update_bodies (two, each
    // reused once its copy has completed)
    BodyDev *hbd_pin[2] = {nullptr, nullptr};
    cudaEvent_t up_ev[2] = {nullptr, nullptr};
    int up_k = 0;

    void *alloc(size_t n) {
        if (n == 0) n = 256;
        void *ptr = nullptr;
        if (d.alloc) ptr = d.alloc(n, d.alloc_ctx);
        else if (cudaMalloc(&ptr, n) != cudaSuccess) ptr = nullptr;
        return ptr;
    }
    void release(void *ptr) {
        if (!ptr) return;
        if (d.free) d.free(ptr, d.alloc_ctx);
        else cudaFree(ptr);
    }
};

namespace {

int alloc_into(lbm_domain *D, void **slot, size_t n, std::vector<void *> *track) {
    void *ptr = D->alloc(n);
    if (!ptr) return fail(LBM_ERR_OOM, "device allocation of " + std::to_string(n) + " bytes failed");
    D->bytes += n;
    if (cudaMemsetAsync(ptr, 0, n, D->s) != cudaSuccess) return fail(LBM_ERR_CUDA, "cudaMemsetAsync failed");
    *slot = ptr;
    if (track) track->push_back(ptr);
    D->state_bufs.emplace_back(ptr, n);
    return LBM_OK;
}

template <class T> int alloc_t(lbm_domain *D, T **slot, size_t count, std::vector<void *> *track) {
    void *v = nullptr;
    int rc = alloc_into(D, &v, count * sizeof(T), track);
    *slot = (T *)v;
    return rc;
}

void free_body_buffers(lbm_domain *D) {
    for (void *ptr : D->body_allocs) {
        for (size_t k = 0; k < D->state_bufs.size(); ++k)
            if (D->state_bufs[k].first == ptr) {
                D->state_bufs.erase(D->state_bufs.begin() + (long)k);
                break;
            }
        D->release(ptr);
    }
    D->body_allocs.clear();
    for (int k = 0; k < 2; ++k) { // pinned body staging: sized for the body count it was made for
        if (!D->hbd_pin[k]) continue;
        cudaEventSynchronize(D->up_ev[k]);
        cudaFreeHost(D->hbd_pin[k]);
        D->hbd_pin[k] = nullptr;
    }
    D->dbodies = nullptr;
    D->dmoving = nullptr;
    D->chunk_all = D->chunk_mov = nullptr;
    D->chunk_cnt_apm = D->chunk_cnt_link = nullptr;
    for (int k = 0; k < 2; ++k) {
        D->Lcell[k] = nullptr;
        D->Ldir[k] = nullptr;
        D->Ldelta[k] = nullptr;
        D->link_cnt[k] = nullptr;
    }
    D->me = nullptr;
    D->apm_cell = nullptr;
    D->apm_sign = nullptr;
    D->apm_cnt = nullptr;
    D->imp_prev = nullptr;
    D->apm_pred_cell = nullptr;
    D->apm_pred_sign = nullptr;
    D->apm_pred_cnt = nullptr;
    D->series = nullptr;
    D->poses = nullptr;
    D->link_pre = nullptr;
    D->tile_pre = nullptr;
    D->acc = nullptr;
    D->chg_cnt = nullptr;
    D->chg_cell = nullptr;
    D->chg_val = nullptr;
    D->chg_cap = 0;
    D->bn_static = nullptr;
    D->bn_mov[0] = D->bn_mov[1] = nullptr;
    D->bn_cnt = nullptr;
    D->bn_static_cap = D->bn_mov_cap = 0;
    D->lists_dirty = true;
    D->prep_dirty = true;
    D->nb = D->n_moving = D->n_free = 0;
    D->nchunk_all = D->nchunk_mov = 0;
    D->link_cap_total = D->apm_cap_total = 0;
}

bool is_moving(const lbm_body &b) {
    if (b.free_body) return true; // its velocity is set by the flow
    for (int k = 0; k < 3; ++k)
        if (b.U[k] != 0.0 || b.W[k] != 0.0) return true;
    return false;
}

// upper bound of the cut links of a body: boundary nodes lie in the shell
// R < |x - X| <= R + sqrt(2); their unit cells fit in the shell widened by
// half a cell diagonal, so the shell volume bounds their number.
long long link_capacity(const lbm_domain *D, const lbm_body &b) {
    const double cmax = std::sqrt(2.0);
    double nodes;
    if (b.shape == LBM_SHAPE_SPHERE) {
        const double h = std::sqrt(3.0) / 2.0;
        double ro = b.R + cmax + h, ri = std::max(0.0, b.R - h);
        nodes = 4.0 / 3.0 * PI * (ro * ro * ro - ri * ri * ri);
    } else {
        const double h = std::sqrt(2.0) / 2.0;
        double ro = b.R + cmax + h, ri = std::max(0.0, b.R - h);
        nodes = PI * (ro * ro - ri * ri) * D->p.nz;
    }
    return (long long)std::ceil(nodes) * (D->Q - 1) + 256;
}

void body_params(const lbm_domain *D, const lbm_body &b, BodyDev &o) {
    std::memset(&o, 0, sizeof(o));
    o.shape = b.shape;
    o.halfway = b.halfway;
    o.moving = is_moving(b) ? 1 : 0;
    o.R = b.R;
    for (int k = 0; k < 3; ++k) {
        o.X0[k] = b.X0[k];
        o.U[k] = b.U[k];
        o.W[k] = b.W[k];
    }
    o.t0 = b.t0;
    o.free = b.free_body ? 1 : 0;
    o.density_ratio = b.density_ratio;
    o.R2 = b.shape == LBM_SHAPE_ELLIPSE ? b.R2 : b.R;
    o.theta0 = b.shape == LBM_SHAPE_ELLIPSE ? b.theta0 : 0.0;
    const int n[3] = {D->p.nx, D->p.ny, D->p.nz};
    for (int a = 0; a < 3; ++a) {
        int e = 2 * (int)std::ceil(b.R) + 2 * REGION_MARGIN + 5;
        if ((a == 2 && along_z(b.shape)) || e >= n[a]) e = n[a];
        o.ext[a] = e;
    }
    long long vol = (long long)o.ext[0] * o.ext[1] * o.ext[2];
    o.nchunks = (int)((vol + GEOM_CHUNK - 1) / GEOM_CHUNK);
    o.link_cap = link_capacity(D, b);
    o.apm_cap = vol;
}

double min_image(double v, int n, bool per) {
    if (!per) return v;
    return v - n * std::floor(v / n + 0.5);
}

int validate_bodies(const lbm_domain *D, const lbm_body *b, int n) {
    const int nn[3] = {D->p.nx, D->p.ny, D->p.nz};
    for (int k = 0; k < n; ++k) {
        const lbm_body &B = b[k];
        if (B.shape != LBM_SHAPE_CYLINDER && B.shape != LBM_SHAPE_SPHERE && B.shape != LBM_SHAPE_ELLIPSE)
            return fail(LBM_ERR_ARG, "body " + std::to_string(k) + ": unknown shape");
        if (B.shape == LBM_SHAPE_ELLIPSE && !(B.R2 > 0.0 && B.R2 <= B.R && std::isfinite(B.theta0)))
            return fail(LBM_ERR_ARG, "an ellipse needs 0 < R2 <= R and a finite theta0");
        if (B.shape == LBM_SHAPE_SPHERE && D->Q == 9)
            return fail(LBM_ERR_ARG, "body " + std::to_string(k) + ": spheres need D3Q19 (use a cylinder in 2-D)");
        if (!(B.R > 0.0) || !std::isfinite(B.R)) return fail(LBM_ERR_ARG, "body radius must be positive");
        if (B.reserved) return fail(LBM_ERR_ARG, "reserved body fields must be 0");
        if (B.free_body != 0 && B.free_body != 1) return fail(LBM_ERR_ARG, "free_body must be 0 or 1");
        if (B.free_body && !(B.density_ratio > 0.0 && std::isfinite(B.density_ratio)))
            return fail(LBM_ERR_ARG, "a free body needs a positive density ratio");
        if (B.halfway != 0 && B.halfway != 1) return fail(LBM_ERR_ARG, "halfway must be 0 or 1");
        for (int a = 0; a < 3; ++a) {
            if (a == 2 && along_z(B.shape)) continue;
            if (!std::isfinite(B.X0[a]) || !std::isfinite(B.U[a]) || !std::isfinite(B.W[a]))
                return fail(LBM_ERR_ARG, "body state must be finite");
            if (D->p.per[a]) {
                if (2.0 * B.R + 4.0 >= nn[a])
                    return fail(LBM_ERR_ARG, "body " + std::to_string(k) + " is too large for the periodic axis");
                if (is_moving(B) && 2.0 * B.R + 14.0 >= nn[a])
                    return fail(LBM_ERR_ARG, "moving body " + std::to_string(k) +
                                                 " needs 2R + 14 cells along each periodic axis");
            } else {
                if (B.X0[a] - B.R < 3.0 || B.X0[a] + B.R > nn[a] - 4.0)
                    return fail(LBM_ERR_ARG, "body " + std::to_string(k) +
                                                 " must keep 3 cells from non-periodic faces");
                if (B.U[a] != 0.0 && !B.free_body)
                    return fail(LBM_ERR_ARG, "bodies may not translate along a non-periodic axis");
            }
        }
        double umax = std::sqrt(B.U[0] * B.U[0] + B.U[1] * B.U[1] + B.U[2] * B.U[2]) +
                      B.R * std::sqrt(B.W[0] * B.W[0] + B.W[1] * B.W[1] + B.W[2] * B.W[2]);
        if (umax > 0.25) // keeps the fluid next to it below the |u| = 0.3 stability check
            return fail(LBM_ERR_ARG, "body surface may move at most 0.25 cells per step");
        for (int m = 0; m < k; ++m) {
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                if (a == 2 && (along_z(B.shape) || along_z(b[m].shape))) continue;
                double v = min_image(B.X0[a] + (0 - B.t0) * B.U[a] - (b[m].X0[a] + (0 - b[m].t0) * b[m].U[a]),
                                     nn[a], D->p.per[a] != 0);
                d2 += v * v;
            }
            if (std::sqrt(d2) - B.R - b[m].R < 2.0)
                return fail(LBM_ERR_ARG, "bodies " + std::to_string(m) + " and " + std::to_string(k) +
                                             " are closer than a 2-cell gap");
        }
    }
    return LBM_OK;
}

StepBufs step_bufs(lbm_domain *D) {
    const int cur = (int)(D->t & 1), nxt = cur ^ 1;
    StepBufs sb{};
    sb.src = D->pop[cur];
    sb.dst = D->pop[nxt];
    sb.mac_t = D->mac[cur];
    sb.mac_t1 = D->mac[nxt];
    sb.flags = D->flags;
    sb.owner_t = D->owner[cur];
    sb.bodies = D->dbodies;
    sb.moving_ids = D->dmoving;
    sb.n_moving = D->n_moving;
    sb.link_cnt = D->link_cnt[cur];
    sb.link_pre = D->link_pre;
    sb.tile_pre = D->tile_pre;
    sb.acc = D->acc;
    sb.poses = D->poses;
    sb.Lcell = D->Lcell[cur];
    sb.Ldir = D->Ldir[cur];
    sb.Ldelta = D->Ldelta[cur];
    sb.me = D->me;
    sb.apm_cnt = D->apm_cnt;
    sb.apm_cell = D->apm_cell;
    sb.apm_sign = D->apm_sign;
    sb.series = D->series;
    sb.counters = D->counters;
    sb.t = D->t;
    sb.par = (int)(D->t & 1);
    sb.phase = PH_ALL;
    sb.imp_prev = D->imp_prev;
    sb.apm_pred_cell = D->apm_pred_cell;
    sb.apm_pred_sign = D->apm_pred_sign;
    sb.apm_pred_cnt = D->apm_pred_cnt;
    return sb;
}

GeomArgs geom_args(lbm_domain *D, bool moving_step) {
    const int cur = (int)(D->t & 1), nxt = cur ^ 1;
    GeomArgs g{};
    g.bodies = D->dbodies;
    g.poses = D->poses;
    g.chunk_map = moving_step ? D->chunk_mov : D->chunk_all;
    g.nchunks = moving_step ? D->nchunk_mov : D->nchunk_all;
    g.owner_t = D->owner[cur];
    g.owner_t1 = moving_step ? D->owner[nxt] : D->owner[cur];
    g.flags = D->flags;
    g.chunk_cnt_apm = D->chunk_cnt_apm;
    g.chunk_cnt_link = D->chunk_cnt_link;
    g.apm_cell = D->apm_cell;
    g.apm_sign = D->apm_sign;
    g.apm_cnt = D->apm_cnt;
    const int lb = moving_step ? nxt : cur;
    g.Lcell = D->Lcell[lb];
    g.Ldir = D->Ldir[lb];
    g.Ldelta = D->Ldelta[lb];
    g.link_cnt = D->link_cnt[lb];
    g.t = D->t;
    g.t_link = moving_step ? D->t + 1 : D->t;
    g.do_apm = moving_step ? 1 : 0;
    g.chg_cnt = D->chg_cnt;
    g.chg_cell = D->chg_cell;
    g.chg_val = D->chg_val;
    g.chg_cap = D->chg_cap;
    g.bn_static = D->bn_static;
    g.bn_static_cnt = D->bn_cnt;
    g.bn_mov = D->bn_mov[nxt];
    g.bn_mov_cnt = D->bn_cnt + 1 + nxt;
    g.bn_static_cap = D->bn_static_cap;
    g.bn_mov_cap = D->bn_mov_cap;
    g.do_flags = (moving_step && D->prec == LBM_FP64) ? 1 : 0;
    return g;
}

int init_populations(lbm_domain *D) {
    CK(launch_init(D->Q, D->prec, D->p, D->pop[D->t & 1], D->mac[D->t & 1], D->flags, D->d.u0, D->s));
    return LBM_OK;
}

// body records -> device through a pinned staging buffer, in stream order
// after the steps already enqueued (no host synchronisation)
int upload_body_array(lbm_domain *D) {
    const int k = D->up_k;
    D->up_k ^= 1;
    if (!D->hbd_pin[k]) CK(cudaMallocHost((void **)&D->hbd_pin[k], sizeof(BodyDev) * (size_t)std::max(D->nb, 1)));
    CK(cudaEventSynchronize(D->up_ev[k])); // the copy that last read this buffer is done
    std::memcpy(D->hbd_pin[k], D->hbd.data(), sizeof(BodyDev) * D->nb);
    CK(cudaMemcpyAsync(D->dbodies, D->hbd_pin[k], sizeof(BodyDev) * D->nb, cudaMemcpyHostToDevice, D->s));
    CK(cudaEventRecord(D->up_ev[k], D->s));
    D->h2d += (long long)(sizeof(BodyDev) * D->nb);
    return LBM_OK;
}

int upload_bodies(lbm_domain *D) {
    // moving list and chunk maps
    std::vector<int> mov;
    std::vector<int2> all, mv;
    for (int b = 0; b < D->nb; ++b) {
        BodyDev &B = D->hbd[b];
        B.chunk_base = (int)all.size();
        for (int c = 0; c < B.nchunks; ++c) all.push_back(make_int2(b, c));
        if (B.moving) {
            mov.push_back(b);
            for (int c = 0; c < B.nchunks; ++c) mv.push_back(make_int2(b, c));
        }
    }
    D->n_moving = (int)mov.size();
    D->n_free = 0;
    for (int b = 0; b < D->nb; ++b) D->n_free += D->hbd[b].free ? 1 : 0;
    D->nchunk_all = (int)all.size();
    D->nchunk_mov = (int)mv.size();
    D->graph_dirty = true; // launch shapes follow the body maps
    CK(cudaMemcpyAsync(D->dbodies, D->hbd.data(), sizeof(BodyDev) * D->nb, cudaMemcpyHostToDevice, D->s));
    D->h2d += (long long)(sizeof(BodyDev) * D->nb);
    if (!mov.empty()) CK(cudaMemcpyAsync(D->dmoving, mov.data(), sizeof(int) * mov.size(), cudaMemcpyHostToDevice, D->s));
    CK(cudaMemcpyAsync(D->chunk_all, all.data(), sizeof(int2) * all.size(), cudaMemcpyHostToDevice, D->s));
    if (!mv.empty()) CK(cudaMemcpyAsync(D->chunk_mov, mv.data(), sizeof(int2) * mv.size(), cudaMemcpyHostToDevice, D->s));
    CK(cudaStreamSynchronize(D->s)); // host vectors go out of scope
    return LBM_OK;
}

int do_step_overlapped(lbm_domain *D);

// reduced-precision modes: boundary-node lists of step t from scratch
int build_bnd_lists(lbm_domain *D) {
    if (D->p.linkmode) { // link mode keeps cut-link lists instead
        D->lists_dirty = false;
        return LBM_OK;
    }
    const int cur = (int)(D->t & 1);
    CK(cudaMemsetAsync(D->bn_cnt, 0, 3 * sizeof(unsigned long long), D->s));
    GeomArgs gl = geom_args(D, false);
    gl.bn_mov = D->bn_mov[cur];
    gl.bn_mov_cnt = D->bn_cnt + 1 + cur;
    CK(launch_bnd_lists(D->Q, D->p, gl, D->s));
    D->lists_dirty = false;
    return LBM_OK;
}

// a timing event: while a graph is captured it must be an external event
// record (a plain record inside a capture only orders the graph's branches)
cudaError_t record_timing(lbm_domain *D, cudaEvent_t e) {
    return D->capturing ? cudaEventRecordWithFlags(e, D->s, cudaEventRecordExternal) : cudaEventRecord(e, D->s);
}

// events around the bulk kernel of this step (kernel timing): the graph's own
// pair while a graph is captured, else the next pair of the ring
int timing_events(lbm_domain *D, cudaEvent_t &a, cudaEvent_t &b) {
    if (D->capturing) {
        a = D->gev[2 * D->cap_k];
        b = D->gev[2 * D->cap_k + 1];
        return LBM_OK;
    }
    if (D->ev_used + 2 > D->ev.size()) {
        for (int k = 0; k < 64; ++k) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            D->ev.push_back(e);
        }
    }
    a = D->ev[D->ev_used];
    b = D->ev[D->ev_used + 1];
    D->ev_used += 2;
    return LBM_OK;
}

// the free-body scheme a step runs (the explicit one when no body is free)
int step_scheme(const lbm_domain *D) { return D->n_free ? D->p.free_scheme : LBM_FREE_EXPLICIT; }

// semi-implicit schemes, after the stream-collide pass: the force row of step
// t (with the impulsive terms of the previous displacement, or of the
// predicted one whose lists sb_pred names), the velocities of t+1, the poses
// of t+1 they give, the owners, lists and cut links of the displacement made,
// then its impulsive terms and refill (scheme 1) or the refill of the nodes
// the prediction did not uncover (scheme 2).  All on stream s.
int finish_semi(lbm_domain *D, int scheme, const StepBufs &sb) {
    const int Q = D->Q, prec = D->prec;
    StepBufs s1 = sb;
    if (scheme == LBM_FREE_AIDUN) {
        s1.phase = PH_REDUCE;
    } else {
        s1.apm_cell = D->apm_pred_cell;
        s1.apm_sign = D->apm_pred_sign;
        s1.apm_cnt = D->apm_pred_cnt;
    }
    CK(launch_finish(Q, prec, D->p, s1, D->s));
    const unsigned long long *tdev = D->counters + 9 + (D->t & 1);
    CK(launch_free(D->p, D->dbodies, D->series, D->counters, tdev, D->s));
    CK(launch_pose1(D->p, D->dbodies, D->poses, tdev, D->s));
    GeomArgs g = geom_args(D, true);
    if (prec == LBM_FP64) {
        CK(launch_geom_a(Q, D->p, g, D->s));
        CK(launch_geom_b(Q, D->p, g, D->s));
        CK(launch_geom_c(Q, D->p, g, D->s));
    } else {
        CK(launch_fgeom1(Q, D->p, g, D->s));
        CK(launch_fgeom2(Q, D->p, g, D->s));
    }
    StepBufs s2 = sb;
    s2.phase = scheme == LBM_FREE_AIDUN ? PH_IMP : PH_FIX;
    CK(launch_finish(Q, prec, D->p, s2, D->s));
    return LBM_OK;
}

// scheme 2, before the stream-collide pass: owners and covered / uncovered
// lists of the displacement predicted with U(t), into the prediction's lists
GeomArgs predicted_geom(lbm_domain *D) {
    GeomArgs g = geom_args(D, true);
    g.apm_cell = D->apm_pred_cell;
    g.apm_sign = D->apm_pred_sign;
    g.apm_cnt = D->apm_pred_cnt;
    return g;
}

int do_step(lbm_domain *D) {
    const int Q = D->Q, prec = D->prec;
    if (prec != LBM_FP64 && D->nb) return do_step_overlapped(D);
    D->lists_dirty = false; // boundary-node lists belong to the overlapped path only
    const int scheme = step_scheme(D);
    if (D->nb && (D->n_moving || D->prep_dirty)) {
        // the A+/A- lists of the previous step update the solid flags of t
        CK(launch_prep(D->p, D->dbodies, D->link_cnt[D->t & 1], D->link_pre, D->tile_pre, D->poses, D->t,
                       D->counters + 9 + (D->t & 1), D->flags, D->apm_cnt, D->apm_cell, D->apm_sign, D->s));
        D->prep_dirty = false;
    }
    if (D->n_moving) {
        // semi-implicit schemes: the node flags of t+1 (moments kept on a band
        // around the free bodies) from the displacement with U(t), and scheme
        // 2's predicted lists; the cut links follow the displacement made
        GeomArgs g = scheme == LBM_FREE_PREDICTOR ? predicted_geom(D) : geom_args(D, true);
        CK(launch_geom_a(Q, D->p, g, D->s));
        CK(launch_geom_b(Q, D->p, g, D->s));
        if (scheme == LBM_FREE_EXPLICIT) CK(launch_geom_c(Q, D->p, g, D->s));
    }
    StepBufs sb = step_bufs(D);
    if (D->nb) CK(launch_links(Q, prec, D->p, sb, D->links_grid, D->s));
    cudaEvent_t ta = nullptr, tb = nullptr;
    if (D->timing) {
        int trc = timing_events(D, ta, tb);
        if (trc) return trc;
        CK(record_timing(D, ta));
    }
    CK(launch_bulk(Q, prec, D->p, sb, D->s));
    if (D->timing) CK(record_timing(D, tb));
    if (scheme != LBM_FREE_EXPLICIT) {
        int rc = finish_semi(D, scheme, sb);
        if (rc) return rc;
    } else {
        if (D->nb) CK(launch_finish(Q, prec, D->p, sb, D->s));
        if (D->n_free) CK(launch_free(D->p, D->dbodies, D->series, D->counters, D->counters + 9 + (D->t & 1), D->s));
    }
    D->t += 1;
    if (D->capturing) D->cap_k += 1;
    return LBM_OK;
}

// Reduced-precision modes.  Stream s: prep -> bulk (every fluid node that is
// not a boundary node).  Side stream, after prep: owner and flag changes of
// t+1 (moving bodies), the boundary-node kernel (cut links, momentum
// exchange, collision of the boundary nodes) and the end-of-step kernel
// (series row, impulsive terms, refill).  The bulk kernel reads fhat(t) and
// the flags of t and writes fhat(t+1) of the non-boundary fluid nodes; the
// side stream writes fhat(t+1) of the boundary and refilled nodes, the owner
// array of t+1, the lists and the accumulators: the two streams touch
// disjoint data.  Flag changes are applied by the next prep.
int do_step_links(lbm_domain *D);

int do_step_overlapped(lbm_domain *D) {
    if (D->p.linkmode) return do_step_links(D);
    const int Q = D->Q, prec = D->prec;
    const int cur = (int)(D->t & 1), nxt = cur ^ 1;
    if (D->n_moving || D->prep_dirty || D->lists_dirty) {
        CK(launch_fprep(D->p, D->dbodies, D->poses, D->t, D->counters + 9 + (D->t & 1), D->flags, D->chg_cnt, D->chg_cell,
                        D->chg_val, D->chg_cap,
                        D->apm_cnt, D->bn_cnt + 1 + nxt, nullptr, nullptr, nullptr, D->s));
        D->prep_dirty = false;
    }
    if (D->lists_dirty) {
        int rc = build_bnd_lists(D);
        if (rc) return rc;
    }
    // side stream, or the main stream itself in the serial arrangement
    cudaStream_t ss = D->side_serial ? D->s : D->s2;
    if (!D->side_serial) {
        CK(cudaEventRecord(D->ev_prep, D->s));
        CK(cudaStreamWaitEvent(D->s2, D->ev_prep, 0));
    }
    StepBufs sb = step_bufs(D);
    GeomArgs g = geom_args(D, true);
    g.grid_cap = D->side_serial ? 0 : D->side_blocks;
    if (D->n_moving) {
        CK(launch_fgeom1(Q, D->p, g, ss));
        CK(launch_fgeom2(Q, D->p, g, ss));
    }
    BndArgs ba{};
    ba.static_cells = D->bn_static;
    ba.static_cnt = D->bn_cnt;
    ba.mov_cells = D->bn_mov[cur];
    ba.mov_cnt = D->bn_cnt + 1 + cur;
    ba.static_cap = D->bn_static_cap;
    ba.mov_cap = D->bn_mov_cap;
    ba.owner_t = D->owner[cur];
    ba.owner_t1 = D->owner[nxt];
    ba.bodies = D->dbodies;
    ba.poses = D->poses;
    CK(launch_bnd(Q, prec, D->p, ba, sb, D->side_serial ? D->bnd_grid_full : D->bnd_grid, ss));
    CK(launch_finish(Q, prec, D->p, sb, ss));
    if (D->n_free) CK(launch_free(D->p, D->dbodies, D->series, D->counters, D->counters + 9 + (D->t & 1), ss));
    if (!D->side_serial) CK(cudaEventRecord(D->ev_side, D->s2));
    cudaEvent_t ta = nullptr, tb = nullptr;
    if (D->timing) {
        int trc = timing_events(D, ta, tb);
        if (trc) return trc;
        CK(record_timing(D, ta));
    }
    CK(launch_bulk(Q, prec, D->p, sb, D->s));
    if (D->timing) CK(record_timing(D, tb));
    if (!D->side_serial) CK(cudaStreamWaitEvent(D->s, D->ev_side, 0));
    D->t += 1;
    if (D->capturing) D->cap_k += 1;
    return LBM_OK;
}

// Link mode (reduced precision, single domain).  Stream s: prep -> cut links
// (wall values into the solid nodes' slots, momentum exchange) -> stream-collide
// of every fluid node (boundary nodes included; moments kept at the nodes near
// bodies).  Side stream: after prep, the owners, covered/uncovered lists, flag
// changes and cut links of t+1 of the moving bodies; after the cut links, the
// end of step (series row, impulsive terms with covered nodes re-pulled from
// fhat(t) and its wall values, refill of uncovered nodes) and the free-body
// update.  The side stream overlaps the stream-collide pass and touches no
// data it reads or writes: the links of t+1 go to the other list buffer, the
// kept-moment band only gains flags, refilled nodes were solid at t.
int do_step_links(lbm_domain *D) {
    const int Q = D->Q, prec = D->prec;
    const int cur = (int)(D->t & 1), nxt = cur ^ 1;
    if (D->n_moving || D->prep_dirty || D->lists_dirty) {
        CK(launch_fprep(D->p, D->dbodies, D->poses, D->t, D->counters + 9 + (D->t & 1), D->flags, D->chg_cnt, D->chg_cell,
                        D->chg_val, D->chg_cap, D->apm_cnt, D->bn_cnt + 1 + nxt, D->link_cnt[cur], D->link_cnt[nxt],
                        D->tile_pre, D->s));
        D->prep_dirty = false;
        D->lists_dirty = false;
    }
    const int scheme = step_scheme(D);
    if (scheme != LBM_FREE_EXPLICIT) { // semi-implicit free-body schemes: one stream
        StepBufs sb = step_bufs(D);
        if (scheme == LBM_FREE_PREDICTOR) {
            CK(cudaMemsetAsync(D->apm_pred_cnt, 0, sizeof(long long) * (size_t)D->nb, D->s));
            CK(launch_fgeom1(Q, D->p, predicted_geom(D), D->s));
        }
        CK(launch_links(Q, prec, D->p, sb, D->links_grid, D->s));
        cudaEvent_t ta = nullptr, tb = nullptr;
        if (D->timing) {
            int trc = timing_events(D, ta, tb);
            if (trc) return trc;
            CK(record_timing(D, ta));
        }
        CK(launch_bulk(Q, prec, D->p, sb, D->s));
        if (D->timing) CK(record_timing(D, tb));
        int rc = finish_semi(D, scheme, sb);
        if (rc) return rc;
        D->t += 1;
        if (D->capturing) D->cap_k += 1;
        return LBM_OK;
    }
    const bool side = !D->side_serial;
    cudaStream_t ss = side ? D->s2 : D->s;
    StepBufs sb = step_bufs(D);
    if (side) {
        CK(cudaEventRecord(D->ev_prep, D->s));
        CK(cudaStreamWaitEvent(D->s2, D->ev_prep, 0));
    }
    if (D->n_moving) {
        GeomArgs g = geom_args(D, true);
        g.grid_cap = side ? D->side_blocks : 0;
        CK(launch_fgeom1(Q, D->p, g, ss));
        CK(launch_fgeom2(Q, D->p, g, ss));
    }
    CK(launch_links(Q, prec, D->p, sb, D->links_grid, D->s));
    if (side) {
        CK(cudaEventRecord(D->ev_links, D->s));
        CK(cudaStreamWaitEvent(D->s2, D->ev_links, 0));
    }
    CK(launch_finish(Q, prec, D->p, sb, ss));
    if (D->n_free) CK(launch_free(D->p, D->dbodies, D->series, D->counters, D->counters + 9 + (D->t & 1), ss));
    if (side) CK(cudaEventRecord(D->ev_side, D->s2));
    cudaEvent_t ta = nullptr, tb = nullptr;
    if (D->timing) {
        int trc = timing_events(D, ta, tb);
        if (trc) return trc;
        CK(record_timing(D, ta));
    }
    CK(launch_bulk(Q, prec, D->p, sb, D->s));
    if (D->timing) CK(record_timing(D, tb));
    if (side) CK(cudaStreamWaitEvent(D->s, D->ev_side, 0));
    D->t += 1;
    if (D->capturing) D->cap_k += 1;
    return LBM_OK;
}

} // namespace

extern "C" {

const char *lbm_last_error(void) { return g_err.c_str(); }

const char *lbm_version(void) { return "lbm-gb300 0.1 (sm_103a)"; }

int lbm_lattice_table(int lattice, int *c, double *w, int *opp) {
    if (!c || !w || !opp) return fail(LBM_ERR_ARG, "null output");
    LatTab t;
    if (lattice == LBM_D2Q9) t = make_tab<Lat<9>>();
    else if (lattice == LBM_D3Q19) t = make_tab<Lat<19>>();
    else return fail(LBM_ERR_ARG, "lattice must be 9 or 19");
    for (int i = 0; i < lattice; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = t.c[i][a];
        w[i] = t.w[i];
        opp[i] = t.opp[i];
    }
    return LBM_OK;
}

namespace {
int create_domain_impl(const lbm_domain_desc *desc, lbm_domain **out, bool batch);
} // namespace

int lbm_create_domain(const lbm_domain_desc *desc, lbm_domain **out) { return create_domain_impl(desc, out, false); }

namespace {
// batch: a serving batch's solve (the boundary-node kernel steps its
// boundary nodes; no cut-link lists, no kept moments)
int create_domain_impl(const lbm_domain_desc *desc, lbm_domain **out, bool batch) {
    if (!desc || !out) return fail(LBM_ERR_ARG, "null argument");
    *out = nullptr;
    const lbm_domain_desc &d = *desc;
    if (d.lattice != LBM_D2Q9 && d.lattice != LBM_D3Q19) return fail(LBM_ERR_ARG, "lattice must be LBM_D2Q9 or LBM_D3Q19");
    if (d.nx < 1 || d.ny < 1 || d.nz < 1) return fail(LBM_ERR_ARG, "grid sizes must be >= 1");
    if (d.lattice == LBM_D2Q9 && d.nz != 1) return fail(LBM_ERR_ARG, "D2Q9 needs nz = 1");
    if ((long long)d.nx * d.ny * d.nz >= (1ll << 32)) return fail(LBM_ERR_ARG, "more than 2^32 cells");
    if (d.ny > 65535 || d.nz > 65535) return fail(LBM_ERR_ARG, "ny and nz must be <= 65535");
    if (d.precision < LBM_FP64 || d.precision > LBM_FP16) return fail(LBM_ERR_ARG, "unknown precision");
    if (d.equilibrium != LBM_EQ_INCOMP && d.equilibrium != LBM_EQ_STANDARD) return fail(LBM_ERR_ARG, "unknown equilibrium");
    if (!(d.tau > 0.5) || !std::isfinite(d.tau)) return fail(LBM_ERR_ARG, "tau must be > 1/2");
    if (!(d.rho0 > 0.0)) return fail(LBM_ERR_ARG, "rho0 must be > 0");
    for (int a = 0; a < 3; ++a)
        if ((d.edge[2 * a] == LBM_EDGE_PERIODIC) != (d.edge[2 * a + 1] == LBM_EDGE_PERIODIC))
            return fail(LBM_ERR_ARG, "an axis is periodic on both faces or on neither");
    for (int e = 0; e < 6; ++e) {
        if (d.edge[e] < 0 || d.edge[e] > 3) return fail(LBM_ERR_ARG, "unknown edge kind");
        if (d.edge[e] == LBM_EDGE_INLET && e != 0) return fail(LBM_ERR_ARG, "the inlet must be the x-low face");
        if (d.edge[e] == LBM_EDGE_OUTLET && e != 1) return fail(LBM_ERR_ARG, "the outlet must be the x-high face");
    }
    if (d.lattice == LBM_D2Q9 && d.edge[4] != LBM_EDGE_PERIODIC) return fail(LBM_ERR_ARG, "D2Q9: z must be periodic");
    if (d.refill != LBM_REFILL_RHOBAR_UB && d.refill != LBM_REFILL_RHOBAR_UBAR && d.refill != LBM_REFILL_EXTRAP)
        return fail(LBM_ERR_ARG, "unknown refill rule");
    if (d.inlet_profile != LBM_INLET_UNIFORM && d.inlet_profile != LBM_INLET_PARABOLIC)
        return fail(LBM_ERR_ARG, "unknown inlet profile");
    if (d.edge_rule != LBM_EDGE_RULE_LINK && d.edge_rule != LBM_EDGE_RULE_ZOUHE)
        return fail(LBM_ERR_ARG, "unknown edge rule");
    if (d.free_scheme < LBM_FREE_EXPLICIT || d.free_scheme > LBM_FREE_PREDICTOR)
        return fail(LBM_ERR_ARG, "unknown free-body scheme");
    if (d.edge_rule == LBM_EDGE_RULE_ZOUHE) {
        const int nn[3] = {d.nx, d.ny, d.nz};
        for (int a = 0; a < 3; ++a)
            if (d.edge[2 * a] != LBM_EDGE_PERIODIC && nn[a] < 3)
                return fail(LBM_ERR_ARG, "Zou-He faces need at least 3 nodes along their axis");
    }
    if ((d.alloc == nullptr) != (d.free == nullptr)) return fail(LBM_ERR_ARG, "alloc and free go together");

    DEVICE_SCOPE(d.device);
    cudaError_t e = cudaSuccess;
    noalloc_scratch_setup(d.device); // before any allocation or stream capture of this domain

    lbm_domain *D = new lbm_domain();
    D->d = d;
    D->batch = batch;
    D->Q = d.lattice;
    D->prec = d.precision;
    D->s = (cudaStream_t)d.stream;
    D->Ssize = d.precision == LBM_FP64 ? 8 : (d.precision == LBM_FP32 ? 4 : 2);
    D->Csize = d.precision == LBM_FP64 ? 8 : 4;
    Params &p = D->p;
    p.nx = d.nx;
    p.ny = d.ny;
    p.nz = d.nz;
    p.N = (long long)d.nx * d.ny * d.nz;
    for (int a = 0; a < 3; ++a) p.per[a] = d.edge[2 * a] == LBM_EDGE_PERIODIC;
    for (int k = 0; k < 6; ++k) p.edge[k] = d.edge[k];
    p.nonper = !(p.per[0] && p.per[1] && p.per[2]);
    p.exact = d.precision == LBM_FP64;
    p.linkmode = (!batch && d.precision != LBM_FP64) ? 1 : 0;
    p.free_scheme = d.free_scheme;
    {
        // LBM_STAGED=1 selects the stream-collide kernel that stages the
        // source rows in shared memory by bulk copies (same results bit for
        // bit; slower than the direct kernels with row-sized copies, so not
        // the default)
        const char *es = std::getenv("LBM_STAGED");
        p.staged = (es && es[0] == '1') ? 1 : 0;
        // LBM_STAGED_TEST_EXPIRE=1 (tests only): the staged kernel's waits
        // expire, which must surface as LBM_ERR_TIMEOUT
        // LBM_PAIR=0 keeps the single-node stream-collide kernel where the
        // two-node one applies (same results bit for bit)
        const char *ep = std::getenv("LBM_PAIR");
        p.pair = (ep && ep[0] == '0') ? 0 : 1;
        const char *ex = std::getenv("LBM_STAGED_TEST_EXPIRE");
        p.stage_expire_test = (ex && ex[0] == '1') ? 1 : 0;
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d.device);
        p.nsm = sms;
    }
    p.eq = d.equilibrium;
    p.inlet_parabolic = d.inlet_profile == LBM_INLET_PARABOLIC;
    p.has_force = d.has_force ? 1 : 0;
    p.refill = d.refill;
    p.zouhe = d.edge_rule == LBM_EDGE_RULE_ZOUHE;
    p.tau = d.tau;
    p.omega = 1.0 / d.tau;
    p.rho0 = d.rho0;
    p.u_in = d.u_in;
    for (int k = 0; k < 3; ++k) {
        p.g[k] = d.has_force ? d.force[k] : 0.0;
        p.gf[k] = (float)p.g[k];
        p.gravity[k] = d.gravity[k];
    }
    p.omegaf = (float)p.omega;
    p.rho0f = (float)d.rho0;
    p.inv_rho0f = 1.0f / p.rho0f;
    p.keepf = 1.0f - p.omegaf;
    p.u_inf = (float)d.u_in;
    p.nb = 0;
    D->series_cap = d.series_capacity > 0 ? d.series_capacity : 8192;
    p.series_cap = D->series_cap;

    auto bail = [&](int rc) {
        lbm_destroy_domain(D);
        return rc;
    };
    const size_t N = (size_t)p.N;
    int rc;
    for (int k = 0; k < 2; ++k) {
        if ((rc = alloc_into(D, &D->pop[k], N * D->Q * D->Ssize, nullptr))) return bail(rc);
        // moments near bodies: FP64 (rho, u) in the FP64 mode, float4 (rho - 1, u)
        // in link mode; serving solves take them from the collided populations
        const size_t macb = d.precision == LBM_FP64 ? N * 4 * D->Csize : (p.linkmode ? N * 16 : 256);
        if ((rc = alloc_into(D, &D->mac[k], macb, nullptr))) return bail(rc);
        if ((rc = alloc_t(D, &D->owner[k], N, nullptr))) return bail(rc);
    }
    if ((rc = alloc_t(D, &D->flags, N, nullptr))) return bail(rc);
    if ((rc = alloc_t(D, &D->counters, N_COUNTERS, nullptr))) return bail(rc);
    {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d.device);
        // one block per multiprocessor for the side-stream kernels: measured
        // against 2 and 3, the stream-collide pass beside them loses least
        int per = 1;
        if (const char *ev = std::getenv("LBM_SIDE_BLOCKS_PER_SM")) per = std::max(1, std::atoi(ev));
        D->side_blocks = std::max(1, sms) * per;
        // LBM_SIDE_SERIAL=1: surface kernels before k_bulk on one stream
        const char *es = std::getenv("LBM_SIDE_SERIAL");
        D->side_serial = es && es[0] == '1';
    }
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    // high priority: blocks of the short side-stream kernels are dispatched
    // as soon as bulk-kernel blocks retire, instead of after the whole grid
    if ((e = cudaStreamCreateWithPriority(&D->s2, cudaStreamNonBlocking, prio_hi)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&D->ev_prep, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&D->ev_links, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&D->ev_side, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&D->sio, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&D->up_ev[0], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&D->up_ev[1], cudaEventDisableTiming)) != cudaSuccess)
        return bail(fail(LBM_ERR_CUDA, std::string("stream/event creation: ") + cudaGetErrorString(e)));
    for (int k = 0; k < lbm_domain::N_STEP_EV; ++k) {
        if ((e = cudaEventCreateWithFlags(&D->step_ev[k], cudaEventDisableTiming)) != cudaSuccess)
            return bail(fail(LBM_ERR_CUDA, std::string("event creation: ") + cudaGetErrorString(e)));
        D->step_ev_t[k] = -1;
    }
    if ((e = launch_flags_full(D->Q, p, D->owner[0], D->flags, D->s)) != cudaSuccess)
        return bail(fail(LBM_ERR_CUDA, std::string("flags: ") + cudaGetErrorString(e)));
    if ((rc = init_populations(D))) return bail(rc);
    if ((e = cudaStreamSynchronize(D->s)) != cudaSuccess)
        return bail(fail(LBM_ERR_CUDA, std::string("create: ") + cudaGetErrorString(e)));
    *out = D;
    return LBM_OK;
}
} // namespace

int lbm_destroy_domain(lbm_domain *D) {
    if (!D) return LBM_OK;
    DEVICE_SCOPE(D->d.device);
    cudaStreamSynchronize(D->s);
    free_body_buffers(D);
    for (int k = 0; k < 2; ++k) {
        D->release(D->pop[k]);
        D->release(D->mac[k]);
        D->release(D->owner[k]);
    }
    D->release(D->flags);
    D->release(D->counters);
    for (cudaEvent_t e : D->ev) cudaEventDestroy(e);
    if (D->s2) {
        cudaStreamSynchronize(D->s2);
        cudaStreamDestroy(D->s2);
    }
    if (D->ev_prep) cudaEventDestroy(D->ev_prep);
    if (D->ev_links) cudaEventDestroy(D->ev_links);
    if (D->ev_side) cudaEventDestroy(D->ev_side);
    if (D->sio) {
        cudaStreamSynchronize(D->sio);
        cudaStreamDestroy(D->sio);
    }
    for (int k = 0; k < lbm_domain::N_STEP_EV; ++k)
        if (D->step_ev[k]) cudaEventDestroy(D->step_ev[k]);
    if (D->gexec) cudaGraphExecDestroy(D->gexec);
    for (int k = 0; k < 2 * lbm_domain::GRAPH_STEPS; ++k)
        if (D->gev[k]) cudaEventDestroy(D->gev[k]);
    if (D->scap) cudaStreamDestroy(D->scap);
    for (int k = 0; k < 2; ++k) {
        if (D->up_ev[k]) cudaEventDestroy(D->up_ev[k]);
        if (D->hbd_pin[k]) cudaFreeHost(D->hbd_pin[k]);
    }
    delete D;
    return LBM_OK;
}

namespace {

// the state lbm_create_domain leaves: no bodies, every node fluid, the
// initial populations (after a failure part-way through placing bodies)
void reset_to_no_bodies(lbm_domain *D) {
    cudaStreamSynchronize(D->s);
    free_body_buffers(D);
    D->p.nb = 0;
    D->p.me_stride = 0; // as created
    D->hb.clear();
    D->hbd.clear();
    D->graph_dirty = true;
    const size_t N = (size_t)D->p.N;
    for (int k = 0; k < 2; ++k) cudaMemsetAsync(D->owner[k], 0, N * sizeof(uint16_t), D->s);
    launch_flags_full(D->Q, D->p, D->owner[0], D->flags, D->s);
    init_populations(D);
    cudaStreamSynchronize(D->s);
}

int place_bodies(lbm_domain *D, const lbm_body *hb, int n);

} // namespace

int lbm_set_bodies(lbm_domain *D, const lbm_body *hb, int n) {
    if (!D || n < 0 || (n > 0 && !hb)) return fail(LBM_ERR_ARG, "invalid arguments");
    DEVICE_SCOPE(D->d.device);
    if (D->t != 0) return fail(LBM_ERR_STATE, "bodies can only be placed at t = 0");
    if (n > 65534) return fail(LBM_ERR_ARG, "at most 65534 bodies");
    int rc = validate_bodies(D, hb, n);
    if (rc) return rc;
    rc = place_bodies(D, hb, n);
    if (rc) { // out of memory (or a CUDA error) part-way: the domain goes back to no bodies
        const std::string msg = g_err;
        reset_to_no_bodies(D);
        g_err = msg;
    }
    return rc;
}

namespace {

int place_bodies(lbm_domain *D, const lbm_body *hb, int n) {
    int rc = LBM_OK;
    CK(cudaStreamSynchronize(D->s));
    free_body_buffers(D);
    D->graph_dirty = true;
    D->nb = n;
    D->p.nb = n;
    D->hb.assign(hb, hb + n);
    D->hbd.resize(n);
    long long loff = 0, aoff = 0, chunks = 0;
    for (int b = 0; b < n; ++b) {
        body_params(D, hb[b], D->hbd[b]);
        D->hbd[b].link_off = loff;
        D->hbd[b].apm_off = aoff;
        loff += D->hbd[b].link_cap;
        aoff += D->hbd[b].apm_cap;
        chunks += D->hbd[b].nchunks;
    }
    D->link_cap_total = loff;
    D->apm_cap_total = aoff;
    long long tiles_cap = 0;
    for (int b = 0; b < n; ++b) tiles_cap += (D->hbd[b].link_cap + LINK_THREADS - 1) / LINK_THREADS;
    D->p.me_stride = std::max<long long>(loff, 1);
    auto &T = D->body_allocs;
    const size_t nbx = (size_t)std::max(n, 1);
    if ((rc = alloc_t(D, &D->dbodies, nbx, &T))) return rc;
    if ((rc = alloc_t(D, &D->dmoving, nbx, &T))) return rc;
    if ((rc = alloc_t(D, &D->chunk_all, (size_t)std::max<long long>(chunks, 1), &T))) return rc;
    if ((rc = alloc_t(D, &D->chunk_mov, (size_t)std::max<long long>(chunks, 1), &T))) return rc;
    if ((rc = alloc_t(D, &D->chunk_cnt_apm, (size_t)std::max<long long>(chunks, 1), &T))) return rc;
    if ((rc = alloc_t(D, &D->chunk_cnt_link, (size_t)std::max<long long>(chunks, 1), &T))) return rc;
    // cut-link lists: FP64 mode and link mode (serving solves evaluate links
    // inside the boundary-node kernel); per-link contributions: FP64 mode
    const bool exact = D->prec == LBM_FP64;
    const bool lists = exact || D->p.linkmode;
    const size_t Lsz = lists ? (size_t)std::max<long long>(loff, 1) : 1;
    for (int k = 0; k < 2; ++k) {
        if ((rc = alloc_t(D, &D->Lcell[k], Lsz, &T))) return rc;
        if ((rc = alloc_t(D, &D->Ldir[k], Lsz, &T))) return rc;
        if ((rc = alloc_t(D, &D->Ldelta[k], Lsz, &T))) return rc;
        if ((rc = alloc_t(D, &D->link_cnt[k], nbx, &T))) return rc;
    }
    if ((rc = alloc_t(D, &D->me, (exact ? Lsz : 1) * ME_PER_LINK, &T))) return rc;
    if ((rc = alloc_t(D, &D->apm_cell, (size_t)std::max<long long>(aoff, 1), &T))) return rc;
    if ((rc = alloc_t(D, &D->apm_sign, (size_t)std::max<long long>(aoff, 1), &T))) return rc;
    if ((rc = alloc_t(D, &D->apm_cnt, nbx, &T))) return rc;
    if ((rc = alloc_t(D, &D->imp_prev, nbx * 6, &T))) return rc; // zero: no displacement before t = 0
    if (D->p.free_scheme == LBM_FREE_PREDICTOR) {
        if ((rc = alloc_t(D, &D->apm_pred_cell, (size_t)std::max<long long>(aoff, 1), &T))) return rc;
        if ((rc = alloc_t(D, &D->apm_pred_sign, (size_t)std::max<long long>(aoff, 1), &T))) return rc;
        if ((rc = alloc_t(D, &D->apm_pred_cnt, nbx, &T))) return rc;
    }
    if ((rc = alloc_t(D, &D->series, (size_t)D->series_cap * nbx * SERIES_ROW, &T))) return rc;
    if ((rc = alloc_t(D, &D->poses, nbx * POSE_STRIDE, &T))) return rc;
    if ((rc = alloc_t(D, &D->link_pre, nbx + 1, &T))) return rc;
    if ((rc = alloc_t(D, &D->tile_pre, nbx + 1, &T))) return rc;
    if ((rc = alloc_t(D, &D->acc, nbx * SERIES_ROW, &T))) return rc;
    D->chg_cap = std::max<long long>(aoff, 1);
    if ((rc = alloc_t(D, &D->chg_cnt, 1, &T))) return rc;
    if ((rc = alloc_t(D, &D->chg_cell, (size_t)D->chg_cap, &T))) return rc;
    if ((rc = alloc_t(D, &D->chg_val, (size_t)D->chg_cap, &T))) return rc;
    // boundary nodes of a body lie in the shell R < |x - X| <= R + sqrt(2):
    // link_cap / (Q - 1) bounds their number (see link_capacity)
    long long bns = 0, bnm = 0;
    for (int b = 0; b < n; ++b) {
        const long long nodes = D->hbd[b].link_cap / (D->Q - 1) + 64;
        bns += nodes;
        if (D->hbd[b].moving) bnm += nodes;
    }
    D->bn_static_cap = std::max<long long>(bns, 1);
    D->bn_mov_cap = std::max<long long>(bns, 1); // bodies may start moving later
    (void)bnm;
    if ((rc = alloc_t(D, &D->bn_static, (size_t)D->bn_static_cap, &T))) return rc;
    if ((rc = alloc_t(D, &D->bn_mov[0], (size_t)D->bn_mov_cap, &T))) return rc;
    if ((rc = alloc_t(D, &D->bn_mov[1], (size_t)D->bn_mov_cap, &T))) return rc;
    if ((rc = alloc_t(D, &D->bn_cnt, 3, &T))) return rc;
    D->bnd_grid = (int)std::max<long long>(1, std::min<long long>(D->side_blocks, (bns + 7) / 8));
    D->bnd_grid_full = (int)std::max<long long>(1, std::min<long long>(16ll * D->p.nsm, (bns + 7) / 8));
    D->lists_dirty = true;
    long long maxcnt = 0;
    for (int b = 0; b < n; ++b) maxcnt = std::max(maxcnt, D->hbd[b].link_cap);
    (void)maxcnt;
    D->links_grid = (int)std::max<long long>(1, std::min<long long>(16 * 152, tiles_cap));
    if ((rc = upload_bodies(D))) return rc;

    // solid owners at t = 0, flags, links (both buffers), initial state
    const size_t N = (size_t)D->p.N;
    CK(cudaMemsetAsync(D->owner[0], 0, N * sizeof(uint16_t), D->s));
    CK(launch_prep(D->p, D->dbodies, D->link_cnt[0], D->link_pre, D->tile_pre, D->poses, 0, nullptr, nullptr, nullptr,
                   nullptr, nullptr, D->s));
    GeomArgs g = geom_args(D, false);
    CK(launch_raster(D->Q, D->p, g, D->owner[0], 0, D->s));
    CK(cudaMemcpyAsync(D->owner[1], D->owner[0], N * sizeof(uint16_t), cudaMemcpyDeviceToDevice, D->s));
    CK(launch_flags_full(D->Q, D->p, D->owner[0], D->flags, D->s));
    if (D->p.linkmode) CK(launch_macband(D->p, g, D->s)); // kept moments around every body
    if (lists) {
        CK(launch_geom_b(D->Q, D->p, g, D->s));
        CK(launch_geom_c(D->Q, D->p, g, D->s));
        const size_t L = Lsz;
        CK(cudaMemcpyAsync(D->Lcell[1], D->Lcell[0], L * sizeof(uint32_t), cudaMemcpyDeviceToDevice, D->s));
        CK(cudaMemcpyAsync(D->Ldir[1], D->Ldir[0], L, cudaMemcpyDeviceToDevice, D->s));
        CK(cudaMemcpyAsync(D->Ldelta[1], D->Ldelta[0], L * sizeof(double), cudaMemcpyDeviceToDevice, D->s));
        CK(cudaMemcpyAsync(D->link_cnt[1], D->link_cnt[0], nbx * sizeof(long long), cudaMemcpyDeviceToDevice,
                           D->s));
    }
    CK(launch_prep(D->p, D->dbodies, D->link_cnt[0], D->link_pre, D->tile_pre, D->poses, 0, nullptr, nullptr, nullptr,
                   nullptr, nullptr, D->s));
    D->prep_dirty = false;
    if ((rc = init_populations(D))) return rc;
    CK(cudaStreamSynchronize(D->s));
    return LBM_OK;
}

} // namespace

int lbm_update_bodies(lbm_domain *D, const lbm_body *hb, int n) {
    if (!D || !hb || n != D->nb) return fail(LBM_ERR_ARG, "update needs the same number of bodies");
    DEVICE_SCOPE(D->d.device);
    if (D->n_free) return fail(LBM_ERR_STATE, "free bodies move with the flow; their kinematics cannot be set");
    for (int b = 0; b < n; ++b) {
        const lbm_body &o = D->hb[b], &v = hb[b];
        if (o.shape != v.shape || o.R != v.R || o.halfway != v.halfway)
            return fail(LBM_ERR_ARG, "shape, radius and halfway cannot change");
        for (int a = 0; a < 3; ++a) {
            double xo = o.X0[a] + (double)(D->t - o.t0) * o.U[a];
            double xv = v.X0[a] + (double)(D->t - v.t0) * v.U[a];
            if (std::fabs(xo - xv) > 1e-9) return fail(LBM_ERR_ARG, "the pose at the current step may not jump");
            if (!D->p.per[a] && v.U[a] != 0.0 && !(a == 2 && along_z(v.shape)))
                return fail(LBM_ERR_ARG, "bodies may not translate along a non-periodic axis");
        }
    }
    // no host synchronisation: the new records reach the device in stream
    // order after the steps already enqueued (upload_body_array)
    const int cur = (int)(D->t & 1), nxt = cur ^ 1;
    bool maps_changed = false;
    for (int b = 0; b < n; ++b) {
        bool was = D->hbd[b].moving != 0;
        BodyDev nb = D->hbd[b];
        BodyDev tmp;
        body_params(D, hb[b], tmp);
        nb.moving = tmp.moving;
        for (int a = 0; a < 3; ++a) {
            nb.X0[a] = hb[b].X0[a];
            nb.U[a] = hb[b].U[a];
            nb.W[a] = hb[b].W[a];
        }
        nb.t0 = hb[b].t0;
        D->hbd[b] = nb;
        D->hb[b] = hb[b];
        if (was != (nb.moving != 0)) maps_changed = true;
        if (was && !nb.moving) { // static from now on: both link buffers must hold the links of t
            const size_t off = (size_t)nb.link_off, cap = (size_t)nb.link_cap;
            CK(cudaMemcpyAsync(D->Lcell[nxt] + off, D->Lcell[cur] + off, cap * sizeof(uint32_t), cudaMemcpyDeviceToDevice, D->s));
            CK(cudaMemcpyAsync(D->Ldir[nxt] + off, D->Ldir[cur] + off, cap, cudaMemcpyDeviceToDevice, D->s));
            CK(cudaMemcpyAsync(D->Ldelta[nxt] + off, D->Ldelta[cur] + off, cap * sizeof(double), cudaMemcpyDeviceToDevice, D->s));
            CK(cudaMemcpyAsync(D->link_cnt[nxt] + b, D->link_cnt[cur] + b, sizeof(long long), cudaMemcpyDeviceToDevice, D->s));
            CK(cudaMemcpyAsync(D->owner[nxt], D->owner[cur], (size_t)D->p.N * sizeof(uint16_t), cudaMemcpyDeviceToDevice, D->s));
        }
    }
    D->prep_dirty = true;
    if (maps_changed) D->lists_dirty = true;
    if (maps_changed) return upload_bodies(D);
    return upload_body_array(D);
}

namespace {
// Capture GRAPH_STEPS steps from the current (even) step into D->gexec.  The
// captured steps do not run: D->t is restored.
int capture_graph(lbm_domain *D) {
    if (D->gexec) {
        cudaGraphExecDestroy(D->gexec);
        D->gexec = nullptr;
    }
    for (int k = 0; k < 2 * lbm_domain::GRAPH_STEPS; ++k)
        if (!D->gev[k]) CK(cudaEventCreate(&D->gev[k]));
    if (!D->scap && cudaStreamCreateWithFlags(&D->scap, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        D->graph_failed = true;
        return LBM_OK;
    }
    const int64_t t0 = D->t;
    cudaStream_t user = D->s;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(D->scap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        (void)cudaGetLastError();
        D->graph_failed = true;
        return LBM_OK;
    }
    D->s = D->scap; // the steps are recorded, not run; the graph is launched into the domain's stream
    D->capturing = true;
    D->cap_k = 0;
    int rc = LBM_OK;
    for (int k = 0; k < lbm_domain::GRAPH_STEPS && rc == LBM_OK; ++k) rc = do_step(D);
    cudaError_t e = cudaStreamEndCapture(D->scap, &graph);
    D->s = user;
    D->capturing = false;
    D->t = t0;
    // the side-stream kernels keep their high priority inside the graph
    if (rc == LBM_OK && e == cudaSuccess)
        e = cudaGraphInstantiateWithFlags(&D->gexec, graph, cudaGraphInstantiateFlagUseNodePriority);
    if (graph) cudaGraphDestroy(graph);
    if (rc != LBM_OK || e != cudaSuccess) {
        (void)cudaGetLastError();
        D->gexec = nullptr;
        D->graph_failed = true; // plain launches from now on
        return rc != LBM_OK ? rc : fail(LBM_ERR_CUDA, std::string("step graph: ") + cudaGetErrorString(e));
    }
    D->graph_dirty = false;
    return LBM_OK;
}
} // namespace

int lbm_step(lbm_domain *D, int n) {
    if (!D || n < 0) return fail(LBM_ERR_ARG, "invalid arguments");
    DEVICE_SCOPE(D->d.device);
    const int G = lbm_domain::GRAPH_STEPS;
    for (int k = 0; k < n;) {
        const bool graph = !D->graph_failed && !D->prep_dirty && !D->lists_dirty && (D->t & 1) == 0 && n - k >= G;
        if (graph && (D->graph_dirty || !D->gexec)) {
            int rc = capture_graph(D);
            if (rc && !D->graph_failed) return rc;
        }
        if (graph && D->gexec) {
            CK(cudaGraphLaunch(D->gexec, D->s));
            D->t += G;
            k += G;
            if (D->timing) D->g_timed = true;
            continue;
        }
        int rc = do_step(D);
        if (rc) return rc;
        ++k;
    }
    if (n > 0) { // the steps up to D->t are done when this event is
        const int k = D->step_ev_next;
        CK(cudaEventRecord(D->step_ev[k], D->s));
        D->step_ev_t[k] = D->t;
        D->step_ev_next = (k + 1) % lbm_domain::N_STEP_EV;
    }
    return LBM_OK;
}

int lbm_prepare_graph(lbm_domain *D) {
    if (!D) return fail(LBM_ERR_ARG, "null domain");
    DEVICE_SCOPE(D->d.device);
    if (D->graph_failed) return LBM_OK; // this domain runs plain launches
    if (D->prep_dirty || D->lists_dirty)
        return fail(LBM_ERR_STATE, "the step graph is recorded after the first step of a body set");
    if (D->gexec && !D->graph_dirty) return LBM_OK;
    // a graph starts at an even step (the population buffers alternate with
    // the step parity; the kernels read the step index on the device)
    const int64_t t = D->t;
    D->t = t & ~(int64_t)1;
    const int rc = capture_graph(D);
    D->t = t;
    if (rc && !D->graph_failed) return rc;
    return LBM_OK;
}

namespace {
// Makes D->sio wait until the steps before `t_end` are complete: on the
// earliest recorded step event that covers them, else on all of D->s.
int wait_steps(lbm_domain *D, int64_t t_end) {
    int best = -1;
    for (int k = 0; k < lbm_domain::N_STEP_EV; ++k)
        if (D->step_ev_t[k] >= t_end && (best < 0 || D->step_ev_t[k] < D->step_ev_t[best])) best = k;
    if (best >= 0) {
        CK(cudaStreamWaitEvent(D->sio, D->step_ev[best], 0));
    } else {
        CK(cudaStreamSynchronize(D->s));
    }
    return LBM_OK;
}
} // namespace

int lbm_get_series(lbm_domain *D, int64_t first, int64_t count, double *out) {
    if (!D || !out || first < 0 || count < 0) return fail(LBM_ERR_ARG, "invalid arguments");
    DEVICE_SCOPE(D->d.device);
    if (first + count > D->t) return fail(LBM_ERR_ARG, "rows beyond the current step");
    if (first < D->t - D->series_cap) return fail(LBM_ERR_ARG, "rows older than the series ring");
    if (D->nb == 0 || count == 0) return LBM_OK;
    int wrc = wait_steps(D, first + count);
    if (wrc) return wrc;
    {
        // sticky flags: a flag a later step (still running) sets may show up
        // here already
        unsigned long long flags[3] = {0, 0, 0}; // unstable, timeout, free body out of range
        CK(cudaMemcpyAsync(flags, D->counters + 5, sizeof(flags), cudaMemcpyDeviceToHost, D->sio));
        CK(cudaStreamSynchronize(D->sio));
        if (flags[1]) return fail(LBM_ERR_TIMEOUT, "a stream-collide block gave up waiting for its staged rows");
        if (flags[0])
            return fail(LBM_ERR_UNSTABLE, "the solve went unstable (NaN or |u| > 0.3 at a boundary node, or a "
                                          "non-finite force)");
        if (flags[2])
            return fail(LBM_ERR_STATE, "a free body came within 2 cells of a non-periodic face or moved faster "
                                       "than 0.25 at its surface");
    }
    const size_t row = (size_t)D->nb * SERIES_ROW;
    int64_t done = 0;
    while (done < count) {
        int64_t r = (first + done) % D->series_cap;
        int64_t m = std::min<int64_t>(count - done, D->series_cap - r);
        CK(cudaMemcpyAsync(out + done * row, D->series + r * row, m * row * sizeof(double), cudaMemcpyDeviceToHost,
                           D->sio));
        D->d2h += (long long)(m * row * sizeof(double));
        done += m;
    }
    CK(cudaStreamSynchronize(D->sio));
    return LBM_OK;
}

int lbm_get_force_torque(lbm_domain *D, int64_t first, int64_t count, int kind, double *out) {
    if (!D || !out) return fail(LBM_ERR_ARG, "invalid arguments");
    if (kind < LBM_FT_STATIC || kind > LBM_FT_IMPULSIVE) return fail(LBM_ERR_ARG, "unknown force kind");
    std::vector<double> raw((size_t)std::max<int64_t>(count, 0) * D->nb * SERIES_ROW);
    int rc = lbm_get_series(D, first, count, raw.data());
    if (rc) return rc;
    for (int64_t r = 0; r < count * D->nb; ++r) {
        const double *s = raw.data() + r * SERIES_ROW;
        double *o = out + r * 6;
        for (int k = 0; k < 6; ++k) {
            if (kind == LBM_FT_STATIC) o[k] = s[k];
            else if (kind == LBM_FT_LATTICE) o[k] = s[k] + s[6 + k];
            else if (kind == LBM_FT_MOVING) o[k] = s[12 + k];
            else o[k] = s[6 + k];
        }
    }
    return LBM_OK;
}

int lbm_get_populations(lbm_domain *D, double *out) {
    if (!D || !out) return fail(LBM_ERR_ARG, "invalid arguments");
    DEVICE_SCOPE(D->d.device);
    const size_t n = (size_t)D->p.N * D->Q;
    void *tmp = D->alloc(n * sizeof(double));
    if (!tmp) return fail(LBM_ERR_OOM, "temporary export buffer");
    cudaError_t e = launch_export(D->Q, D->prec, D->p, D->pop[D->t & 1], (double *)tmp, D->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(D->s);
    if (e == cudaSuccess) e = cudaMemcpy(out, tmp, n * sizeof(double), cudaMemcpyDeviceToHost);
    D->release(tmp);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("populations: ") + cudaGetErrorString(e));
    return LBM_OK;
}

// cells per staging chunk of lbm_set_populations / lbm_get_macros
constexpr long long IO_CHUNK = 1ll << 22;

int lbm_set_populations(lbm_domain *D, const double *f) {
    if (!D || !f) return fail(LBM_ERR_ARG, "invalid arguments");
    DEVICE_SCOPE(D->d.device);
    const long long N = D->p.N, chunk = std::min(N, IO_CHUNK);
    double *stage = (double *)D->alloc((size_t)chunk * D->Q * sizeof(double));
    if (!stage) return fail(LBM_ERR_OOM, "temporary staging buffer");
    cudaError_t e = cudaStreamSynchronize(D->s);
    for (long long c0 = 0; c0 < N && e == cudaSuccess; c0 += chunk) {
        const long long n = std::min(chunk, N - c0);
        for (int i = 0; i < D->Q && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync(stage + (long long)i * n, f + (long long)i * N + c0, (size_t)n * sizeof(double),
                                cudaMemcpyHostToDevice, D->s);
        if (e == cudaSuccess)
            e = launch_load(D->Q, D->prec, D->p, stage, c0, n, D->pop[D->t & 1], D->mac[D->t & 1], D->flags, D->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(D->s); // the stage is reused by the next chunk
    }
    D->release(stage);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("set populations: ") + cudaGetErrorString(e));
    D->h2d += N * D->Q * (long long)sizeof(double);
    return LBM_OK;
}

int lbm_get_macros(lbm_domain *D, double *out) {
    if (!D || !out) return fail(LBM_ERR_ARG, "invalid arguments");
    DEVICE_SCOPE(D->d.device);
    const long long N = D->p.N, chunk = std::min(N, IO_CHUNK);
    double *stage = (double *)D->alloc((size_t)chunk * 4 * sizeof(double));
    if (!stage) return fail(LBM_ERR_OOM, "temporary staging buffer");
    cudaError_t e = cudaSuccess;
    for (long long c0 = 0; c0 < N && e == cudaSuccess; c0 += chunk) {
        const long long n = std::min(chunk, N - c0);
        e = launch_macros(D->Q, D->prec, D->p, D->pop[D->t & 1], D->owner[D->t & 1], c0, n, stage, D->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(D->s);
        for (int k = 0; k < 4 && e == cudaSuccess; ++k)
            e = cudaMemcpy(out + (long long)k * N + c0, stage + (long long)k * n, (size_t)n * sizeof(double),
                           cudaMemcpyDeviceToHost);
    }
    D->release(stage);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("macros: ") + cudaGetErrorString(e));
    D->d2h += N * 4 * (long long)sizeof(double);
    return LBM_OK;
}

int lbm_get_body_state(lbm_domain *D, double *out) {
    if (!D || (D->nb && !out)) return fail(LBM_ERR_ARG, "invalid arguments");
    DEVICE_SCOPE(D->d.device);
    if (D->nb == 0) return LBM_OK;
    std::vector<BodyDev> hb((size_t)D->nb);
    CK(cudaStreamSynchronize(D->s));
    CK(cudaMemcpy(hb.data(), D->dbodies, sizeof(BodyDev) * D->nb, cudaMemcpyDeviceToHost));
    D->d2h += (long long)(sizeof(BodyDev) * D->nb);
    for (int b = 0; b < D->nb; ++b) {
        const double dt = (double)(D->t - hb[b].t0);
        for (int a = 0; a < 3; ++a) {
            volatile double step = dt * hb[b].U[a]; // no contraction with the add below
            out[9 * b + a] = hb[b].X0[a] + step;
            out[9 * b + 3 + a] = hb[b].U[a];
            out[9 * b + 6 + a] = hb[b].W[a];
        }
    }
    return LBM_OK;
}

int lbm_get_solid(lbm_domain *D, int32_t *out) {
    if (!D || !out) return fail(LBM_ERR_ARG, "invalid arguments");
    DEVICE_SCOPE(D->d.device);
    const size_t N = (size_t)D->p.N;
    std::vector<uint16_t> o(N);
    CK(cudaStreamSynchronize(D->s));
    CK(cudaMemcpy(o.data(), D->owner[D->t & 1], N * sizeof(uint16_t), cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < N; ++k) out[k] = (int32_t)o[k] - 1;
    return LBM_OK;
}

// ---- state snapshots --------------------------------------------------------
//
// Layout: SnapHeader, the bodies as the host holds them (lbm_body, BodyDev),
// the sizes of the device buffers, then their contents in allocation order.
namespace {
struct SnapHeader {
    char magic[8];
    int32_t lattice, precision, nx, ny, nz, nb;
    int64_t t;
    int32_t prep_dirty, lists_dirty;
    int64_t nbuf;
};
constexpr char SNAP_MAGIC[8] = {'L', 'B', 'M', 'S', 'N', 'A', 'P', '1'};
} // namespace

int64_t lbm_state_bytes(const lbm_domain *D) {
    if (!D) return -1;
    int64_t b = (int64_t)sizeof(SnapHeader) + (int64_t)D->nb * (int64_t)(sizeof(lbm_body) + sizeof(BodyDev));
    b += (int64_t)D->state_bufs.size() * (int64_t)sizeof(int64_t);
    for (const auto &e : D->state_bufs) b += (int64_t)e.second;
    return b;
}

int lbm_save_state(lbm_domain *D, void *out, int64_t cap) {
    if (!D || !out) return fail(LBM_ERR_ARG, "invalid arguments");
    DEVICE_SCOPE(D->d.device);
    const int64_t need = lbm_state_bytes(D);
    if (cap < need) return fail(LBM_ERR_ARG, "snapshot buffer smaller than lbm_state_bytes");
    CK(cudaStreamSynchronize(D->s));
    char *p = (char *)out;
    SnapHeader h{};
    std::memcpy(h.magic, SNAP_MAGIC, 8);
    h.lattice = D->Q;
    h.precision = D->prec;
    h.nx = D->p.nx;
    h.ny = D->p.ny;
    h.nz = D->p.nz;
    h.nb = D->nb;
    h.t = D->t;
    h.prep_dirty = D->prep_dirty ? 1 : 0;
    h.lists_dirty = D->lists_dirty ? 1 : 0;
    h.nbuf = (int64_t)D->state_bufs.size();
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    if (D->nb) {
        std::memcpy(p, D->hb.data(), sizeof(lbm_body) * D->nb);
        p += sizeof(lbm_body) * D->nb;
        std::memcpy(p, D->hbd.data(), sizeof(BodyDev) * D->nb);
        p += sizeof(BodyDev) * D->nb;
    }
    for (const auto &e : D->state_bufs) {
        const int64_t n = (int64_t)e.second;
        std::memcpy(p, &n, sizeof(n));
        p += sizeof(n);
    }
    for (const auto &e : D->state_bufs) {
        CK(cudaMemcpy(p, e.first, e.second, cudaMemcpyDeviceToHost));
        p += e.second;
        D->d2h += (long long)e.second;
    }
    return LBM_OK;
}

int lbm_load_state(lbm_domain *D, const void *in, int64_t size) {
    if (!D || !in || size < (int64_t)sizeof(SnapHeader)) return fail(LBM_ERR_ARG, "invalid arguments");
    DEVICE_SCOPE(D->d.device);
    const char *p = (const char *)in;
    SnapHeader h;
    std::memcpy(&h, p, sizeof(h));
    p += sizeof(h);
    if (std::memcmp(h.magic, SNAP_MAGIC, 8) != 0) return fail(LBM_ERR_ARG, "not a domain snapshot");
    if (h.lattice != D->Q || h.precision != D->prec || h.nx != D->p.nx || h.ny != D->p.ny || h.nz != D->p.nz ||
        h.nb != D->nb || h.nbuf != (int64_t)D->state_bufs.size() || size != lbm_state_bytes(D))
        return fail(LBM_ERR_ARG, "the snapshot belongs to a domain of another shape or body set");
    std::vector<lbm_body> hb((size_t)D->nb);
    std::vector<BodyDev> hbd((size_t)D->nb);
    if (D->nb) {
        std::memcpy(hb.data(), p, sizeof(lbm_body) * D->nb);
        p += sizeof(lbm_body) * D->nb;
        std::memcpy(hbd.data(), p, sizeof(BodyDev) * D->nb);
        p += sizeof(BodyDev) * D->nb;
    }
    for (size_t k = 0; k < D->state_bufs.size(); ++k) {
        int64_t n;
        std::memcpy(&n, p, sizeof(n));
        p += sizeof(n);
        if (n != (int64_t)D->state_bufs[k].second)
            return fail(LBM_ERR_ARG, "the snapshot's buffers do not match this domain's");
    }
    CK(cudaStreamSynchronize(D->s));
    if (D->nb) { // the host's body records and the body maps they imply, then the device state over them
        D->hb = hb;
        D->hbd = hbd;
        int rc = upload_bodies(D);
        if (rc) return rc;
    }
    for (const auto &e : D->state_bufs) {
        CK(cudaMemcpy(e.first, p, e.second, cudaMemcpyHostToDevice));
        p += e.second;
        D->h2d += (long long)e.second;
    }
    D->t = h.t;
    D->prep_dirty = h.prep_dirty != 0;
    D->lists_dirty = h.lists_dirty != 0;
    D->graph_dirty = true;
    D->ev_used = 0;
    D->g_timed = false;
    for (int k = 0; k < lbm_domain::N_STEP_EV; ++k) D->step_ev_t[k] = -1;
    return LBM_OK;
}

int lbm_get_stats(lbm_domain *D, lbm_stats *out) {
    if (!D || !out) return fail(LBM_ERR_ARG, "invalid arguments");
    DEVICE_SCOPE(D->d.device);
    std::memset(out, 0, sizeof(*out));
    CK(cudaStreamSynchronize(D->s));
    unsigned long long c[N_COUNTERS] = {};
    CK(cudaMemcpy(c, D->counters, sizeof(c), cudaMemcpyDeviceToHost));
    out->step = D->t;
    out->cells = D->p.N;
    out->fallback_links = (int64_t)c[0];
    out->covered = (int64_t)c[1];
    out->uncovered = (int64_t)c[2];
    out->device_bytes = (int64_t)D->bytes;
    out->timeouts = (int64_t)c[6];
    out->unstable = (int64_t)c[5];
    out->extrapolated = (int64_t)c[8];
    out->h2d_bytes = D->h2d;
    out->d2h_bytes = D->d2h;
    if (D->nb && D->prec != LBM_FP64 && !D->p.linkmode && D->t > 0) {
        out->links = (int64_t)c[4]; // counted by the boundary-node kernel in the last step
    } else if (D->nb) {
        std::vector<long long> lc(D->nb);
        CK(cudaMemcpy(lc.data(), D->link_cnt[D->t & 1], sizeof(long long) * D->nb, cudaMemcpyDeviceToHost));
        for (long long v : lc) out->links += v;
    }
    std::vector<int32_t> s((size_t)D->p.N);
    int rc = lbm_get_solid(D, s.data());
    if (rc) return rc;
    for (int32_t v : s) out->fluid_cells += v < 0;
    return LBM_OK;
}

int64_t lbm_time(const lbm_domain *D) { return D ? D->t : -1; }

int lbm_set_stream(lbm_domain *D, void *stream) {
    if (!D) return fail(LBM_ERR_ARG, "null domain");
    CK(cudaStreamSynchronize(D->s));
    D->s = (cudaStream_t)stream;
    return LBM_OK;
}

int lbm_set_kernel_timing(lbm_domain *D, int enable) {
    if (!D) return fail(LBM_ERR_ARG, "null domain");
    DEVICE_SCOPE(D->d.device);
    CK(cudaStreamSynchronize(D->s));
    if (D->timing != (enable != 0)) D->graph_dirty = true; // the graph holds the timing events or not
    D->timing = enable != 0;
    D->ev_used = 0;
    D->g_timed = false;
    return LBM_OK;
}

int lbm_kernel_time(lbm_domain *D, int64_t *launches, double *total_ms) {
    if (!D || !launches || !total_ms) return fail(LBM_ERR_ARG, "invalid arguments");
    DEVICE_SCOPE(D->d.device);
    CK(cudaStreamSynchronize(D->s));
    double tot = 0.0;
    for (size_t k = 0; k + 1 < D->ev_used; k += 2) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, D->ev[k], D->ev[k + 1]));
        tot += ms;
    }
    int64_t n = (int64_t)(D->ev_used / 2);
    if (D->g_timed) { // the bulk kernels of the last graph replay
        for (int k = 0; k < lbm_domain::GRAPH_STEPS; ++k) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, D->gev[2 * k], D->gev[2 * k + 1]));
            tot += ms;
        }
        n += lbm_domain::GRAPH_STEPS;
    }
    *launches = n;
    *total_ms = tot;
    D->ev_used = 0;
    D->g_timed = false;
    return LBM_OK;
}

int lbm_launches_per_step(const lbm_domain *D, int *out) {
    if (!D || !out) return fail(LBM_ERR_ARG, "invalid arguments");
    if (D->prec != LBM_FP64 && D->nb)
        *out = 3 + (D->n_moving ? 3 : (D->prep_dirty ? 1 : 0)); // bulk, bnd, finish (+ prep, geometry)
    else
        *out = 1 + (D->nb ? 2 : 0) + (D->n_moving ? 4 : 0) + (D->nb && D->prep_dirty && !D->n_moving ? 1 : 0);
    if (D->n_free) *out += 1; // free-body update
    if (step_scheme(D) != LBM_FREE_EXPLICIT) // poses of t+1, second end-of-step pass, geometry after the force
        *out += D->prec == LBM_FP64 ? 4 : (D->p.free_scheme == LBM_FREE_PREDICTOR ? 3 : 2);
    if (D->p.zouhe) *out += 1; // Zou-He face nodes
    return LBM_OK;
}

} // extern "C"

// ---- serving: continuous batching ------------------------------------------
//
// A batch holds up to max_slots solves, each a complete lbm_domain (reduced
// precision, static bodies) created on the batch's stream and allocator.  The
// device keeps a table of SolveDev records (one per slot) that the batched
// kernels read; for each (lattice, precision) group the host keeps a block
// work table (slot, first cell) for the bulk kernel and a prefix of the
// boundary-node counts for the boundary-node kernel.  A tick is: fork; the
// stream-collide passes (one launch per resident solve on parallel branches
// for up to PER_SOLVE_MAX solves, else the batched kernel of every group) and
// the boundary-node kernels on the high-priority side stream (disjoint nodes,
// both read fhat(t)); join; one end-of-step kernel for every resident solve.  ticks_per_launch ticks are
// captured once into a CUDA graph, re-captured whenever the resident set
// changes.  Admission and release synchronise the batch stream, so the tables
// are never rewritten under a running graph.

struct lbm_batch {
    lbm_batch_desc d{};
    cudaStream_t s = nullptr, s2 = nullptr;
    bool own_s = false;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // extra capture streams: the bulk kernels of different groups run on
    // parallel branches of the tick graph (their solves are disjoint)
    static constexpr int NBRANCH = 7;
    cudaStream_t sb[NBRANCH] = {};
    cudaEvent_t ev_branch[NBRANCH] = {};
    int tpl = 32;
    int side_blocks = 0;
    int64_t used = 0;
    struct Slot {
        lbm_domain *D = nullptr;
        int64_t t_end = 0;
        long long nodes = 0;
        bool reported = false;
    };
    std::vector<Slot> slots;
    SolveDev *dsolves = nullptr;
    struct Group {
        int Q = 0, prec = 0, kind = 0, fm = 0;
        int4 *work = nullptr;
        int nwork = 0;
        int *slots = nullptr;
        long long *node_pre = nullptr;
        int nslots = 0;
        int grid = 0;
    };
    static constexpr int NGROUPS = 12; // lattice x storage x face mode
    Group g[NGROUPS];
    int *dall = nullptr;
    int nall = 0;
    std::vector<void *> table_allocs;
    cudaGraphExec_t exec = nullptr;
    bool dirty = true;
    // stream-collide launches per resident solve (up to PER_SOLVE_MAX solves)
    // instead of one batched kernel per group; LBM_BATCH_GROUPED=1 turns it off
    static constexpr int PER_SOLVE_MAX = 32;
    bool per_solve = true;

    void *alloc(size_t n) {
        if (n == 0) n = 256;
        void *ptr = nullptr;
        if (d.alloc) ptr = d.alloc(n, d.alloc_ctx);
        else if (cudaMalloc(&ptr, n) != cudaSuccess) ptr = nullptr;
        return ptr;
    }
    void release(void *ptr) {
        if (!ptr) return;
        if (d.free) d.free(ptr, d.alloc_ctx);
        else cudaFree(ptr);
    }
};

namespace {

// bulk kind of a solve (lbm_internal.h) and its group: lattice x kind x face mode
int bulk_kind(const lbm_domain *D) { return D->prec == LBM_FP16 ? BK_FP16 : BK_FP32; }
int group_of(const lbm_domain *D) { return ((D->Q == 19 ? 2 : 0) + bulk_kind(D)) * 3 + face_mode(D->p); }

// Device bytes lbm_create_domain + lbm_set_bodies request for this problem
// (the same sizes, in the same order, without allocating).
int domain_bytes(const lbm_domain_desc &d, const lbm_body *hb, int n, int64_t *bytes) {
    lbm_domain T;
    T.d = d;
    T.Q = d.lattice;
    T.prec = d.precision;
    T.p.nx = d.nx;
    T.p.ny = d.ny;
    T.p.nz = d.nz;
    T.p.N = (long long)d.nx * d.ny * d.nz;
    for (int a = 0; a < 3; ++a) T.p.per[a] = d.edge[2 * a] == LBM_EDGE_PERIODIC;
    int rc = validate_bodies(&T, hb, n);
    if (rc) return rc;
    const long long N = T.p.N;
    const long long S = d.precision == LBM_FP64 ? 8 : (d.precision == LBM_FP32 ? 4 : 2);
    const long long C = d.precision == LBM_FP64 ? 8 : 4;
    const long long cap = d.series_capacity > 0 ? d.series_capacity : 8192;
    long long b = 0;
    b += 2 * (N * T.Q * S + (d.precision == LBM_FP64 ? N * 4 * C : 256) + N * 2); // pop, mac, owner
    b += N + 8 * N_COUNTERS;                                                      // flags, counters
    const long long nbx = std::max(n, 1);
    long long loff = 0, aoff = 0, chunks = 0, bns = 0;
    for (int k = 0; k < n; ++k) {
        BodyDev o;
        body_params(&T, hb[k], o);
        loff += o.link_cap;
        aoff += o.apm_cap;
        chunks += o.nchunks;
        bns += o.link_cap / (T.Q - 1) + 64;
    }
    const long long ch = std::max<long long>(chunks, 1);
    const long long Lsz = d.precision == LBM_FP64 ? std::max<long long>(loff, 1) : 1;
    const long long A = std::max<long long>(aoff, 1);
    const long long B = std::max<long long>(bns, 1);
    b += nbx * (long long)sizeof(BodyDev) + nbx * 4;             // bodies, moving ids
    b += 2 * ch * 8 + 2 * ch * 4;                                // chunk maps, chunk counts
    b += 2 * (Lsz * 4 + Lsz * 1 + Lsz * 8 + nbx * 8);            // link lists and counts
    b += Lsz * ME_PER_LINK * 8;                                  // per-link contributions
    b += A * 4 + A * 1 + nbx * 8;                                // covered/uncovered lists
    b += nbx * 6 * 8;                                            // impulsive terms of the last displacement
    if (d.free_scheme == LBM_FREE_PREDICTOR) b += A * 4 + A * 1 + nbx * 8; // predicted lists
    b += cap * nbx * SERIES_ROW * 8 + nbx * POSE_STRIDE * 8;     // series, poses
    b += 2 * (nbx + 1) * 8 + nbx * SERIES_ROW * 8;               // prefixes, accumulators
    b += 8 + A * 4 + A * 1;                                      // flag-change list
    b += B * 4 * 3 + 3 * 8;                                      // boundary-node lists
    *bytes = b;
    return LBM_OK;
}

int batch_check_desc(const lbm_domain_desc &d, const lbm_body *hb, int n, int64_t steps) {
    if (steps < 1) return fail(LBM_ERR_ARG, "a served solve needs at least one step");
    if (d.precision != LBM_FP32 && d.precision != LBM_FP16)
        return fail(LBM_ERR_ARG, "served solves run in LBM_FP32 or LBM_FP16");
    if ((long long)d.nx * d.ny * d.nz >= (1ll << 31)) return fail(LBM_ERR_ARG, "a served solve has < 2^31 cells");
    if (n < 0 || (n > 0 && !hb)) return fail(LBM_ERR_ARG, "invalid body list");
    for (int k = 0; k < n; ++k)
        if (is_moving(hb[k])) return fail(LBM_ERR_ARG, "served solves take static bodies only");
    if (d.has_force) return fail(LBM_ERR_ARG, "served solves take no body force");
    if (d.edge_rule != LBM_EDGE_RULE_LINK) return fail(LBM_ERR_ARG, "served solves take the link edge rule");
    return LBM_OK;
}

void batch_free_tables(lbm_batch *B) {
    for (void *ptr : B->table_allocs) B->release(ptr);
    B->table_allocs.clear();
    for (auto &G : B->g) {
        G.work = nullptr;
        G.slots = nullptr;
        G.node_pre = nullptr;
        G.nwork = G.nslots = G.grid = 0;
    }
    B->dall = nullptr;
    B->nall = 0;
}

template <class T> int batch_upload(lbm_batch *B, T **dst, const std::vector<T> &v) {
    *dst = nullptr;
    if (v.empty()) return LBM_OK;
    void *ptr = B->alloc(v.size() * sizeof(T));
    if (!ptr) return fail(LBM_ERR_OOM, "batch table allocation failed");
    B->table_allocs.push_back(ptr);
    CK(cudaMemcpyAsync(ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, B->s));
    *dst = (T *)ptr;
    return LBM_OK;
}

// work tables of the resident unfinished solves, then the tick graph
int batch_rebuild(lbm_batch *B) {
    CK(cudaStreamSynchronize(B->s));
    batch_free_tables(B);
    if (B->exec) {
        cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
    }
    constexpr int NG = lbm_batch::NGROUPS;
    std::vector<int4> work[NG];
    std::vector<int> gslots[NG], all;
    std::vector<long long> pre[NG];
    for (int k = 0; k < NG; ++k) pre[k].push_back(0);
    for (int sl = 0; sl < (int)B->slots.size(); ++sl) {
        const auto &S = B->slots[sl];
        if (!S.D || S.D->t >= S.t_end) continue;
        const int gi = group_of(S.D);
        const int rows = S.D->p.ny * S.D->p.nz;
        for (int r = 0; r < rows; ++r)
            for (int x0 = 0; x0 < S.D->p.nx; x0 += BBULK_THREADS) work[gi].push_back(make_int4(sl, r, x0, 0));
        gslots[gi].push_back(sl);
        pre[gi].push_back(pre[gi].back() + S.nodes);
        all.push_back(sl);
    }
    int rc;
    for (int k = 0; k < NG; ++k) {
        auto &G = B->g[k];
        G.Q = k / 3 >= 2 ? 19 : 9;
        G.kind = (k / 3) % 2;
        G.fm = k % 3;
        G.prec = G.kind == BK_FP32 ? LBM_FP32 : LBM_FP16;
        if ((rc = batch_upload(B, &G.work, work[k]))) return rc;
        if ((rc = batch_upload(B, &G.slots, gslots[k]))) return rc;
        if (!gslots[k].empty() && (rc = batch_upload(B, &G.node_pre, pre[k]))) return rc;
        G.nwork = (int)work[k].size();
        G.nslots = (int)gslots[k].size();
        const long long nodes = pre[k].back();
        G.grid = (int)std::min<long long>(B->side_blocks, (nodes + 7) / 8);
    }
    if ((rc = batch_upload(B, &B->dall, all))) return rc;
    B->nall = (int)all.size();
    B->dirty = false;
    if (B->nall == 0) return LBM_OK;

    // capture ticks_per_launch ticks
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(B->s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    // one tick: fork; the boundary kernels of every group on the high-priority
    // branch, the bulk kernel of each group on a branch of its own (groups
    // beyond the branches share them); join; end-of-tick kernel
    // With few resident solves each solve's stream-collide pass is a launch of
    // the standalone kernel on a branch of its own (its parameters in the
    // constant bank, its source and destination arrays fixed per tick: the
    // solves advance in lockstep, an even number of ticks per replay, so each
    // keeps the parity it had at capture); with many solves, or an odd tick
    // count, one batched kernel per group.  A solve that finishes inside a replay keeps being streamed (not
    // read: its series rows stop at t_end) until the tables are rebuilt.
    int ngrp = 0;
    for (int k = 0; k < NG; ++k) ngrp += B->g[k].nslots ? 1 : 0;
    std::vector<int> live; // resident unfinished slots, largest first
    for (int sl = 0; sl < (int)B->slots.size(); ++sl)
        if (B->slots[sl].D && B->slots[sl].D->t < B->slots[sl].t_end) live.push_back(sl);
    std::sort(live.begin(), live.end(), [&](int a, int b) { return B->slots[a].D->p.N > B->slots[b].D->p.N; });
    // (an even tick count per replay keeps each solve's parity pattern from one
    // replay to the next)
    const bool per_solve = B->per_solve && B->tpl % 2 == 0 && (int)live.size() <= lbm_batch::PER_SOLVE_MAX;
    const int nbr = std::min(per_solve ? (int)live.size() : ngrp, lbm_batch::NBRANCH + 1); // branch 0 is B->s
    for (int t = 0; t < B->tpl && e == cudaSuccess; ++t) {
        if ((e = cudaEventRecord(B->ev_fork, B->s)) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(B->s2, B->ev_fork, 0)) != cudaSuccess) break;
        for (int b = 1; b < nbr && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(B->sb[b - 1], B->ev_fork, 0);
        int gi = 0;
        for (int k = 0; k < NG && e == cudaSuccess; ++k) {
            const auto &G = B->g[k];
            if (G.nslots == 0) continue;
            if (G.grid > 0)
                e = launch_bbnd(G.Q, G.prec, B->dsolves, G.slots, G.node_pre, G.nslots, G.grid, B->s2);
            if (per_solve) continue;
            const int b = gi++ % nbr;
            cudaStream_t bs = b == 0 ? B->s : B->sb[b - 1];
            if (e == cudaSuccess) e = launch_bbulk(G.Q, G.kind, G.fm, B->dsolves, G.work, G.nwork, bs);
        }
        if (per_solve) {
            for (int q = 0; q < (int)live.size() && e == cudaSuccess; ++q) {
                lbm_domain *D = B->slots[live[q]].D;
                const int par = (int)((D->t + t) & 1);
                StepBufs sbuf{};
                sbuf.src = D->pop[par];
                sbuf.dst = D->pop[par ^ 1];
                sbuf.mac_t = D->mac[par];
                sbuf.mac_t1 = D->mac[par ^ 1];
                sbuf.flags = D->flags;
                const int b = q % nbr;
                e = launch_bulk(D->Q, D->prec, D->p, sbuf, b == 0 ? B->s : B->sb[b - 1]);
            }
        }
        for (int b = 1; b < nbr && e == cudaSuccess; ++b) {
            if ((e = cudaEventRecord(B->ev_branch[b - 1], B->sb[b - 1])) != cudaSuccess) break;
            e = cudaStreamWaitEvent(B->s, B->ev_branch[b - 1], 0);
        }
        if (e != cudaSuccess) break;
        if ((e = cudaEventRecord(B->ev_join, B->s2)) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(B->s, B->ev_join, 0)) != cudaSuccess) break;
        e = launch_bfinish(B->dsolves, B->dall, B->nall, B->s);
    }
    cudaError_t e2 = cudaStreamEndCapture(B->s, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiateWithFlags(&B->exec, graph, cudaGraphInstantiateFlagUseNodePriority);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        B->exec = nullptr;
        B->dirty = true;
        return fail(LBM_ERR_CUDA, std::string("batch tick graph: ") + cudaGetErrorString(e));
    }
    return LBM_OK;
}

} // namespace

extern "C" {

int lbm_batch_create(const lbm_batch_desc *desc, lbm_batch **out) {
    if (!desc || !out) return fail(LBM_ERR_ARG, "null argument");
    *out = nullptr;
    const lbm_batch_desc &d = *desc;
    if (d.max_slots < 1 || d.max_slots > 4096) return fail(LBM_ERR_ARG, "max_slots must be in [1, 4096]");
    if (d.ticks_per_launch < 0 || d.ticks_per_launch > 4096) return fail(LBM_ERR_ARG, "ticks_per_launch in [0, 4096]");
    if (d.budget_bytes <= 0) return fail(LBM_ERR_ARG, "budget_bytes must be > 0");
    if (d.reserved != 0) return fail(LBM_ERR_ARG, "reserved must be 0");
    if ((d.alloc == nullptr) != (d.free == nullptr)) return fail(LBM_ERR_ARG, "alloc and free go together");
    DEVICE_SCOPE(d.device);
    cudaError_t e = cudaSuccess;
    lbm_batch *B = new lbm_batch();
    B->d = d;
    B->tpl = d.ticks_per_launch > 0 ? d.ticks_per_launch : 32;
    B->slots.resize(d.max_slots);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d.device);
    B->side_blocks = std::max(1, sms) * 3;
    if (const char *eg = std::getenv("LBM_BATCH_GROUPED")) B->per_solve = eg[0] != '1';
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (d.stream) {
        B->s = (cudaStream_t)d.stream;
    } else {
        B->own_s = true;
        e = cudaStreamCreateWithFlags(&B->s, cudaStreamNonBlocking);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&B->s2, cudaStreamNonBlocking, prio_hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming);
    for (int k = 0; k < lbm_batch::NBRANCH && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&B->sb[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_branch[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        lbm_batch_destroy(B);
        return fail(LBM_ERR_CUDA, std::string("batch streams: ") + cudaGetErrorString(e));
    }
    B->dsolves = (SolveDev *)B->alloc(sizeof(SolveDev) * d.max_slots);
    if (!B->dsolves) {
        lbm_batch_destroy(B);
        return fail(LBM_ERR_OOM, "batch solve table");
    }
    if ((e = cudaMemsetAsync(B->dsolves, 0, sizeof(SolveDev) * d.max_slots, B->s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(B->s)) != cudaSuccess) {
        lbm_batch_destroy(B);
        return fail(LBM_ERR_CUDA, std::string("batch create: ") + cudaGetErrorString(e));
    }
    *out = B;
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch *B) {
    if (!B) return LBM_OK;
    DEVICE_SCOPE(B->d.device);
    if (B->s) cudaStreamSynchronize(B->s);
    for (auto &S : B->slots)
        if (S.D) lbm_destroy_domain(S.D);
    batch_free_tables(B);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    B->release(B->dsolves);
    if (B->ev_fork) cudaEventDestroy(B->ev_fork);
    if (B->ev_join) cudaEventDestroy(B->ev_join);
    for (int k = 0; k < lbm_batch::NBRANCH; ++k) {
        if (B->ev_branch[k]) cudaEventDestroy(B->ev_branch[k]);
        if (B->sb[k]) cudaStreamDestroy(B->sb[k]);
    }
    if (B->s2) cudaStreamDestroy(B->s2);
    if (B->own_s && B->s) cudaStreamDestroy(B->s);
    delete B;
    return LBM_OK;
}

int lbm_batch_solve_bytes(const lbm_domain_desc *desc, const lbm_body *hb, int n, int64_t steps, int64_t *bytes) {
    if (!desc || !bytes) return fail(LBM_ERR_ARG, "null argument");
    int rc = batch_check_desc(*desc, hb, n, steps);
    if (rc) return rc;
    lbm_domain_desc d = *desc;
    if (d.series_capacity <= 0) d.series_capacity = steps;
    return domain_bytes(d, hb, n, bytes);
}

int lbm_batch_admit(lbm_batch *B, const lbm_domain_desc *desc, const lbm_body *hb, int n, int64_t steps,
                    int *slot_out) {
    if (!B || !desc || !slot_out) return fail(LBM_ERR_ARG, "null argument");
    *slot_out = -1;
    int rc = batch_check_desc(*desc, hb, n, steps);
    if (rc) return rc;
    lbm_domain_desc d = *desc;
    d.device = B->d.device;
    d.stream = B->s;
    d.alloc = B->d.alloc;
    d.free = B->d.free;
    d.alloc_ctx = B->d.alloc_ctx;
    if (d.series_capacity <= 0) d.series_capacity = steps;
    int64_t need = 0;
    if ((rc = domain_bytes(d, hb, n, &need))) return rc;
    int sl = -1;
    for (int k = 0; k < (int)B->slots.size() && sl < 0; ++k)
        if (!B->slots[k].D) sl = k;
    if (sl < 0) return fail(LBM_ERR_OOM, "no free slot");
    if (B->used + need > B->d.budget_bytes)
        return fail(LBM_ERR_OOM, "solve needs " + std::to_string(need) + " bytes, " +
                                     std::to_string(B->d.budget_bytes - B->used) + " left in the budget");
    DEVICE_SCOPE(B->d.device);
    lbm_domain *D = nullptr;
    if ((rc = create_domain_impl(&d, &D, true))) return rc;
    if ((rc = lbm_set_bodies(D, hb, n))) {
        lbm_destroy_domain(D);
        return rc;
    }
    long long nodes = 0;
    if (n > 0) {
        // poses of t = 0 and the boundary-node list (all static)
        cudaError_t e = launch_fprep(D->p, D->dbodies, D->poses, 0, nullptr, D->flags, D->chg_cnt, D->chg_cell, D->chg_val,
                                     D->chg_cap, D->apm_cnt, D->bn_cnt + 2, nullptr, nullptr, nullptr, D->s);
        if (e == cudaSuccess && (rc = build_bnd_lists(D))) {
            lbm_destroy_domain(D);
            return rc;
        }
        unsigned long long cnt = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, D->bn_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, D->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(D->s);
        if (e != cudaSuccess) {
            lbm_destroy_domain(D);
            return fail(LBM_ERR_CUDA, std::string("admit: ") + cudaGetErrorString(e));
        }
        nodes = (long long)std::min<unsigned long long>(cnt, (unsigned long long)D->bn_static_cap);
        D->prep_dirty = false;
    }
    SolveDev sv{};
    sv.p = D->p;
    sv.Q = D->Q;
    sv.active = 1;
    sv.t = 0;
    sv.t_end = steps;
    sv.pop[0] = D->pop[0];
    sv.pop[1] = D->pop[1];
    sv.flags = D->flags;
    sv.owner = D->owner[0];
    sv.bodies = D->dbodies;
    sv.poses = D->poses;
    sv.bn_static = D->bn_static;
    sv.bn_cnt = D->bn_cnt;
    sv.bn_cap = D->bn_static_cap;
    sv.acc = D->acc;
    sv.series = D->series;
    sv.counters = D->counters;
    cudaError_t e = cudaMemcpyAsync(B->dsolves + sl, &sv, sizeof(sv), cudaMemcpyHostToDevice, B->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->s);
    if (e != cudaSuccess) {
        lbm_destroy_domain(D);
        return fail(LBM_ERR_CUDA, std::string("admit: ") + cudaGetErrorString(e));
    }
    auto &S = B->slots[sl];
    S.D = D;
    S.t_end = steps;
    S.nodes = nodes;
    S.reported = false;
    B->used += (int64_t)D->bytes;
    B->dirty = true;
    *slot_out = sl;
    return LBM_OK;
}

int lbm_batch_run(lbm_batch *B, int n) {
    if (!B || n < 0) return fail(LBM_ERR_ARG, "invalid arguments");
    DEVICE_SCOPE(B->d.device);
    if (B->dirty) {
        int rc = batch_rebuild(B);
        if (rc) return rc;
    }
    if (!B->exec || n == 0) return LBM_OK;
    for (int k = 0; k < n; ++k) CK(cudaGraphLaunch(B->exec, B->s));
    const int64_t ticks = (int64_t)n * B->tpl;
    bool finished = false;
    for (auto &S : B->slots) {
        if (!S.D || S.D->t >= S.t_end) continue;
        S.D->t = std::min<int64_t>(S.D->t + ticks, S.t_end); // the device stops each solve at t_end
        if (S.D->t >= S.t_end) finished = true;
    }
    if (finished) B->dirty = true; // drop finished solves from the tables
    return LBM_OK;
}

int lbm_batch_poll(lbm_batch *B, int *slots_out, int cap, int *count_out) {
    if (!B || !count_out || cap < 0 || (cap > 0 && !slots_out)) return fail(LBM_ERR_ARG, "invalid arguments");
    DEVICE_SCOPE(B->d.device);
    CK(cudaStreamSynchronize(B->s));
    int c = 0;
    for (int sl = 0; sl < (int)B->slots.size() && c < cap; ++sl) {
        auto &S = B->slots[sl];
        if (S.D && !S.reported && S.D->t >= S.t_end) {
            S.reported = true;
            slots_out[c++] = sl;
        }
    }
    *count_out = c;
    return LBM_OK;
}

int lbm_batch_get_force_torque(lbm_batch *B, int slot, int64_t first, int64_t count, int kind, double *out) {
    if (!B || slot < 0 || slot >= (int)B->slots.size() || !B->slots[slot].D)
        return fail(LBM_ERR_ARG, "no solve in this slot");
    return lbm_get_force_torque(B->slots[slot].D, first, count, kind, out);
}

int64_t lbm_batch_time(const lbm_batch *B, int slot) {
    if (!B || slot < 0 || slot >= (int)B->slots.size() || !B->slots[slot].D) return -1;
    return B->slots[slot].D->t;
}

int lbm_batch_release(lbm_batch *B, int slot) {
    if (!B || slot < 0 || slot >= (int)B->slots.size() || !B->slots[slot].D)
        return fail(LBM_ERR_ARG, "no solve in this slot");
    DEVICE_SCOPE(B->d.device);
    CK(cudaStreamSynchronize(B->s));
    auto &S = B->slots[slot];
    const bool running = S.D->t < S.t_end;
    B->used -= (int64_t)S.D->bytes;
    SolveDev zero{};
    CK(cudaMemcpyAsync(B->dsolves + slot, &zero, sizeof(zero), cudaMemcpyHostToDevice, B->s));
    CK(cudaStreamSynchronize(B->s));
    lbm_destroy_domain(S.D);
    S = lbm_batch::Slot{};
    if (running) B->dirty = true;
    return LBM_OK;
}

int lbm_batch_usage(const lbm_batch *B, int *resident, int64_t *bytes) {
    if (!B || !resident || !bytes) return fail(LBM_ERR_ARG, "invalid arguments");
    int r = 0;
    for (const auto &S : B->slots) r += S.D != nullptr;
    *resident = r;
    *bytes = B->used;
    return LBM_OK;
}

} // extern "C"

// ---- population export without device allocation -----------------------------
//
// lbm_get_populations stages its FP64 copy in a buffer allocated per call.
// Callers that must not allocate at that moment (a serving batch that holds
// its memory to an exact budget; a monitoring thread that must not trigger
// the device-wide synchronisation of releasing CUDA memory) use
// lbm_get_populations_noalloc, which runs the same export kernel into this
// fixed scratch array instead.  The array is part of this file's device
// module: it takes its 32 MiB on a device when that module is loaded there.
// lbm_create_domain resolves its address once per device (with the device
// current), which also loads the module under lazy module loading, and
// caches it; the export itself then never looks the symbol up, loads a
// module or allocates.  Nothing in it has to start at zero: each call writes
// all N*Q values it copies out.  Calls that overlap on the GPU share it and
// race.

static __device__ __align__(256) double g_export_scratch[LBM_NOALLOC_MAX_VALUES];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::atomic<double *> g_export_scratch_ptr[NOALLOC_MAX_DEVICES] = {};
std::mutex g_export_scratch_mu;
} // namespace

// called by lbm_create_domain with `dev` current; a failed lookup leaves the
// domain usable (only the no-allocation export then reports LBM_ERR_STATE)
void noalloc_scratch_setup(int dev) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES || g_export_scratch_ptr[dev].load()) return;
    std::lock_guard<std::mutex> lk(g_export_scratch_mu);
    if (g_export_scratch_ptr[dev].load()) return;
    double *ptr = nullptr;
    if (cudaGetSymbolAddress((void **)&ptr, g_export_scratch) == cudaSuccess && ptr)
        g_export_scratch_ptr[dev].store(ptr);
    else
        cudaGetLastError(); // not sticky: clear it, the domain does not depend on the scratch
}

extern "C" int lbm_get_populations_noalloc(lbm_domain *D, double *out) {
    if (!D || !out) return fail(LBM_ERR_ARG, "invalid arguments");
    const long long n = D->p.N * D->Q;
    if (n > (long long)LBM_NOALLOC_MAX_VALUES)
        return fail(LBM_ERR_ARG, "lbm_get_populations_noalloc: the domain holds " + std::to_string(n) +
                                     " population values; the fixed scratch holds at most " +
                                     std::to_string((long long)LBM_NOALLOC_MAX_VALUES) +
                                     " (use lbm_get_populations)");
    const int dev = D->d.device;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(LBM_ERR_ARG, "device index out of range");
    double *scratch = g_export_scratch_ptr[dev].load();
    if (!scratch) return fail(LBM_ERR_STATE, "the fixed export scratch could not be set up on this device");
    DEVICE_SCOPE(dev);
    CK(launch_export(D->Q, D->prec, D->p, D->pop[D->t & 1], scratch, D->s));
    CK(cudaMemcpyAsync(out, scratch, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, D->s));
    CK(cudaStreamSynchronize(D->s));
    return LBM_OK;
}
