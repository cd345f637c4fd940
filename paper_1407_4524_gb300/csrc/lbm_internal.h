// lbm_internal.h -- host-side launcher interface between the C ABI
// (lbm_api.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include "lbm_dev.cuh"
#include "lbm_step.cuh"

namespace lbm {

struct GeomArgs {
    const BodyDev *bodies;
    const double *poses; // POSE_STRIDE doubles per body: X(t), Xw(t), X(t+1), Xw(t+1)
    const int2 *chunk_map; // (body, chunk within the body's region)
    int nchunks;
    const uint16_t *owner_t;
    uint16_t *owner_t1;
    uint8_t *flags;
    int *chunk_cnt_apm;
    int *chunk_cnt_link;
    uint32_t *apm_cell;
    int8_t *apm_sign;
    long long *apm_cnt;
    uint32_t *Lcell;
    uint8_t *Ldir;
    double *Ldelta;
    long long *link_cnt;
    long long t;      // current step
    long long t_link; // pose time of the links being built
    int do_apm;       // covered/uncovered lists (moving step)
    int do_flags;     // rewrite flags in the regions
    // reduced-precision modes: flag changes for t+1, applied by the next prep
    unsigned long long *chg_cnt;
    uint32_t *chg_cell;
    uint8_t *chg_val;
    long long chg_cap;
    // reduced-precision modes: boundary-node lists (static bodies; moving
    // bodies of the step being built)
    uint32_t *bn_static;
    unsigned long long *bn_static_cnt;
    uint32_t *bn_mov;
    unsigned long long *bn_mov_cnt;
    long long bn_static_cap, bn_mov_cap;
    int grid_cap; // > 0: at most this many blocks (side-stream kernels)
};

// arguments of the boundary-node kernel (reduced-precision modes)
struct BndArgs {
    const uint32_t *static_cells;
    const unsigned long long *static_cnt;
    const uint32_t *mov_cells; // nodes of step t next to moving bodies
    const unsigned long long *mov_cnt;
    long long static_cap, mov_cap;
    const uint16_t *owner_t, *owner_t1;
    const BodyDev *bodies;
    const double *poses;
};

// One resident solve of a serving batch (reduced-precision modes, static
// bodies): everything the batched kernels need to step it.
struct SolveDev {
    Params p;
    int Q;
    int active;         // 0 once t reaches t_end
    long long t, t_end; // current step, step at which the solve is complete
    void *pop[2];
    uint8_t *flags;
    const uint16_t *owner; // solid owner (static bodies: constant)
    const BodyDev *bodies;
    const double *poses;
    const uint32_t *bn_static;
    const unsigned long long *bn_cnt;
    long long bn_cap;
    unsigned long long *acc;
    double *series;
    unsigned long long *counters;
};

// precision: 0 FP64, 1 FP32, 2 FP16; Q: 9 or 19
cudaError_t launch_init(int Q, int prec, const Params &p, void *dst, void *mac, const uint8_t *flags,
                        const double u0[3], cudaStream_t s);
cudaError_t launch_links(int Q, int prec, const Params &p, const StepBufs &sb, int grid, cudaStream_t s);
cudaError_t launch_bulk(int Q, int prec, const Params &p, const StepBufs &sb, cudaStream_t s);
cudaError_t launch_finish(int Q, int prec, const Params &p, const StepBufs &sb, cudaStream_t s);

// per step: wrapped poses at t and t+1 and the prefix of the link counts
cudaError_t launch_prep(const Params &p, const BodyDev *bodies, const long long *link_cnt, long long *link_pre,
                        long long *tile_pre, double *poses, long long t, const unsigned long long *tdev,
                        uint8_t *flags, const long long *apm_cnt, const uint32_t *apm_cell, const int8_t *apm_sign,
                        cudaStream_t s);
// reduced-precision modes: poses, and the flag changes of the previous step;
// clears the change list and the covered/uncovered counters
// link mode (link_cnt_t given): the tile prefix of the links of t, and the
// moving bodies' link counts of t+1 cleared
cudaError_t launch_fprep(const Params &p, const BodyDev *bodies, double *poses, long long t,
                         const unsigned long long *tdev, uint8_t *flags, unsigned long long *chg_cnt,
                         const uint32_t *chg_cell, const uint8_t *chg_val, long long chg_cap, long long *apm_cnt,
                         unsigned long long *bn_mov_next_cnt, const long long *link_cnt_t, long long *link_cnt_t1,
                         long long *tile_pre, cudaStream_t s);
// link mode: FL_MAC on the nodes within R + MAC_BAND of every body at t
cudaError_t launch_macband(const Params &p, const GeomArgs &g, cudaStream_t s);

// geometry (all FP64, mode independent)
cudaError_t launch_raster(int Q, const Params &p, const GeomArgs &g, uint16_t *owner, long long t_pose,
                          cudaStream_t s);
cudaError_t launch_geom_a(int Q, const Params &p, const GeomArgs &g, cudaStream_t s);
cudaError_t launch_geom_b(int Q, const Params &p, const GeomArgs &g, cudaStream_t s);
cudaError_t launch_geom_c(int Q, const Params &p, const GeomArgs &g, cudaStream_t s);
cudaError_t launch_flags_full(int Q, const Params &p, const uint16_t *owner, uint8_t *flags, cudaStream_t s);
// reduced-precision modes: owner(t+1) + unordered A+/A- lists; flag changes
cudaError_t launch_fgeom1(int Q, const Params &p, const GeomArgs &g, cudaStream_t s);
cudaError_t launch_fgeom2(int Q, const Params &p, const GeomArgs &g, cudaStream_t s);
// reduced-precision modes: boundary nodes of every body (pull, wall values,
// momentum exchange, collision) -- runs beside k_bulk
cudaError_t launch_bnd(int Q, int prec, const Params &p, const BndArgs &a, const StepBufs &sb, int grid,
                       cudaStream_t s);
// batched serving kernels: one tick = bulk (per group), boundary nodes (per
// group), finish (every solve).  A group is a lattice, a storage type
// (BK_FP32 / BK_FP16) and a face mode; a bulk work item (slot, row, x0, 0)
// covers BBULK_THREADS nodes of one row of one solve.
constexpr int BK_FP32 = 0, BK_FP16 = 1;
constexpr int BBULK_THREADS = 64;
// fm: face mode of the group's solves (FM_PERIODIC / FM_XFACES / FM_GENERAL)
cudaError_t launch_bbulk(int Q, int kind, int fm, const SolveDev *solves, const int4 *work, int nwork,
                         cudaStream_t s);
cudaError_t launch_bbnd(int Q, int prec, const SolveDev *solves, const int *slots, const long long *node_pre,
                        int nslots, int grid, cudaStream_t s);
cudaError_t launch_bfinish(SolveDev *solves, const int *slots, int nslots, cudaStream_t s);
// boundary-node lists of step t from scratch (all bodies)
cudaError_t launch_bnd_lists(int Q, const Params &p, const GeomArgs &g, cudaStream_t s);

// free bodies: Newton-Euler update after the force/torque row of step t
cudaError_t launch_free(const Params &p, BodyDev *bodies, const double *series, unsigned long long *counters,
                        const unsigned long long *tdev, cudaStream_t s);

// semi-implicit free-body schemes: poses of t+1 of the free bodies from the
// records k_free left
cudaError_t launch_pose1(const Params &p, const BodyDev *bodies, double *poses, const unsigned long long *tdev,
                         cudaStream_t s);

// population export: fhat as FP64 f (adds w back for the shifted modes)
cudaError_t launch_export(int Q, int prec, const Params &p, const void *pop, double *out, cudaStream_t s);
cudaError_t launch_import(int Q, int prec, const Params &p, const double *in, void *pop, cudaStream_t s);

} // namespace lbm
