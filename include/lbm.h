/*
 * lbm.h -- C ABI of the GB300 lattice-Boltzmann library (liblbm.so).
 *
 * One library call advances a lattice-Boltzmann domain by BGK collision and
 * streaming (Giovacchini & Ortiz, arXiv:1407.4524, Sec. 2, Eqs. LBE,
 * collision, streaming) on the D2Q9 or D3Q19 lattice, applies the curved-wall
 * rule on every cut solid link (Sec. 2.1, Eqs. Fillipova_interpolation and
 * Fillipova_equilibrium) and accumulates, per body and per step, the
 * momentum-exchange force and torque in the paper's static, moving
 * (impulsive-correction) and moving-frame forms (Sec. 3, Eqs. flow_force_2,
 * flow_torque_2, ForceInMovement, TorqueInMovement,
 * ForceInMovementMovingFrame, TorqueInMovementMovingFrame).
 *
 * Conventions shared by every entry point
 *  - Every function returns an int status (LBM_OK = 0 on success).  On
 *    failure lbm_last_error() returns a message for the calling thread.  The
 *    library never aborts the process and never traps on the device.
 *  - Pointers named host_* / out are HOST memory owned by the caller.  The
 *    library owns every device buffer of a domain; it allocates them through
 *    the optional allocator callbacks of the descriptor (so a caller can plug
 *    in its own caching allocator) or with cudaMalloc.
 *  - Work is enqueued asynchronously on the domain's CUDA stream; functions
 *    that return data to the host synchronise that stream first.
 *  - An entry point that works on a domain or batch makes that object's
 *    device current while it runs and restores the calling thread's current
 *    device before it returns (on success and on failure).
 *  - Lattice units: delta_x = delta_t = 1; velocities in cells per step.
 *    Node (x, y, z) sits at integer coordinates; cell index
 *    (z * ny + y) * nx + x; populations are laid out [Q][nz][ny][nx].
 *  - Direction order (shared with every array the library returns):
 *      D2Q9 : 0 rest, 1 (1,0), 2 (0,1), 3 (-1,0), 4 (0,-1),
 *             5 (1,1), 6 (-1,1), 7 (-1,-1), 8 (1,-1)
 *      D3Q19: 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z,
 *             7 (1,1,0), 8 (-1,-1,0), 9 (1,-1,0), 10 (-1,1,0),
 *             11 (1,0,1), 12 (-1,0,-1), 13 (1,0,-1), 14 (-1,0,1),
 *             15 (0,1,1), 16 (0,-1,-1), 17 (0,1,-1), 18 (0,-1,1)
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define LBM_OK 0
#define LBM_ERR_ARG 1      /* invalid argument or descriptor */
#define LBM_ERR_OOM 2      /* device or host allocation failed */
#define LBM_ERR_CUDA 3     /* a CUDA runtime call failed (message has the reason) */
#define LBM_ERR_UNSTABLE 4 /* a NaN or |u| > 0.3 was detected in a checked step
                             (returned by the series / force reads of that solve) */
#define LBM_ERR_TIMEOUT 5  /* a bounded device wait gave up (the mbarrier waits of
                             the staged stream-collide kernel, LBM_STAGED=1) */
#define LBM_ERR_STATE 6    /* call not allowed in the current state */

/* ---- enumerations -------------------------------------------------------------- */
#define LBM_D2Q9 9
#define LBM_D3Q19 19

/* Precision modes.  FP64: FP64 arithmetic and FP64 storage of f.
 * FP32 / FP16: FP32 arithmetic, populations stored as deviations f_i - w_i
 * in FP32 / FP16.  The per-body momentum-exchange sums are FP64 (sequential,
 * in link order) in the FP64 mode and exact 64-bit fixed point (units of
 * 2^-36, order independent) in the FP32 / FP16 modes, read out as FP64. */
#define LBM_FP64 0
#define LBM_FP32 1
#define LBM_FP16 2

/* Equilibrium: quasi-incompressible model (Sec. 2, rho replaced by rho0 in
 * the momentum) or the standard truncated Maxwellian. */
#define LBM_EQ_INCOMP 0
#define LBM_EQ_STANDARD 1

/* Edge kinds for the six faces.  Under LBM_EDGE_RULE_LINK (default) walls
 * and the inlet are links at Delta = 1/2 handled by the same curved-wall rule
 * (u_B = 0 for walls, u_B = inlet profile at the wall point for the inlet;
 * walls half-way, at -1/2 and n - 1/2); the outlet copies the last interior
 * column (zero gradient).  Inlet only on x-low, outlet only on x-high; a wall
 * takes precedence at corners. */
#define LBM_EDGE_PERIODIC 0
#define LBM_EDGE_WALL 1
#define LBM_EDGE_INLET 2
#define LBM_EDGE_OUTLET 3

/* Edge rule (the test section of the paper imposes its no-slip walls with
 * the Zou-He velocity condition of its cited reference).
 * LBM_EDGE_RULE_ZOUHE: the nodes of wall and inlet faces lie ON the boundary
 * (walls at the node layers 0 and n - 1) with velocity 0 (walls) or the
 * inlet profile (u_in, or 4 u_in y (H - y) / H^2 with H = ny - 1); after
 * streaming, the populations entering from outside are closed at each face
 * node so that its momentum sum_i c_i f_i equals rho u_w - g/2 (rho0 u_w - g/2
 * in the quasi-incompressible model; g the body force): bounce-back of the
 * non-equilibrium part plus the tangential correction.  Edge and corner nodes
 * (two or three such faces) take u = 0 without the force shift, bounce-back,
 * a tangential correction along a 3-D edge, and share the density of their
 * inner diagonal neighbour at t among the remaining unknown pairs.  Needs at
 * least 3 nodes along each such axis; not available in serving batches. */
#define LBM_EDGE_RULE_LINK 0
#define LBM_EDGE_RULE_ZOUHE 1

#define LBM_INLET_UNIFORM 0
#define LBM_INLET_PARABOLIC 1 /* u_x(y) = 4 u_in (y+1/2)(ny-1/2-y)/ny^2 */

/* Refill of nodes uncovered by a moving body (Sec. 3, after Eq.
 * ForceInMovement, which lists three rules): equilibrium at the mean density
 * of the fluid neighbours with the body velocity at the node (default) or the
 * neighbour-mean velocity; or the quadratic extrapolation
 * f_i(A) = 3 fhat_i(A+c*) - 3 fhat_i(A+2c*) + fhat_i(A+3c*) of the
 * post-collision values at t along the lattice direction c* closest to the
 * body's outward normal at A (largest n.c/|c|), falling back to the default
 * rule where one of the three nodes is solid at t or outside a non-periodic
 * face. */
#define LBM_REFILL_RHOBAR_UB 0
#define LBM_REFILL_RHOBAR_UBAR 1
#define LBM_REFILL_EXTRAP 2

#define LBM_SHAPE_CYLINDER 0 /* disc in the x-y plane (infinite along z in 3-D) */
#define LBM_SHAPE_SPHERE 1
#define LBM_SHAPE_ELLIPSE 2  /* ellipse in the x-y plane, semi-axes R and R2,
                                orientation theta (infinite along z in 3-D) */

/* Which force/torque form lbm_get_force_torque returns. */
#define LBM_FT_STATIC 0    /* Eqs. flow_force_2 / flow_torque_2 */
#define LBM_FT_LATTICE 1   /* Eqs. ForceInMovement / TorqueInMovement */
#define LBM_FT_MOVING 2    /* Eqs. ForceInMovementMovingFrame / ... (last two terms dropped) */
#define LBM_FT_IMPULSIVE 3 /* the A+/A- impulsive terms alone */

/* Number of doubles per body per step in the raw series:
 * Fs[3] Ts[3] (static form), Fi[3] Ti[3] (impulsive terms),
 * Fm[3] Tm[3] (moving frame).  Torques are about the body centre at step t,
 * r = x_A - X(t) taken at the fluid node x_A (Eq. H). */
#define LBM_SERIES_ROW 18

typedef void *(*lbm_alloc_fn)(size_t bytes, void *ctx);
typedef void (*lbm_free_fn)(void *ptr, void *ctx);

typedef struct lbm_domain_desc {
    int lattice;       /* LBM_D2Q9 or LBM_D3Q19 */
    int nx, ny, nz;    /* nz = 1 for D2Q9; each >= 1 */
    int precision;     /* LBM_FP64 / LBM_FP32 / LBM_FP16 */
    int equilibrium;   /* LBM_EQ_* */
    int edge[6];       /* x-lo, x-hi, y-lo, y-hi, z-lo, z-hi: LBM_EDGE_* */
    int inlet_profile; /* LBM_INLET_* */
    int refill;        /* LBM_REFILL_* */
    int has_force;     /* 1: Guo body force `force` (channel checks) */
    int device;        /* CUDA device ordinal */
    double tau;        /* BGK relaxation time, > 1/2 */
    double rho0;       /* reference density (quasi-incompressible model) */
    double u_in;       /* inlet velocity (maximum of the parabolic profile) */
    double force[3];   /* body-force density */
    double u0[3];      /* initial uniform velocity: f(x,0) = f^eq(1, u0) */
    int64_t series_capacity; /* steps kept in the device force ring; 0 -> 8192 */
    void *stream;            /* cudaStream_t to enqueue on; NULL -> default stream */
    lbm_alloc_fn alloc;      /* optional device allocator (NULL -> cudaMalloc) */
    lbm_free_fn free;        /* matching free */
    void *alloc_ctx;         /* passed through to alloc / free */
    double gravity[3];       /* acceleration of the free bodies: each feels its
                                weight less buoyancy, (rho_b - rho0) V gravity */
    int edge_rule;           /* LBM_EDGE_RULE_* */
    int free_scheme;         /* LBM_FREE_*: covered / uncovered sets of free bodies */
} lbm_domain_desc;

typedef struct lbm_body {
    int shape;       /* LBM_SHAPE_* */
    int halfway;     /* 1: every cut link of the body takes Delta = 1/2 */
    int free_body;   /* 0: prescribed motion; 1: free -- moved by the flow (below) */
    int reserved;    /* must be 0 */
    double R;        /* radius */
    double X0[3];    /* centre at step t0 */
    double U[3];     /* translation velocity: X(t) = X0 + (t - t0) U (free: initial) */
    double W[3];     /* angular velocity (2-D: W[2]) (free: initial) */
    int64_t t0;      /* step at which the body is at X0 */
    double density_ratio; /* free bodies: body density / rho0 (> 0) */
    double R2;       /* LBM_SHAPE_ELLIPSE: second semi-axis, 0 < R2 <= R */
    double theta0;   /* LBM_SHAPE_ELLIPSE: angle of the R axis to x at step t0;
                        theta(t) = theta0 + (t - t0) W[2] */
} lbm_body;
/* Free bodies follow Newton's and Euler's equations by forward Euler, as the
 * paper's sedimentation tests do:
 *   U(t+1) = U(t) + (F(t) + (rho_b - rho0) V gravity) / M,  M = rho_b V
 *   W(t+1) = W(t) + T(t) / I
 * with F, T the lattice-frame force and torque of step t (Eqs. ForceInMovement,
 * TorqueInMovement: static plus impulsive terms), V = pi R^2 nz (cylinder),
 * pi R R2 nz (ellipse) or 4/3 pi R^3 (sphere), I = M R^2 / 2 (cylinder, about
 * z), M (R^2 + R2^2) / 4 (ellipse) or 2/5 M R^2 (sphere).  The impulsive terms
 * need the nodes a body covers and uncovers, which for a free body depend on
 * its motion; the descriptor's free_scheme picks how (Sec. 3, after Eq.
 * ForceInMovement):
 *   LBM_FREE_EXPLICIT (0): in step t the body moves with U(t), W(t), so the
 *     sets of the step are known before its force;
 *   LBM_FREE_AIDUN (1): the force at t takes the impulsive terms of the nodes
 *     covered and uncovered between t-1 and t (the Aidun-type approximation;
 *     the series row of step t reports those), and the body moves from t to
 *     t+1 with U(t+1), W(t+1);
 *   LBM_FREE_PREDICTOR (2): the force at t takes the sets of a displacement
 *     predicted with U(t), W(t); then the displacement is recomputed with
 *     U(t+1), W(t+1) (two displacements per step); a node uncovered by both
 *     keeps the refill the force used, one uncovered only by the second is
 *     refilled then.
 * These schemes act on free bodies; prescribed bodies always take the exact
 * sets of their motion.  A free body that comes within 2 cells of a
 * non-periodic face or whose surface speed exceeds 0.25 makes the series
 * reads return LBM_ERR_STATE. */
#define LBM_FREE_EXPLICIT 0
#define LBM_FREE_AIDUN 1
#define LBM_FREE_PREDICTOR 2

typedef struct lbm_stats {
    int64_t step;            /* current time step t */
    int64_t cells;           /* nx*ny*nz */
    int64_t fluid_cells;     /* cells outside every body at t */
    int64_t links;           /* cut body links at t */
    int64_t fallback_links;  /* Delta < 1/2 links whose u_G node was missing
                                (plain bounce-back used), summed over steps */
    int64_t covered;         /* A+ nodes, summed over steps */
    int64_t uncovered;       /* A- nodes, summed over steps */
    int64_t device_bytes;    /* device memory held by the domain */
    int64_t h2d_bytes;       /* bytes copied host -> device by API calls */
    int64_t d2h_bytes;       /* bytes copied device -> host by API calls */
    int64_t timeouts;        /* non-zero: a kernel gave up a bounded wait (the
                                step's results are invalid; LBM_ERR_TIMEOUT) */
    int64_t unstable;        /* non-zero: a NaN or |u| > 0.3 was seen at a boundary
                                node, or a force was not finite (LBM_ERR_UNSTABLE);
                                domains without bodies are not checked */
    int64_t extrapolated;    /* A- nodes refilled by extrapolation (LBM_REFILL_EXTRAP),
                                summed over steps */
} lbm_stats;

typedef struct lbm_domain lbm_domain;

/* Message describing the last failure on this thread ("" if none). */
const char *lbm_last_error(void);

/* Library version string. */
const char *lbm_version(void);

/* Lattice tables in the direction order above: c[Q][3], w[Q], opp[Q]
 * (host arrays, caller-owned).  Needs no GPU. */
int lbm_lattice_table(int lattice, int *c, double *w, int *opp);

/* Create a domain: validates the descriptor, allocates its device buffers,
 * and sets f(x, 0) = f^eq(1, u0) everywhere (collided state of step 0).
 * LBM_ERR_ARG for an invalid descriptor, LBM_ERR_OOM / LBM_ERR_CUDA on
 * allocation or device failure (nothing is leaked). */
int lbm_create_domain(const lbm_domain_desc *desc, lbm_domain **out);

/* Free every device buffer of the domain (synchronises its stream). */
int lbm_destroy_domain(lbm_domain *dom);

/* Place n bodies (host array, copied).  Allowed only at t = 0; rebuilds the
 * solid flags and cut-link lists and re-initialises f(x,0).  Bodies must not
 * overlap, must keep a surface gap >= 2 cells from each other and >= 3 cells
 * from non-periodic faces, and must be smaller than half the domain on
 * periodic axes (LBM_ERR_ARG otherwise).  Bodies with U or W != 0 move by the
 * prescribed motion and have their links and A+/A- sets rebuilt every step.
 * LBM_ERR_ARG / LBM_ERR_STATE leave the domain unchanged; LBM_ERR_OOM (or
 * LBM_ERR_CUDA) part-way through puts it back into its created state: no
 * bodies, every node fluid, f(x,0) re-initialised, its buffers released. */
int lbm_set_bodies(lbm_domain *dom, const lbm_body *host_bodies, int n);

/* Replace the motion of existing bodies between steps (free-body coupling):
 * new X0, U, W, t0 for each body; shape and R must stay the same.  The pose
 * at the current step must equal the pose the domain already holds within
 * 1e-9 cells (the solid set at t does not jump); LBM_ERR_ARG otherwise.  The
 * records go to the device through pinned staging in stream order after the
 * steps already enqueued: the call does not wait for them (unless a body
 * starts or stops moving, which rebuilds the body maps and synchronises). */
int lbm_update_bodies(lbm_domain *dom, const lbm_body *host_bodies, int n);

/* Advance n steps, asynchronously on the domain's stream.  Step t -> t+1
 * appends one row per body to the force/torque series (the force at time t
 * of Sec. 3). */
int lbm_step(lbm_domain *dom, int n);

/* Record the domain's step graph now without taking a step.  lbm_step
 * replays a captured CUDA graph of 16 steps for every run of >= 16 steps that
 * starts at an even step, and records that graph at the first such run; a
 * caller that wants no recording cost inside a later timed or
 * latency-critical run calls this once beforehand (the graph is recorded for
 * even starts whatever the parity of the current step).  It needs one step
 * taken since the bodies were placed or changed (LBM_ERR_STATE before);
 * LBM_OK without recording when the domain runs plain launches. */
int lbm_prepare_graph(lbm_domain *dom);

/* Copy series rows [first, first+count) of every body into host memory:
 * out[count][n_bodies][6] = (Fx, Fy, Fz, Tx, Ty, Tz) in form `kind`
 * (LBM_FT_*).  Waits only for the steps that wrote those rows (the end of
 * the lbm_step call that reached step first+count), so steps enqueued after
 * them keep running: reading the row of step t after enqueuing step t+1
 * overlaps the copy with the GPU's work.  Rows older than the ring capacity
 * are gone (LBM_ERR_ARG).  LBM_ERR_UNSTABLE / LBM_ERR_TIMEOUT / LBM_ERR_STATE
 * report a flag the device set in any step so far. */
int lbm_get_force_torque(lbm_domain *dom, int64_t first, int64_t count, int kind, double *out);

/* Raw series rows: out[count][n_bodies][LBM_SERIES_ROW]. */
int lbm_get_series(lbm_domain *dom, int64_t first, int64_t count, double *out);

/* Post-collision populations fhat(x, t) of the current step as FP64 f (not
 * f - w), out[Q][nz][ny][nx]; values at solid nodes are unspecified.
 * Synchronises. */
int lbm_get_populations(lbm_domain *dom, double *out);

/* lbm_get_populations without any device allocation (the paper has no
 * counterpart; this is an interface for callers that may not allocate).
 * lbm_get_populations stages the FP64 copy in a fresh N*Q-double device
 * buffer.  A caller that holds its device memory to an exact budget (a
 * serving batch filled up to its limit) has no room for that buffer, and a
 * monitoring thread reading a domain while other streams run should not
 * allocate either, since releasing plain CUDA memory synchronises the whole
 * device.  This variant stages through one fixed scratch array that the
 * library holds in its own device memory: at most
 * LBM_NOALLOC_MAX_VALUES = 4,194,304 doubles (32 MiB), so it serves domains
 * with N*Q <= 4,194,304 and returns LBM_ERR_ARG, with a message naming the
 * limit, for larger ones (nothing is copied then).
 * - The scratch is a static reservation of 32 MiB per device, taken when
 *   the first domain (or serving batch) is created on that device and held
 *   until the process exits.  A serving batch's budget_bytes does not count
 *   it: it is the same fixed 32 MiB however many solves are admitted.
 *   lbm_create_domain looks its address up (with the device current), so
 *   the export itself neither looks anything up nor allocates; if that
 *   lookup failed, the call returns LBM_ERR_STATE and the domain is
 *   otherwise unaffected.
 * - Like every entry point, it restores the calling thread's current device
 *   before it returns.
 * - No part of the scratch has to start at zero: a call writes every value it
 *   copies out.
 * - The scratch is shared by every domain on the device: calls that overlap
 *   in time (other host threads, or work still in flight on another stream)
 *   race on it, so the caller serialises them.
 * Output, layout and synchronisation as lbm_get_populations. */
#define LBM_NOALLOC_MAX_VALUES 4194304
int lbm_get_populations_noalloc(lbm_domain *dom, double *out);

/* Sets the populations of the current step t: `f` is host FP64 f_i(x, t)
 * (pre-collision), layout [Q][nz][ny][nx], as lbm_get_populations returns
 * (SoA, x fastest).  The library computes the moments (Eqs.
 * LBMmacroscopics_0/1) and the BGK collision (Eq. collision) of every node
 * and stores fhat(x, t), from which the next lbm_step streams; in the reduced
 * modes f - w is rounded to the storage precision.  The values at solid
 * nodes are ignored by the step.  Bodies (lbm_set_bodies) re-initialise the
 * populations, so set the bodies first.  Synchronous; the caller keeps `f`.
 * Errors: LBM_ERR_ARG (NULL), LBM_ERR_OOM (staging buffer), LBM_ERR_CUDA. */
int lbm_set_populations(lbm_domain *dom, const double *f);

/* Moments of the current step t into host `out` [4][nz][ny][nx]: rho, u_x,
 * u_y, u_z, with rho_u u = sum_i c_i f_i + g/2 (rho_u = rho0 in the
 * quasi-incompressible model, else rho; g the body force), evaluated from the
 * stored post-collision populations (the collision keeps rho and adds g to the
 * momentum).  Zero at solid nodes.  Synchronous.
 * Errors: LBM_ERR_ARG (NULL), LBM_ERR_OOM (staging buffer), LBM_ERR_CUDA. */
int lbm_get_macros(lbm_domain *dom, double *out);

/* State snapshots (checkpoint / resume; no counterpart in the paper).
 * lbm_state_bytes: size of a snapshot of this domain (-1 for NULL).
 * lbm_save_state: copies the whole state at the current step -- every device
 * buffer (populations, moments, solid owners and flags, cut-link and
 * boundary-node lists, body records, the force/torque ring, counters), the
 * step index and the host's body records -- into `out` (caller-owned, at
 * least lbm_state_bytes).  Synchronises.
 * lbm_load_state: restores such a snapshot into a domain created with the
 * same descriptor and given the same number of bodies by lbm_set_bodies, so
 * that its buffers have the snapshot's sizes (LBM_ERR_ARG otherwise); the
 * steps that follow reproduce those of the saved domain bit for bit.
 * A snapshot is raw host-endian memory of this library version: it is not a
 * portable file format.  Every check runs before anything is changed, so
 * LBM_ERR_ARG leaves the domain as it was; after LBM_ERR_CUDA its state is
 * undefined (load the snapshot again or destroy the domain).  Synchronises. */
int64_t lbm_state_bytes(const lbm_domain *dom);
int lbm_save_state(lbm_domain *dom, void *out, int64_t cap);
int lbm_load_state(lbm_domain *dom, const void *in, int64_t size);

/* Body state at the current step: out[n_bodies][9] = X(t), U(t), W(t).
 * Synchronises.  (Free bodies: their integrated motion.) */
int lbm_get_body_state(lbm_domain *dom, double *out);

/* Owning body index of every node at the current step (-1: fluid),
 * out[nz][ny][nx].  Synchronises. */
int lbm_get_solid(lbm_domain *dom, int32_t *out);

/* Counters of the domain (synchronises). */
int lbm_get_stats(lbm_domain *dom, lbm_stats *out);

/* Current step t. */
int64_t lbm_time(const lbm_domain *dom);

/* Change the stream work is enqueued on (the old stream is synchronised). */
int lbm_set_stream(lbm_domain *dom, void *stream);

/* Kernel timing for roofline reports: while enabled, lbm_step records CUDA
 * events around every launch of the bulk stream-collide kernel on the
 * domain's stream.  lbm_kernel_time returns (and clears) the number of timed
 * launches and their total device time in milliseconds.  Synchronises. */
int lbm_set_kernel_timing(lbm_domain *dom, int enable);
int lbm_kernel_time(lbm_domain *dom, int64_t *launches, double *total_ms);

/* Number of kernel launches lbm_step(dom, 1) issues at the current state. */
int lbm_launches_per_step(const lbm_domain *dom, int *out);

/* ---- serving: continuous batching of many solves ------------------------------
 * A batch keeps up to max_slots independent solves resident on one GPU (each
 * with its own populations, admitted against a device-memory budget) and
 * advances all unfinished ones together: one tick is five kernel launches
 * (bulk and boundary-node kernels per lattice, one end-of-step kernel) for
 * the whole batch, replayed as a CUDA graph.  Supported: reduced-precision
 * modes (LBM_FP32 / LBM_FP16) and static bodies.  Each solve runs the same
 * arithmetic as a standalone domain of the same descriptor and its
 * force/torque sums are exact, so its results are bit-identical alone and in
 * any mix. */

typedef struct lbm_batch lbm_batch;

typedef struct lbm_batch_desc {
    int device;
    int max_slots;           /* resident solves at most (>= 1) */
    int ticks_per_launch;    /* steps per lbm_batch_run launch; 0 -> 32 */
    int reserved;
    int64_t budget_bytes;    /* device memory the resident solves may hold */
    void *stream;            /* cudaStream_t; NULL -> default stream */
    lbm_alloc_fn alloc;      /* optional allocator for the solves' buffers */
    lbm_free_fn free;
    void *alloc_ctx;
} lbm_batch_desc;

int lbm_batch_create(const lbm_batch_desc *desc, lbm_batch **out);
int lbm_batch_destroy(lbm_batch *batch);

/* Device bytes a solve with this descriptor and body list would hold. */
int lbm_batch_solve_bytes(const lbm_domain_desc *desc, const lbm_body *host_bodies, int n, int64_t steps,
                          int64_t *bytes);

/* Admit a solve of `steps` steps (desc->stream / alloc are ignored: the
 * batch's are used).  LBM_ERR_OOM if it does not fit the remaining budget or
 * no slot is free (nothing is allocated then); LBM_ERR_ARG for moving bodies
 * or FP64.  *slot_out receives the slot index. */
int lbm_batch_admit(lbm_batch *batch, const lbm_domain_desc *desc, const lbm_body *host_bodies, int n,
                    int64_t steps, int *slot_out);

/* Advance every resident unfinished solve by n * ticks_per_launch steps
 * (each stops at its own step count).  Asynchronous. */
int lbm_batch_run(lbm_batch *batch, int n);

/* Slots that completed since the previous poll (synchronises):
 * up to cap indices into slots_out, their number in *count_out. */
int lbm_batch_poll(lbm_batch *batch, int *slots_out, int cap, int *count_out);

/* Force/torque rows of a slot's solve, as lbm_get_force_torque. */
int lbm_batch_get_force_torque(lbm_batch *batch, int slot, int64_t first, int64_t count, int kind, double *out);

/* Current step of a slot's solve. */
int64_t lbm_batch_time(const lbm_batch *batch, int slot);

/* Free a slot (finished or not) and return its memory to the budget. */
int lbm_batch_release(lbm_batch *batch, int slot);

/* Resident solves and bytes held. */
int lbm_batch_usage(const lbm_batch *batch, int *resident, int64_t *bytes);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
