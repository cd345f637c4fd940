/*
 * lbm_oracle.c -- plain FP64 CPU oracle for the lattice-Boltzmann BGK step
 * with the curved-wall condition on cut links and the momentum-exchange (ME)
 * force and torque of Giovacchini & Ortiz, "Flow force and torque on
 * submerged bodies in lattice-Boltzmann via momentum exchange"
 * (arXiv:1407.4524).
 *
 * TEST INFRASTRUCTURE. This is the slow, obviously-correct reference that the
 * CUDA library is checked against. Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it; the product library never
 * links, includes or calls it, and the two share no code, header or table.
 *
 * One call of or_step() advances t -> t+1 in the order the paper gives
 * (Sec. 2, Sec. 3):
 *   1. moments rho, u of f(t) at fluid nodes          (Eqs. LBMmacroscopics_0/1,
 *                                                        quasi-incompressible rho0)
 *   2. BGK collision  fhat = f - (f - feq)/tau         (Eq. collision)
 *   3. streaming f_i(x, t+1) = fhat_i(x - c_i, t); where x - c_i is a solid
 *      node the value comes from the curved-wall rule (Eqs. Fillipova_
 *      interpolation / Fillipova_equilibrium, chi and u_bf of Sec. 2.1)
 *   4. ME force/torque per body over the cut links    (Eqs. flow_force_2,
 *      flow_torque_2, ForceInMovementMovingFrame, TorqueInMovementMovingFrame)
 *      using the identities of Eq. Equalities
 *   5. prescribed body motion, covered / uncovered node sets A+ and A-,
 *      impulsive terms (Eqs. ForceInMovement, TorqueInMovement) and the
 *      refill of uncovered nodes (Sec. 3, discussion after Eq. ForceInMovement)
 *   6. free bodies: forward-Euler Newton-Euler update of their velocity from
 *      the step's lattice-frame force and torque, weight and buoyancy
 *
 * Floating point: everything is FP64, loops run in cell order
 * ((z*ny + y)*nx + x) and direction order, and every formula is written as a
 * single fixed expression (compile with -ffp-contract=off).  Where the paper
 * leaves a choice open (sign of the moving-wall term, equilibrium of the
 * quasi-incompressible model, time levels, refill rules, edge treatment) the
 * comment at the function states the reading taken.
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * against closed forms, conservation laws, symmetry and exact special cases;
 * the absolute drag of a static cylinder and sphere by the Stokes drag of
 * periodic arrays (Hasimoto; Sangani & Acrivos).  Absolute drag/lift/torque
 * VALUES of the paper's own benchmark geometries are "parity unpinned": the
 * paper prints no numbers for them.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_OOM 2
#define OR_ERR_STATE 3

#define OR_PERIODIC 0
#define OR_WALL 1
#define OR_INLET 2
#define OR_OUTLET 3

#define OR_SHAPE_CYLINDER 0 /* disc in the x-y plane, infinite along z */
#define OR_SHAPE_SPHERE 1
#define OR_SHAPE_ELLIPSE 2 /* ellipse in the x-y plane (semi-axes R, R2), infinite along z */

#define OR_ROW 18 /* Fs Ts Fi Ti Fm Tm, 3 components each */

typedef struct {
    int q;               /* 9 (D2Q9) or 19 (D3Q19) */
    int nx, ny, nz;      /* nz = 1 for D2Q9 */
    int eq;              /* 0: quasi-incompressible (He-Luo), 1: standard */
    int edge[6];         /* x-lo, x-hi, y-lo, y-hi, z-lo, z-hi: OR_PERIODIC.. */
    int inlet_parabolic; /* 0: uniform u_in, 1: parabolic in y, maximum u_in */
    int has_force;       /* Guo body force (used only by the Poiseuille check) */
    int refill;          /* 0: feq(rho_bar, u_B); 1: feq(rho_bar, u_bar); 2: extrapolation */
    double tau;
    double rho0;
    double u_in;
    double g[3];
    double u0[3];
    double gravity[3]; /* acceleration of the free bodies (weight less buoyancy) */
    int edge_rule;     /* 0: wall / inlet faces are half-way links; 1: Zou-He nodes on the faces */
    int free_scheme;   /* free bodies: 0 explicit, 1 backward sets (Aidun), 2 predictor-corrector */
} or_desc;

typedef struct {
    int shape;    /* OR_SHAPE_* */
    int halfway;  /* 1: every link of this body takes Delta = 1/2 */
    int invert;   /* 1: the solid is OUTSIDE the surface (test geometry) */
    int free;     /* 1: moved by the flow force and torque (Newton-Euler), else prescribed */
    double R;
    double X0[3]; /* centre at step t0 */
    double U[3];  /* translation velocity (lattice units per step) */
    double W[3];  /* angular velocity */
    long long t0;
    double density_ratio; /* free bodies: body density / rho0 */
    double R2;            /* ellipse: the second semi-axis (along the body's y axis) */
    double theta0;        /* ellipse: angle of the body's x axis at step t0 */
} or_body;

typedef struct {
    or_desc d;
    int D, Q;
    int n[3];
    long N;
    int c[19][3];
    double w[19];
    int opp[19];
    double *f, *fhat, *fnew, *rho, *u;
    int *solid, *solid_next; /* owning body index, or -1 for fluid */
    int nb;
    or_body *b;
    long long t;
    long long nrec, cap;
    double *series; /* [nrec][nb][OR_ROW] */
    double edge_me[6];
    long long n_fallback;
    long long n_extrap; /* uncovered nodes refilled by extrapolation */
    double *imp_prev;   /* free_scheme 1: impulsive terms of the previous displacement [nb][6] */
    double *pre;        /* free_scheme 2: refill of the predicted uncovered nodes [Q][N] */
    char *pre_set;      /* free_scheme 2: node uncovered by the prediction */
    long long n_mismatch; /* free_scheme 2: nodes whose change the prediction got wrong */
} or_dom;

/* ---- lattice tables (standard D2Q9 / D3Q19; direction order fixed here) -- */

static const int C9[9][3] = {{0, 0, 0},  {1, 0, 0},   {0, 1, 0},
                             {-1, 0, 0}, {0, -1, 0},  {1, 1, 0},
                             {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const int C19[19][3] = {
    {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
    {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
    {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

int or_lattice(int q, int *c_out, double *w_out, int *opp_out)
{
    const int (*C)[3];
    if (q == 9) C = C9;
    else if (q == 19) C = C19;
    else return OR_ERR_ARG;
    for (int i = 0; i < q; ++i) {
        int n2 = C[i][0] * C[i][0] + C[i][1] * C[i][1] + C[i][2] * C[i][2];
        double w;
        if (q == 9) w = n2 == 0 ? 4.0 / 9.0 : (n2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
        else w = n2 == 0 ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        for (int k = 0; k < 3; ++k) c_out[3 * i + k] = C[i][k];
        w_out[i] = w;
        opp_out[i] = -1;
        for (int j = 0; j < q; ++j)
            if (C[j][0] == -C[i][0] && C[j][1] == -C[i][1] && C[j][2] == -C[i][2])
                opp_out[i] = j;
    }
    return OR_OK;
}

/* ---- small helpers --------------------------------------------------------- */

static long cell(const or_dom *o, int x, int y, int z)
{
    return ((long)z * o->n[1] + y) * o->n[0] + x;
}

static int periodic(const or_dom *o, int axis) { return o->d.edge[2 * axis] == OR_PERIODIC; }

/* minimum-image displacement x - X along one axis (the torque lever arm of
 * Eq. H and the body geometry on periodic axes): the plain definition
 * v - L * round(v / L), with halves rounded up, for v = x - X */
static double axis_disp(const or_dom *o, int axis, double x, double X)
{
    double v = x - X;
    if (!periodic(o, axis)) return v;
    double L = (double)o->n[axis];
    return v - L * floor(v / L + 0.5);
}

/* prescribed pose: X(t) = X0 + (t - t0) U (the body Omega(t) of the problem
 * statement, Sec. 3, moving with a given velocity) */
static void pose(const or_body *b, long long t, double X[3])
{
    double dt = (double)(t - b->t0);
    for (int k = 0; k < 3; ++k) X[k] = b->X0[k] + dt * b->U[k];
}

/* orientation about z at step t: theta(t) = theta0 + (t - t0) W_z */
static double orient(const or_body *b, long long t)
{
    double dt = (double)(t - b->t0);
    return b->theta0 + dt * b->W[2];
}

/*
 * sin and cos by the Cody-Waite reduction (Cody & Waite, "Software Manual for
 * the Elementary Functions", 1980): k = nearest integer to x 2/pi, r = x - k pi/2
 * with pi/2 split into three parts (the first two of 33 significant bits, so
 * k P1 and k P2 are exact for |k| < 2^20), then the Taylor series of sin and
 * cos on |r| <= pi/4 (terms to r^19 / r^18: truncation below 1e-19) in
 * Horner form, and the quadrant of k.  Written out here so that the result is
 * the same on every machine (the library evaluates the same formula).
 */
static void sincos_cw(double x, double *s_out, double *c_out)
{
    const double P1 = 0x1.921fb544p+0;
    const double P2 = 0x1.0b4611a6p-34;
    const double P3 = 0x1.3198a2e037073p-69;
    double kf = nearbyint(x * 0.6366197723675814);
    double r = ((x - kf * P1) - kf * P2) - kf * P3;
    double r2 = r * r;
    double ps = 8.22063524662433e-18;
    ps = ps * r2 - 2.8114572543455206e-15;
    ps = ps * r2 + 7.647163731819816e-13;
    ps = ps * r2 - 1.6059043836821613e-10;
    ps = ps * r2 + 2.505210838544172e-08;
    ps = ps * r2 - 2.7557319223985893e-06;
    ps = ps * r2 + 0.0001984126984126984;
    ps = ps * r2 - 0.008333333333333333;
    ps = ps * r2 + 0.16666666666666666;
    double sr = r - r * r2 * ps; /* r - r^3/3! + ... */
    double pc = 1.5619206968586225e-16;
    pc = pc * r2 - 4.779477332387385e-14;
    pc = pc * r2 + 1.1470745597729725e-11;
    pc = pc * r2 - 2.08767569878681e-09;
    pc = pc * r2 + 2.755731922398589e-07;
    pc = pc * r2 - 2.48015873015873e-05;
    pc = pc * r2 + 0.001388888888888889;
    pc = pc * r2 - 0.041666666666666664;
    pc = pc * r2 + 0.5;
    double cr = 1.0 - r2 * pc; /* 1 - r^2/2! + ... */
    long q = (long)kf & 3;
    if (q == 0) {
        *s_out = sr;
        *c_out = cr;
    } else if (q == 1) {
        *s_out = cr;
        *c_out = -sr;
    } else if (q == 2) {
        *s_out = -sr;
        *c_out = -cr;
    } else {
        *s_out = -cr;
        *c_out = sr;
    }
}

static void disp(const or_dom *o, const double X[3], int x, int y, int z, double r[3])
{
    r[0] = axis_disp(o, 0, (double)x, X[0]);
    r[1] = axis_disp(o, 1, (double)y, X[1]);
    r[2] = axis_disp(o, 2, (double)z, X[2]);
}

static void cross(const double a[3], const double b[3], double out[3])
{
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

/* rigid-body velocity at offset r from the centre: U + W x r (the wall
 * velocity u_B of Eq. Fillipova_interpolation at the wall point, and the
 * frame velocity v of Eqs. ForceInMovementMovingFrame /
 * TorqueInMovementMovingFrame) */
static void body_velocity(const or_body *b, const double r[3], double v[3])
{
    double wr[3];
    cross(b->W, r, wr);
    for (int k = 0; k < 3; ++k) v[k] = b->U[k] + wr[k];
}

/* coordinates of an offset in the ellipse's own axes (orientation co, si) */
static void body_axes(double co, double si, const double v[3], double *xi, double *eta)
{
    *xi = co * v[0] + si * v[1];
    *eta = co * v[1] - si * v[0];
}

/* membership of Omega(t): |r| <= R (sphere), the x-y distance (cylinder), the
 * body-axes form (ellipse, the test section's sedimenting ellipse); r: offset
 * from the centre; co, si: cos and sin of the body's orientation */
static int inside(const or_body *b, const double r[3], double co, double si)
{
    int in;
    if (b->shape == OR_SHAPE_ELLIPSE) {
        double xi, eta;
        body_axes(co, si, r, &xi, &eta);
        double qx = xi / b->R, qy = eta / b->R2;
        in = qx * qx + qy * qy <= 1.0;
    } else {
        double s = r[0] * r[0] + r[1] * r[1];
        if (b->shape == OR_SHAPE_SPHERE) s = s + r[2] * r[2];
        in = s <= b->R * b->R;
    }
    return b->invert ? !in : in;
}

/*
 * Fractional distance Delta = |x_F - x_B| / |x_F - x_A| (Sec. 2.1): the
 * root s in (0,1] of |d - s c|^2 = R^2 with d = x_F - X (fluid node relative
 * to the centre) and c = c_i, so that x_B = x_F - Delta c_i.  For an ellipse
 * the same quadratic in the scaled body axes (the surface is the unit circle
 * there).
 */
static double link_delta(const or_body *b, const double d[3], const int ci[3], double co, double si)
{
    if (b->halfway) return 0.5;
    double cx = ci[0], cy = ci[1], cz = ci[2];
    double a, bb, cc;
    if (b->shape == OR_SHAPE_ELLIPSE) {
        /* |d' - s c'|^2 in the metric diag(1/R^2, 1/R2^2) of the body's axes */
        const double cv[3] = {cx, cy, cz};
        double dx, dy, kx, ky;
        body_axes(co, si, d, &dx, &dy);
        body_axes(co, si, cv, &kx, &ky);
        dx = dx / b->R;
        dy = dy / b->R2;
        kx = kx / b->R;
        ky = ky / b->R2;
        a = kx * kx + ky * ky;
        bb = dx * kx + dy * ky;
        cc = (dx * dx + dy * dy) - 1.0;
    } else if (b->shape == OR_SHAPE_SPHERE) {
        a = cx * cx + cy * cy + cz * cz;
        bb = d[0] * cx + d[1] * cy + d[2] * cz;
        cc = (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - b->R * b->R;
    } else {
        a = cx * cx + cy * cy;
        bb = d[0] * cx + d[1] * cy;
        cc = (d[0] * d[0] + d[1] * d[1]) - b->R * b->R;
    }
    double disc = bb * bb - a * cc;
    if (disc < 0.0) disc = 0.0;
    double s;
    if (!b->invert) {
        s = cc / (bb + sqrt(disc)); /* x_F outside: the smaller root */
    } else {                        /* x_F inside, link leaves the surface */
        if (bb >= 0.0) s = (bb + sqrt(disc)) / a;
        else s = cc / (bb - sqrt(disc));
    }
    if (s > 1.0) s = 1.0;
    if (s < 0.0) s = 0.0;
    return s;
}

/* ---- equilibria ------------------------------------------------------------ */

/* f_i^eq(rho, u): quasi-incompressible (He-Luo, Sec. 2) or standard form */
static double feq(const or_dom *o, int i, double rho, const double u[3])
{
    const int *c = o->c[i];
    double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if (o->d.eq == 0) return o->w[i] * (rho + o->d.rho0 * (3.0 * cu + 4.5 * cu * cu - 1.5 * usq));
    return o->w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
}

/* fictitious equilibrium g_ib of Eq. Fillipova_equilibrium: u_bf in the
 * linear term, u_F in the quadratic terms, density rho_F of the fluid node */
static double geq(const or_dom *o, int ib, double rhoF, const double ubf[3], const double uF[3])
{
    const int *c = o->c[ib];
    double cbu = c[0] * ubf[0] + c[1] * ubf[1] + c[2] * ubf[2];
    double cbF = c[0] * uF[0] + c[1] * uF[1] + c[2] * uF[2];
    double uFsq = uF[0] * uF[0] + uF[1] * uF[1] + uF[2] * uF[2];
    if (o->d.eq == 0)
        return o->w[ib] * (rhoF + o->d.rho0 * (3.0 * cbu + 4.5 * cbF * cbF - 1.5 * uFsq));
    return o->w[ib] * rhoF * (1.0 + 3.0 * cbu + 4.5 * cbF * cbF - 1.5 * uFsq);
}

/* moments of the populations of one node (Eqs. LBMmacroscopics_0/1); the
 * momentum is divided by rho0 in the quasi-incompressible model */
static void moments(const or_dom *o, const double *fa, long x, double *rho_out, double u_out[3])
{
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < o->Q; ++i) {
        double fi = fa[(long)i * o->N + x];
        rho += fi;
        j[0] += o->c[i][0] * fi;
        j[1] += o->c[i][1] * fi;
        j[2] += o->c[i][2] * fi;
    }
    if (o->d.has_force)
        for (int k = 0; k < 3; ++k) j[k] += 0.5 * o->d.g[k];
    double den = o->d.eq == 0 ? o->d.rho0 : rho;
    *rho_out = rho;
    for (int k = 0; k < 3; ++k) u_out[k] = j[k] / den;
}

/* BGK collision of one node (Eq. collision), Guo source if a force is set */
static void collide_node(const or_dom *o, const double *fin, double *fout, long x, double rho,
                         const double u[3])
{
    double omega = 1.0 / o->d.tau;
    for (int i = 0; i < o->Q; ++i) {
        double fi = fin[(long)i * o->N + x];
        double v = fi - omega * (fi - feq(o, i, rho, u));
        if (o->d.has_force) {
            const int *c = o->c[i];
            const double *g = o->d.g;
            double cg = c[0] * g[0] + c[1] * g[1] + c[2] * g[2];
            double ug = u[0] * g[0] + u[1] * g[1] + u[2] * g[2];
            double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
            v = v + (1.0 - 0.5 * omega) * o->w[i] * (3.0 * (cg - ug) + 9.0 * cu * cg);
        }
        fout[(long)i * o->N + x] = v;
    }
}

/* ---- link classification ---------------------------------------------------- */

enum { K_FLUID = 0, K_BODY = 1, K_WALL = 2, K_INLET = 3, K_OUTLET = 4 };

/*
 * Where does population i of fluid node (x,y,z) stream from?  The source is
 * s = x - c_i.  Periodic axes wrap.  An out-of-range source on a wall axis
 * is a wall link; otherwise on the inlet side an inlet link, on the outlet
 * side an outlet copy.  A wall takes precedence at corners.
 */
static int classify(const or_dom *o, int x, int y, int z, int i, long *src, int *body)
{
    int p[3] = {x - o->c[i][0], y - o->c[i][1], z - o->c[i][2]};
    int wall = 0, inlet = 0, outlet = 0;
    for (int a = 0; a < 3; ++a) {
        int side = -1;
        if (p[a] < 0) side = 0;
        else if (p[a] >= o->n[a]) side = 1;
        if (side < 0) continue;
        int e = o->d.edge[2 * a + side];
        if (e == OR_PERIODIC) p[a] += side == 0 ? o->n[a] : -o->n[a];
        else if (e == OR_WALL) wall = 1;
        else if (e == OR_INLET) inlet = 1;
        else if (e == OR_OUTLET) {
            outlet = 1;
            p[a] = o->n[a] - 1; /* zero-gradient: copy the last interior column */
        }
    }
    *body = -1;
    if (wall) return K_WALL;
    if (inlet) return K_INLET;
    if (outlet) {
        *src = cell(o, p[0], p[1], p[2]);
        return K_OUTLET;
    }
    *src = cell(o, p[0], p[1], p[2]);
    if (o->solid[*src] >= 0) {
        *body = o->solid[*src];
        return K_BODY;
    }
    return K_FLUID;
}

/* boundary velocity of an edge link at the wall point x_B = x_F - c_i / 2 */
static void edge_velocity(const or_dom *o, int kind, int y, int i, double uB[3])
{
    uB[0] = uB[1] = uB[2] = 0.0;
    if (kind != K_INLET) return;
    if (!o->d.inlet_parabolic) {
        uB[0] = o->d.u_in;
        return;
    }
    double ny = (double)o->n[1];
    double yb = (double)y - 0.5 * (double)o->c[i][1];
    uB[0] = 4.0 * o->d.u_in * (yb + 0.5) * ((ny - 0.5) - yb) / (ny * ny);
}

/*
 * Curved-wall value fhat_i(x_A, t) of Eq. Fillipova_interpolation for the
 * link from solid node A = x - c_i to fluid node F = x (c_i points A -> F).
 * The moving-wall term is read as +2 w_i rho_w 3 c_i.u_B (c_i pointing into
 * the fluid): this makes a co-moving uniform flow a fixed point.
 */
static double wall_value(const or_dom *o, long x, int xx, int yy, int zz, int i, double delta,
                         const double uB[3], long long *fallback)
{
    int ib = o->opp[i];
    double fb = o->fhat[(long)ib * o->N + x];
    double rhoF = o->rho[x];
    double uF[3] = {o->u[3 * x], o->u[3 * x + 1], o->u[3 * x + 2]};
    double ubf[3], chi;
    if (delta < 0.5) {
        /* u_bf = u_G = u(x_F + c_i, t), chi = (2 Delta - 1)/(tau - 2) */
        int p[3] = {xx + o->c[i][0], yy + o->c[i][1], zz + o->c[i][2]};
        int ok = 1;
        for (int a = 0; a < 3; ++a) {
            if (p[a] >= 0 && p[a] < o->n[a]) continue;
            if (!periodic(o, a)) ok = 0;
            else p[a] += p[a] < 0 ? o->n[a] : -o->n[a];
        }
        long G = ok ? cell(o, p[0], p[1], p[2]) : -1;
        if (ok && o->solid[G] < 0) {
            for (int k = 0; k < 3; ++k) ubf[k] = o->u[3 * G + k];
            chi = (2.0 * delta - 1.0) / (o->d.tau - 2.0);
        } else {
            /* no fluid node G: plain (moving) bounce-back, counted */
            for (int k = 0; k < 3; ++k) ubf[k] = uF[k];
            chi = 0.0;
            ++*fallback;
        }
    } else {
        /* u_bf = u_F + 3/(2 Delta) (u_B - u_F), chi = (2 Delta - 1)/(tau + 1/2) */
        double k3 = 3.0 / (2.0 * delta);
        for (int k = 0; k < 3; ++k) ubf[k] = uF[k] + k3 * (uB[k] - uF[k]);
        chi = (2.0 * delta - 1.0) / (o->d.tau + 0.5);
    }
    double g = geq(o, ib, rhoF, ubf, uF);
    double rhow = o->d.eq == 0 ? o->d.rho0 : rhoF;
    const int *c = o->c[i];
    double cuB = c[0] * uB[0] + c[1] * uB[1] + c[2] * uB[2];
    return (1.0 - chi) * fb + chi * g + 2.0 * o->w[i] * rhow * 3.0 * cuB;
}

/* ---- geometry ----------------------------------------------------------------- */

/* solid owner of every node for the body poses at step t (bounding boxes):
 * the solid set whose change from t to t+1 gives the covered and uncovered
 * nodes A+ / A- of Sec. 3 */
static void rasterise(or_dom *o, long long t, int *owner)
{
    for (long x = 0; x < o->N; ++x) owner[x] = -1;
    for (int bi = 0; bi < o->nb; ++bi) {
        const or_body *b = &o->b[bi];
        double X[3], so, co;
        pose(b, t, X);
        sincos_cw(orient(b, t), &so, &co);
        if (b->invert) { /* solid outside: test the whole lattice */
            for (int z = 0; z < o->n[2]; ++z)
                for (int y = 0; y < o->n[1]; ++y)
                    for (int x = 0; x < o->n[0]; ++x) {
                        double r[3];
                        disp(o, X, x, y, z, r);
                        if (inside(b, r, co, so)) owner[cell(o, x, y, z)] = bi;
                    }
            continue;
        }
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            int use = a < 2 || b->shape == OR_SHAPE_SPHERE;
            if (!use) {
                lo[a] = 0;
                hi[a] = o->n[a] - 1;
                continue;
            }
            lo[a] = (int)floor(X[a] - b->R) - 1;
            hi[a] = (int)ceil(X[a] + b->R) + 1;
            if (hi[a] - lo[a] + 1 > o->n[a]) {
                lo[a] = 0;
                hi[a] = o->n[a] - 1;
            }
        }
        for (int zz = lo[2]; zz <= hi[2]; ++zz)
            for (int yy = lo[1]; yy <= hi[1]; ++yy)
                for (int xx = lo[0]; xx <= hi[0]; ++xx) {
                    int p[3] = {xx, yy, zz}, ok = 1;
                    for (int a = 0; a < 3; ++a) {
                        if (p[a] >= 0 && p[a] < o->n[a]) continue;
                        if (!periodic(o, a)) ok = 0;
                        else p[a] = ((p[a] % o->n[a]) + o->n[a]) % o->n[a];
                    }
                    if (!ok) continue;
                    double r[3];
                    disp(o, X, p[0], p[1], p[2], r);
                    if (inside(b, r, co, so)) owner[cell(o, p[0], p[1], p[2])] = bi;
                }
    }
}

/* ---- public API ------------------------------------------------------------------- */

void or_destroy(or_dom *o)
{
    if (!o) return;
    free(o->f);
    free(o->fhat);
    free(o->fnew);
    free(o->rho);
    free(o->u);
    free(o->solid);
    free(o->solid_next);
    free(o->b);
    free(o->series);
    free(o->imp_prev);
    free(o->pre);
    free(o->pre_set);
    free(o);
}

/* initial state: f = f^eq(rho = 1, u0) at every node (Eq. collision's
 * equilibrium in the quasi-incompressible form of Eqs. LBMmacroscopics) */
static void init_state(or_dom *o)
{
    for (long x = 0; x < o->N; ++x)
        for (int i = 0; i < o->Q; ++i) o->f[(long)i * o->N + x] = feq(o, i, 1.0, o->d.u0);
}

or_dom *or_create(const or_desc *d)
{
    if (!d || (d->q != 9 && d->q != 19)) return NULL;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return NULL;
    if (d->q == 9 && d->nz != 1) return NULL;
    for (int a = 0; a < 3; ++a)
        if ((d->edge[2 * a] == OR_PERIODIC) != (d->edge[2 * a + 1] == OR_PERIODIC)) return NULL;
    if (d->q == 9 && d->edge[4] != OR_PERIODIC) return NULL;
    for (int e = 0; e < 6; ++e) {
        if (d->edge[e] == OR_INLET && e != 0) return NULL;
        if (d->edge[e] == OR_OUTLET && e != 1) return NULL;
    }
    if (!(d->tau > 0.5)) return NULL;
    if (d->edge_rule != 0 && d->edge_rule != 1) return NULL;
    if (d->free_scheme < 0 || d->free_scheme > 2) return NULL;
    if (d->edge_rule == 1) { /* Zou-He faces: an inner neighbour distinct from both faces */
        const int nn[3] = {d->nx, d->ny, d->nz};
        for (int a = 0; a < 3; ++a)
            if (d->edge[2 * a] != OR_PERIODIC && nn[a] < 3) return NULL;
    }
    or_dom *o = (or_dom *)calloc(1, sizeof(or_dom));
    if (!o) return NULL;
    o->d = *d;
    o->Q = d->q;
    o->D = d->q == 9 ? 2 : 3;
    o->n[0] = d->nx;
    o->n[1] = d->ny;
    o->n[2] = d->nz;
    o->N = (long)d->nx * d->ny * d->nz;
    int cflat[57];
    or_lattice(o->Q, cflat, o->w, o->opp);
    for (int i = 0; i < o->Q; ++i)
        for (int k = 0; k < 3; ++k) o->c[i][k] = cflat[3 * i + k];
    size_t pq = sizeof(double) * (size_t)o->Q * (size_t)o->N;
    o->f = (double *)malloc(pq);
    o->fhat = (double *)malloc(pq);
    o->fnew = (double *)malloc(pq);
    o->rho = (double *)malloc(sizeof(double) * (size_t)o->N);
    o->u = (double *)calloc(3 * (size_t)o->N, sizeof(double));
    o->solid = (int *)malloc(sizeof(int) * (size_t)o->N);
    o->solid_next = (int *)malloc(sizeof(int) * (size_t)o->N);
    if (d->free_scheme == 2) {
        o->pre = (double *)malloc(pq);
        o->pre_set = (char *)calloc((size_t)o->N, 1);
    }
    if (!o->f || !o->fhat || !o->fnew || !o->rho || !o->u || !o->solid || !o->solid_next ||
        (d->free_scheme == 2 && (!o->pre || !o->pre_set))) {
        or_destroy(o);
        return NULL;
    }
    memset(o->fhat, 0, pq);
    memset(o->fnew, 0, pq);
    for (long x = 0; x < o->N; ++x) o->solid[x] = -1;
    init_state(o);
    return o;
}

int or_set_bodies(or_dom *o, const or_body *b, int nb)
{
    if (!o || nb < 0 || (nb > 0 && !b)) return OR_ERR_ARG;
    if (o->t != 0) return OR_ERR_STATE;
    free(o->b);
    o->b = NULL;
    o->nb = nb;
    if (nb) {
        o->b = (or_body *)malloc(sizeof(or_body) * (size_t)nb);
        if (!o->b) return OR_ERR_OOM;
        memcpy(o->b, b, sizeof(or_body) * (size_t)nb);
    }
    free(o->imp_prev);
    o->imp_prev = (double *)calloc((size_t)(nb ? nb : 1) * 6, sizeof(double));
    if (!o->imp_prev) return OR_ERR_OOM;
    free(o->series);
    o->series = NULL;
    o->nrec = o->cap = 0;
    rasterise(o, o->t, o->solid);
    init_state(o);
    return OR_OK;
}

int or_set_f(or_dom *o, const double *f)
{
    if (!o || !f) return OR_ERR_ARG;
    memcpy(o->f, f, sizeof(double) * (size_t)o->Q * (size_t)o->N);
    return OR_OK;
}

static int record_row(or_dom *o, const double *row)
{
    if (o->nrec == o->cap) {
        long long nc = o->cap ? 2 * o->cap : 64;
        double *s = (double *)realloc(o->series, sizeof(double) * (size_t)nc * (size_t)(o->nb ? o->nb : 1) * OR_ROW);
        if (!s) return OR_ERR_OOM;
        o->series = s;
        o->cap = nc;
    }
    if (o->nb)
        memcpy(o->series + (size_t)o->nrec * o->nb * OR_ROW, row, sizeof(double) * (size_t)o->nb * OR_ROW);
    o->nrec++;
    return OR_OK;
}

/*
 * Extrapolation refill (refill rule 2, after the extrapolation of the cited
 * Lallemand-Luo proposal, Sec. 3, discussion after Eq. ForceInMovement): the
 * node A = (x, y, z) uncovered between t and t+1 takes, per direction i,
 *     f_i(A, t+1) = 3 fhat_i(A + c*, t) - 3 fhat_i(A + 2c*, t) + fhat_i(A + 3c*, t),
 * the quadratic extrapolation along the lattice direction c* closest to the
 * outward surface normal n at A (largest n.c / |c|, the first such direction in
 * direction order).  n is the gradient of the body's shape function at the
 * pose of t+1: r (sphere), (r_x, r_y, 0) (cylinder), and for the ellipse the
 * gradient (xi / R^2, eta / R2^2) of its body-axes form turned back into the
 * lattice axes.  The three nodes must lie in the lattice (periodic axes wrap)
 * and be fluid at t; otherwise the function returns 0 and the equilibrium rule
 * applies.  Returns the direction index of c* and the three cells.
 */
static int extrap_nodes(const or_dom *o, const or_body *b, long long t, int x, int y, int z, long nodes[3])
{
    const double INV_SQRT2 = 0.70710678118654752440;
    double X1[3], r1[3], n[3];
    pose(b, t + 1, X1);
    disp(o, X1, x, y, z, r1);
    if (b->shape == OR_SHAPE_ELLIPSE) {
        double so, co, xi, eta;
        sincos_cw(orient(b, t + 1), &so, &co);
        body_axes(co, so, r1, &xi, &eta);
        double gx = xi / (b->R * b->R), gy = eta / (b->R2 * b->R2);
        n[0] = co * gx - so * gy;
        n[1] = so * gx + co * gy;
        n[2] = 0.0;
    } else {
        n[0] = r1[0];
        n[1] = r1[1];
        n[2] = b->shape == OR_SHAPE_SPHERE ? r1[2] : 0.0;
    }
    if (b->invert)
        for (int a = 0; a < 3; ++a) n[a] = -n[a];
    int best = 0;
    double top = 0.0;
    for (int i = 1; i < o->Q; ++i) {
        const int *c = o->c[i];
        double s = ((double)c[0] * n[0] + (double)c[1] * n[1]) + (double)c[2] * n[2];
        int len2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        double score = len2 == 1 ? s : s * INV_SQRT2;
        if (best == 0 || score > top) {
            best = i;
            top = score;
        }
    }
    for (int k = 1; k <= 3; ++k) {
        int p[3];
        for (int a = 0; a < 3; ++a) {
            p[a] = (a == 0 ? x : a == 1 ? y : z) + k * o->c[best][a];
            if (p[a] >= 0 && p[a] < o->n[a]) continue;
            if (!periodic(o, a)) return 0;
            p[a] = ((p[a] % o->n[a]) + o->n[a]) % o->n[a];
        }
        long q = cell(o, p[0], p[1], p[2]);
        if (o->solid[q] >= 0) return 0;
        nodes[k - 1] = q;
    }
    return best;
}

/*
 * Zou-He velocity condition (edge rule 1; the paper's test section imposes
 * its no-slip walls this way, after its cited reference).  The nodes of a
 * wall or inlet face lie ON the boundary (walls at the node layers 0 and
 * n - 1, not half-way) with a prescribed velocity u_w: 0 on walls; on the
 * inlet u_in, or the on-node parabola 4 u_in y (H - y) / H^2, H = ny - 1.
 * After streaming, the populations that would come from outside the face are
 * closed from the known ones at the same node:
 *   a node on one such face, outward normal n (axis a, sign s):
 *     j = rho_u u_w - g/2  (the Guo-shifted momentum sum_i c_i f_i; rho_u is
 *         rho0 in the quasi-incompressible model, rho otherwise),
 *     rho = S0 + 2 S+ - j.n, i.e. rho (1 + u_w.n) = S0 + 2 S+ + g.n/2 in the
 *         standard model (S0: the populations with c.n = 0, S+: c.n > 0),
 *     f_i = f_ib + 6 w_i c_i.j - sum_t c_i,t N_t   for every c_i.n < 0,
 *     N_t = T_t / 2 - j_t / 3 with T_t = sum over c.n = 0 of f c_t, for the
 *         two (one in 2-D) tangential axes t;
 *   so that sum_i f_i = rho and sum_i c_i f_i = j exactly (up to rounding);
 *   a node on two or three such faces (an edge or corner): u_w = 0 (a wall
 *     wins over the inlet) without the force shift (sum_i c_i f_i = 0 there),
 *     rho = the density at t of the inner diagonal
 *     neighbour (one step inward along each face normal) taken as the sum of
 *     its fhat(t), every unknown population whose opposite is known bounces
 *     back (f_i = f_ib), along the axis of a 3-D edge those bounced
 *     populations carry a correction that cancels the momentum of the known
 *     ones, and the unknown pairs whose opposite is unknown too share the
 *     rest of rho equally.
 */
static int zh_face(const or_dom *o, int a, int side)
{
    int e = o->d.edge[2 * a + side];
    return e == OR_WALL || e == OR_INLET;
}

static void zouhe_node(or_dom *o, int x, int y, int z)
{
    const long N = o->N;
    const int Q = o->Q;
    const int pos[3] = {x, y, z};
    int nface = 0, axis = 0, sgn = 0, wall = 0, inward[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) {
        if (pos[a] == 0 && zh_face(o, a, 0)) {
            nface++;
            axis = a;
            sgn = -1;
            inward[a] = 1;
            wall |= o->d.edge[2 * a] == OR_WALL;
        } else if (pos[a] == o->n[a] - 1 && zh_face(o, a, 1)) {
            nface++;
            axis = a;
            sgn = 1;
            inward[a] = -1;
            wall |= o->d.edge[2 * a + 1] == OR_WALL;
        }
    }
    if (nface == 0) return;
    const long xc = cell(o, x, y, z);
    if (o->solid[xc] >= 0) return;
    double f[19];
    int unknown[19];
    for (int i = 0; i < Q; ++i) {
        long s = -1;
        int body;
        int k = classify(o, x, y, z, i, &s, &body);
        f[i] = o->fnew[(long)i * N + xc];
        unknown[i] = k == K_WALL || k == K_INLET;
    }
    if (nface == 1) {
        double uw[3] = {0.0, 0.0, 0.0}, g[3] = {0.0, 0.0, 0.0}, j[3], T[3] = {0.0, 0.0, 0.0};
        if (!wall) {
            if (!o->d.inlet_parabolic) {
                uw[0] = o->d.u_in;
            } else {
                double H = (double)(o->n[1] - 1);
                uw[0] = 4.0 * o->d.u_in * (double)y * (H - (double)y) / (H * H);
            }
        }
        if (o->d.has_force)
            for (int a = 0; a < 3; ++a) g[a] = o->d.g[a];
        double S0 = 0.0, Sp = 0.0;
        for (int i = 0; i < Q; ++i) {
            int cn = o->c[i][axis] * sgn;
            if (cn == 0) {
                S0 += f[i];
                for (int a = 0; a < 3; ++a) T[a] += o->c[i][a] * f[i];
            } else if (cn > 0) {
                Sp += f[i];
            }
        }
        if (o->d.eq == 0) { /* the density follows: rho = S0 + 2 S+ - j.n */
            for (int a = 0; a < 3; ++a) j[a] = o->d.rho0 * uw[a] - 0.5 * g[a];
        } else {
            double rho = ((S0 + 2.0 * Sp) + (double)sgn * (0.5 * g[axis])) / (1.0 + (double)sgn * uw[axis]);
            for (int a = 0; a < 3; ++a) j[a] = rho * uw[a] - 0.5 * g[a];
        }
        double Nt[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < 3; ++a)
            if (a != axis) Nt[a] = 0.5 * T[a] - j[a] / 3.0;
        for (int i = 0; i < Q; ++i) {
            if (!unknown[i]) continue;
            const int *c = o->c[i];
            double cj = ((double)c[0] * j[0] + (double)c[1] * j[1]) + (double)c[2] * j[2];
            double v = f[o->opp[i]] + (6.0 * o->w[i]) * cj;
            for (int a = 0; a < 3; ++a)
                if (a != axis && c[a] != 0) v = v - (double)c[a] * Nt[a];
            o->fnew[(long)i * N + xc] = v;
        }
        return;
    }
    const long xin = cell(o, x + inward[0], y + inward[1], z + inward[2]);
    double rc = 0.0;
    for (int i = 0; i < Q; ++i) rc += o->fhat[(long)i * N + xin];
    int buried[19], nbur = 0;
    for (int i = 0; i < Q; ++i) {
        buried[i] = unknown[i] && unknown[o->opp[i]];
        nbur += buried[i];
    }
    for (int i = 0; i < Q; ++i)
        if (unknown[i] && !buried[i]) f[i] = f[o->opp[i]];
    /* along an axis with no face at the node (the axis of a 3-D edge) the
     * bounced pairs carry no momentum, the known pairs carry T; the m
     * bounced populations moving along it take -c T / m, so the momentum
     * along it is 0 */
    for (int a = 0; a < 3; ++a) {
        if (inward[a] != 0) continue;
        double T = 0.0;
        int m = 0;
        for (int i = 0; i < Q; ++i) {
            if (o->c[i][a] == 0) continue;
            if (!unknown[i] && !unknown[o->opp[i]]) T += o->c[i][a] * f[i];
            if (unknown[i] && !buried[i]) m++;
        }
        if (m == 0) continue;
        double Nt = T / (double)m;
        for (int i = 0; i < Q; ++i)
            if (unknown[i] && !buried[i] && o->c[i][a] != 0) f[i] = f[i] - (double)o->c[i][a] * Nt;
    }
    double rest = rc;
    for (int i = 0; i < Q; ++i)
        if (!buried[i]) rest = rest - f[i];
    for (int i = 0; i < Q; ++i)
        if (buried[i]) f[i] = rest / (double)nbur;
    for (int i = 0; i < Q; ++i)
        if (unknown[i]) o->fnew[(long)i * N + xc] = f[i];
}

/* Covered (A+) and uncovered (A-) nodes between the solid set of t
 * (o->solid) and o->solid_next, rasterised by the caller for the poses of t+1
 * that the body records give (Sec. 3, after Eq. ForceInMovement).  An
 * uncovered node is refilled (rule of the descriptor, u_B from the body's
 * record at t+1); the impulsive terms of Eqs. ForceInMovement /
 * TorqueInMovement, -sum_{A-} sum_i c_i f_i(A, t+1) + sum_{A+} sum_i c_i
 * f_i(A, t+1) and the same with r(A) x (r about the pose of t, Xt), are added
 * into imp[nb][6] in cell order; f(A, t+1) is the streamed value of a covered
 * node and the refill of an uncovered one.  mode 0: the refill is stored in
 * fnew; mode 1 (a predicted displacement): nothing is stored in fnew, the
 * refill goes to o->pre (o->pre_set marks the node) and the predicted solid
 * set is kept; mode 2 (the recomputed displacement after a prediction): a
 * node the prediction also uncovered takes the refill the prediction
 * computed, any other uncovered node a fresh one; nodes whose change differs
 * from the prediction are counted. */
static void cover_uncover(or_dom *o, long long t, const double *Xt, int mode, double *imp)
{
    const long N = o->N;
    const int Q = o->Q;
    const int nx = o->n[0], ny = o->n[1], nz = o->n[2];
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long A = cell(o, x, y, z);
                int was = o->solid[A], now = o->solid_next[A];
                if (mode == 2 && ((o->pre_set[A] == 2) != (was < 0 && now >= 0) ||
                                  (o->pre_set[A] == 1) != (was >= 0 && now < 0)))
                    o->n_mismatch++;
                if ((was >= 0) == (now >= 0)) {
                    if (mode == 2) o->pre_set[A] = 0;
                    continue;
                }
                int bi = was >= 0 ? was : now;
                const or_body *b = &o->b[bi];
                double fv[19];
                if (was >= 0) {
                    if (mode == 2 && o->pre_set[A] == 1) {
                        for (int i = 0; i < Q; ++i) fv[i] = o->pre[(long)i * N + A];
                    } else {
                        /* uncovered: refill with an equilibrium (Sec. 3) */
                        double X1[3], r1[3], uB[3];
                        pose(b, t + 1, X1);
                        disp(o, X1, x, y, z, r1);
                        body_velocity(b, r1, uB);
                        double sum = 0.0, us[3] = {0.0, 0.0, 0.0};
                        int cnt = 0;
                        for (int i = 1; i < Q; ++i) {
                            int p[3] = {x + o->c[i][0], y + o->c[i][1], z + o->c[i][2]}, ok = 1;
                            for (int a = 0; a < 3; ++a) {
                                if (p[a] >= 0 && p[a] < o->n[a]) continue;
                                if (!periodic(o, a)) ok = 0;
                                else p[a] += p[a] < 0 ? o->n[a] : -o->n[a];
                            }
                            if (!ok) continue;
                            long nbc = cell(o, p[0], p[1], p[2]);
                            if (o->solid[nbc] >= 0) continue;
                            sum += o->rho[nbc];
                            for (int a = 0; a < 3; ++a) us[a] += o->u[3 * nbc + a];
                            cnt++;
                        }
                        double rbar = cnt ? sum / (double)cnt : o->d.rho0;
                        double ufill[3];
                        for (int a = 0; a < 3; ++a)
                            ufill[a] = (o->d.refill == 1 && cnt) ? us[a] / (double)cnt : uB[a];
                        long en[3];
                        if (o->d.refill == 2 && extrap_nodes(o, b, t, x, y, z, en)) {
                            for (int i = 0; i < Q; ++i) {
                                const double *fh = o->fhat + (long)i * N;
                                fv[i] = (3.0 * fh[en[0]] - 3.0 * fh[en[1]]) + fh[en[2]];
                            }
                            if (mode != 1) o->n_extrap++;
                        } else {
                            for (int i = 0; i < Q; ++i) fv[i] = feq(o, i, rbar, ufill);
                        }
                    }
                    if (mode == 1) {
                        for (int i = 0; i < Q; ++i) o->pre[(long)i * N + A] = fv[i];
                        o->pre_set[A] = 1;
                    } else {
                        for (int i = 0; i < Q; ++i) o->fnew[(long)i * N + A] = fv[i];
                        if (mode == 2) o->pre_set[A] = 0;
                    }
                } else {
                    for (int i = 0; i < Q; ++i) fv[i] = o->fnew[(long)i * N + A];
                    if (mode == 1) o->pre_set[A] = 2;
                    if (mode == 2) o->pre_set[A] = 0;
                }
                /* impulsive terms of Eqs. ForceInMovement / TorqueInMovement */
                double m[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < Q; ++i) {
                    double fi = fv[i];
                    m[0] += o->c[i][0] * fi;
                    m[1] += o->c[i][1] * fi;
                    m[2] += o->c[i][2] * fi;
                }
                double r[3], tq[3];
                disp(o, Xt + 3 * bi, x, y, z, r);
                cross(r, m, tq);
                double *R = imp + (size_t)bi * 6;
                if (was >= 0) {
                    for (int a = 0; a < 3; ++a) {
                        R[a] -= m[a];
                        R[3 + a] -= tq[a];
                    }
                } else {
                    for (int a = 0; a < 3; ++a) {
                        R[a] += m[a];
                        R[3 + a] += tq[a];
                    }
                }
            }
}

/* Newton's and Euler's equations of a free body over one step (Sec. 4,
 * forward Euler): with the flow force F and torque T of step t (plus weight
 * less buoyancy (rho_b - rho0) V g) U(t+1) = U(t) + (F + (rho_b - rho0) V
 * g) / M and W(t+1) = W(t) + T / I, M = rho_b V, V = pi R^2 nz (cylinder),
 * pi R R2 nz (ellipse), 4/3 pi R^3 (sphere), I = M R^2 / 2 (cylinder, about
 * z), M (R^2 + R2^2) / 4 (ellipse), 2/5 M R^2 (sphere).  The body record then
 * starts at t+1: X(t+1) = X(t) + U(t) (semi = 0: the displacement the step
 * already made) or X(t) + U(t+1) (semi = 1), likewise the orientation. */
static void free_update(or_dom *o, or_body *b, long long t, const double F[3], const double T[3], int semi)
{
    const double PI = 3.14159265358979323846;
    double V, I;
    if (b->shape == OR_SHAPE_SPHERE) {
        V = 4.0 / 3.0 * PI * b->R * b->R * b->R;
    } else if (b->shape == OR_SHAPE_ELLIPSE) {
        V = PI * b->R * b->R2 * (double)o->n[2];
    } else {
        V = PI * b->R * b->R * (double)o->n[2];
    }
    double M = b->density_ratio * o->d.rho0 * V;
    if (b->shape == OR_SHAPE_SPHERE) I = 0.4 * M * b->R * b->R;
    else if (b->shape == OR_SHAPE_ELLIPSE) I = 0.25 * M * (b->R * b->R + b->R2 * b->R2);
    else I = 0.5 * M * b->R * b->R;
    double X1[3], X0[3];
    pose(b, t + 1, X1);
    pose(b, t, X0);
    double th1 = orient(b, t + 1);
    double th0 = orient(b, t);
    for (int a = 0; a < 3; ++a)
        b->U[a] = b->U[a] + (F[a] + (b->density_ratio - 1.0) * o->d.rho0 * V * o->d.gravity[a]) / M;
    if (b->shape == OR_SHAPE_SPHERE) {
        for (int a = 0; a < 3; ++a) b->W[a] = b->W[a] + T[a] / I;
    } else {
        b->W[2] = b->W[2] + T[2] / I;
    }
    if (semi) {
        for (int a = 0; a < 3; ++a) X1[a] = X0[a] + b->U[a];
        th1 = th0 + b->W[2];
    }
    for (int a = 0; a < 3; ++a) b->X0[a] = X1[a];
    b->theta0 = th1;
    b->t0 = t + 1;
}

static int one_step(or_dom *o)
{
    const long N = o->N;
    const int Q = o->Q;
    const int nx = o->n[0], ny = o->n[1], nz = o->n[2];
    const long long t = o->t;

    /* 1 + 2: moments and collision at the fluid nodes of Omega(t) */
#pragma omp parallel for schedule(static)
    for (long x = 0; x < N; ++x) {
        if (o->solid[x] >= 0) continue;
        double rho, u[3];
        moments(o, o->f, x, &rho, u);
        o->rho[x] = rho;
        for (int k = 0; k < 3; ++k) o->u[3 * x + k] = u[k];
        collide_node(o, o->f, o->fhat, x, rho, u);
    }

    /* 3: streaming, with the curved-wall value on every cut link */
    long long fallback = 0;
#pragma omp parallel for schedule(static) collapse(2) reduction(+ : fallback)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long xc = cell(o, x, y, z);
                if (o->solid[xc] >= 0) continue;
                for (int i = 0; i < Q; ++i) {
                    long s = -1;
                    int body;
                    int k = classify(o, x, y, z, i, &s, &body);
                    double v;
                    if (k == K_FLUID || k == K_OUTLET) {
                        v = o->fhat[(long)i * N + s];
                    } else if (k == K_BODY) {
                        const or_body *b = &o->b[body];
                        double X[3], d[3], uB[3], rB[3], so, co;
                        pose(b, t, X);
                        sincos_cw(orient(b, t), &so, &co);
                        disp(o, X, x, y, z, d);
                        double delta = link_delta(b, d, o->c[i], co, so);
                        for (int a = 0; a < 3; ++a) rB[a] = d[a] - delta * o->c[i][a];
                        body_velocity(b, rB, uB);
                        v = wall_value(o, xc, x, y, z, i, delta, uB, &fallback);
                    } else if (o->d.edge_rule == 1) {
                        v = 0.0; /* closed by zouhe_node below */
                    } else {
                        double uB[3];
                        edge_velocity(o, k, y, i, uB);
                        v = wall_value(o, xc, x, y, z, i, 0.5, uB, &fallback);
                    }
                    o->fnew[(long)i * N + xc] = v;
                }
            }
    o->n_fallback += fallback;
    if (o->d.edge_rule == 1)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) zouhe_node(o, x, y, z);

    /* 4: momentum exchange over the cut links, in cell and direction order.
     * By Eq. Equalities, fhat_i(x_A - c_i, t) is the wall value that streamed
     * into fnew_i(x_A) and fhat_ib(x_A, t) is the collided value at the fluid
     * node. */
    double *row = (double *)calloc((size_t)(o->nb ? o->nb : 1) * OR_ROW, sizeof(double));
    if (!row) return OR_ERR_OOM;
    for (int a = 0; a < 6; ++a) o->edge_me[a] = 0.0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long xc = cell(o, x, y, z);
                if (o->solid[xc] >= 0) continue;
                for (int i = 1; i < Q; ++i) {
                    long s = -1;
                    int body;
                    int k = classify(o, x, y, z, i, &s, &body);
                    if (k == K_FLUID || k == K_OUTLET) continue;
                    if (k != K_BODY && o->d.edge_rule == 1) continue; /* Zou-He faces have no links */
                    const int *c = o->c[i];
                    const int *cb = o->c[o->opp[i]];
                    double fa = o->fnew[(long)i * N + xc];
                    double fb = o->fhat[(long)o->opp[i] * N + xc];
                    double ps[3], tq[3];
                    double sum = fa + fb;
                    for (int a = 0; a < 3; ++a) ps[a] = -c[a] * sum;
                    if (k != K_BODY) { /* edge links: test hook, torque about the origin */
                        double r[3] = {(double)x, (double)y, (double)z};
                        cross(r, ps, tq);
                        for (int a = 0; a < 3; ++a) {
                            o->edge_me[a] += ps[a];
                            o->edge_me[3 + a] += tq[a];
                        }
                        continue;
                    }
                    const or_body *b = &o->b[body];
                    double X[3], d[3], rB[3], v[3], pm[3], so, co;
                    pose(b, t, X);
                    sincos_cw(orient(b, t), &so, &co);
                    disp(o, X, x, y, z, d);
                    double delta = link_delta(b, d, c, co, so);
                    for (int a = 0; a < 3; ++a) rB[a] = d[a] - delta * c[a];
                    body_velocity(b, rB, v);
                    double *R = row + (size_t)body * OR_ROW;
                    /* static form, Eqs. flow_force_2 / flow_torque_2 */
                    cross(d, ps, tq);
                    for (int a = 0; a < 3; ++a) {
                        R[a] += ps[a];
                        R[3 + a] += tq[a];
                    }
                    /* moving-frame form, Eqs. ForceInMovementMovingFrame /
                     * TorqueInMovementMovingFrame without their last two terms */
                    for (int a = 0; a < 3; ++a) pm[a] = -(c[a] - v[a]) * fa + (cb[a] - v[a]) * fb;
                    cross(d, pm, tq);
                    for (int a = 0; a < 3; ++a) {
                        R[12 + a] += pm[a];
                        R[15 + a] += tq[a];
                    }
                }
            }

    /* 5 + 6: body motion.  Prescribed bodies move with their given velocity;
     * the covered (A+) and uncovered (A-) nodes between t and t+1 give the
     * impulsive terms of Eqs. ForceInMovement / TorqueInMovement and the
     * refill of the uncovered nodes (Sec. 3).  Free bodies follow Newton's
     * and Euler's equations (Sec. 4) by one of three schemes:
     *   0  explicit: the body moves from t to t+1 with U(t), so the sets
     *      A+/A- of this step are known before the force; then U(t+1) from
     *      the force of step t (static plus impulsive terms);
     *   1  backward sets (the Aidun-type approximation of Sec. 3): the force
     *      at t takes the impulsive terms of the nodes that entered and left
     *      the body between t-1 and t, so U(t+1) follows before the body
     *      moves, and the displacement from t to t+1 is made with U(t+1);
     *   2  predictor-corrector (the second approximation of Sec. 3): the sets
     *      of a predicted displacement with U(t) give the force at t, U(t+1)
     *      follows, and the displacement is recomputed with U(t+1) -- two
     *      displacements per step; a node uncovered by both keeps the refill
     *      the force used. */
    const int scheme = o->d.free_scheme;
    int moving = 0, any_free = 0;
    for (int bi = 0; bi < o->nb; ++bi) {
        const or_body *b = &o->b[bi];
        for (int a = 0; a < 3; ++a)
            if (b->U[a] != 0.0 || b->W[a] != 0.0) moving = 1;
        if (b->free) moving = any_free = 1;
    }
    const size_t nb6 = (size_t)(o->nb ? o->nb : 1) * 6;
    double *imp = (double *)calloc(nb6, sizeof(double));
    double *imp_pred = (double *)calloc(nb6, sizeof(double));
    double *Xt = (double *)malloc(sizeof(double) * (size_t)(o->nb ? o->nb : 1) * 3);
    if (!imp || !imp_pred || !Xt) {
        free(imp);
        free(imp_pred);
        free(Xt);
        free(row);
        return OR_ERR_OOM;
    }
    for (int bi = 0; bi < o->nb; ++bi) pose(&o->b[bi], t, Xt + 3 * bi);
    const int predict = scheme == 2 && any_free;
    if (moving && predict) {
        rasterise(o, t + 1, o->solid_next); /* free bodies moving with U(t) */
        cover_uncover(o, t, Xt, 1, imp_pred);
    }
    if (scheme != 0) /* semi-implicit schemes: the velocity of t+1 first */
        for (int bi = 0; bi < o->nb; ++bi) {
            if (!o->b[bi].free) continue;
            const double *Rw = row + (size_t)bi * OR_ROW;
            const double *ip = scheme == 1 ? o->imp_prev + 6 * bi : imp_pred + 6 * bi;
            double F[3], T[3];
            for (int k = 0; k < 3; ++k) {
                F[k] = Rw[k] + ip[k];
                T[k] = Rw[3 + k] + ip[3 + k];
            }
            free_update(o, &o->b[bi], t, F, T, 1);
        }
    if (moving) {
        rasterise(o, t + 1, o->solid_next); /* the poses of t+1 */
        cover_uncover(o, t, Xt, predict ? 2 : 0, imp);
        int *tmp = o->solid;
        o->solid = o->solid_next;
        o->solid_next = tmp;
    }
    for (int bi = 0; bi < o->nb; ++bi) {
        double *R = row + (size_t)bi * OR_ROW;
        const or_body *b = &o->b[bi];
        const double *ip = imp + 6 * bi;
        if (b->free && scheme == 1) ip = o->imp_prev + 6 * bi;
        if (b->free && scheme == 2) ip = imp_pred + 6 * bi;
        for (int k = 0; k < 6; ++k) R[6 + k] = ip[k];
        if (b->free && scheme == 1)
            for (int k = 0; k < 6; ++k) o->imp_prev[6 * bi + k] = imp[6 * bi + k];
    }
    if (scheme == 0) /* explicit: U(t+1) from the force of step t */
        for (int bi = 0; bi < o->nb; ++bi) {
            if (!o->b[bi].free) continue;
            const double *Rw = row + (size_t)bi * OR_ROW;
            double F[3], T[3];
            for (int k = 0; k < 3; ++k) {
                F[k] = Rw[k] + Rw[6 + k];
                T[k] = Rw[3 + k] + Rw[9 + k];
            }
            free_update(o, &o->b[bi], t, F, T, 0);
        }
    free(imp);
    free(imp_pred);
    free(Xt);

    double *tmp = o->f;
    o->f = o->fnew;
    o->fnew = tmp;
    o->t = t + 1;
    int rc = record_row(o, row);
    free(row);
    return rc;
}

int or_step(or_dom *o, int n)
{
    if (!o || n < 0) return OR_ERR_ARG;
    for (int s = 0; s < n; ++s) {
        int rc = one_step(o);
        if (rc) return rc;
    }
    return OR_OK;
}

/* threads the OpenMP loops run on (1 when built without OpenMP) */
int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

long long or_time(const or_dom *o) { return o ? o->t : -1; }
long long or_fallbacks(const or_dom *o) { return o ? o->n_fallback : -1; }
long long or_extrapolated(const or_dom *o) { return o ? o->n_extrap : -1; }
long long or_mismatches(const or_dom *o) { return o ? o->n_mismatch : -1; }

/* series rows [first, first+count) of every body: out[count][nb][18] with
 * Fs Ts (static form), Fi Ti (impulsive terms), Fm Tm (moving frame) */
/* test hook: the sin / cos the oracle uses for body orientations */
void or_sincos(double x, double *s, double *c) { sincos_cw(x, s, c); }

/* body state at the current step t: X(t), U(t), W(t) (9 doubles per body) */
int or_get_bodies(const or_dom *o, double *out)
{
    if (!o || (o->nb && !out)) return OR_ERR_ARG;
    for (int bi = 0; bi < o->nb; ++bi) {
        double X[3];
        pose(&o->b[bi], o->t, X);
        for (int a = 0; a < 3; ++a) {
            out[9 * bi + a] = X[a];
            out[9 * bi + 3 + a] = o->b[bi].U[a];
            out[9 * bi + 6 + a] = o->b[bi].W[a];
        }
    }
    return OR_OK;
}

int or_get_series(const or_dom *o, long long first, long long count, double *out)
{
    if (!o || !out || first < 0 || count < 0 || first + count > o->nrec) return OR_ERR_ARG;
    if (o->nb)
        memcpy(out, o->series + (size_t)first * o->nb * OR_ROW, sizeof(double) * (size_t)count * o->nb * OR_ROW);
    return OR_OK;
}

int or_get_f(const or_dom *o, double *out)
{
    if (!o || !out) return OR_ERR_ARG;
    memcpy(out, o->f, sizeof(double) * (size_t)o->Q * (size_t)o->N);
    return OR_OK;
}

/* post-collision populations fhat(t) of the current state (solid nodes: 0) */
int or_get_fhat(const or_dom *o, double *out)
{
    if (!o || !out) return OR_ERR_ARG;
    memset(out, 0, sizeof(double) * (size_t)o->Q * (size_t)o->N);
    for (long x = 0; x < o->N; ++x) {
        if (o->solid[x] >= 0) continue;
        double rho, u[3];
        moments(o, o->f, x, &rho, u);
        collide_node(o, o->f, out, x, rho, u);
    }
    return OR_OK;
}

/* rho, ux, uy, uz of f(t) at every fluid node: out[4][N] (solid nodes: 0) */
int or_get_macro(const or_dom *o, double *out)
{
    if (!o || !out) return OR_ERR_ARG;
    memset(out, 0, sizeof(double) * 4 * (size_t)o->N);
    for (long x = 0; x < o->N; ++x) {
        if (o->solid[x] >= 0) continue;
        double rho, u[3];
        moments(o, o->f, x, &rho, u);
        out[x] = rho;
        for (int k = 0; k < 3; ++k) out[(long)(k + 1) * o->N + x] = u[k];
    }
    return OR_OK;
}

int or_get_solid(const or_dom *o, int *out)
{
    if (!o || !out) return OR_ERR_ARG;
    memcpy(out, o->solid, sizeof(int) * (size_t)o->N);
    return OR_OK;
}

int or_get_edge_me(const or_dom *o, double *out)
{
    if (!o || !out) return OR_ERR_ARG;
    memcpy(out, o->edge_me, sizeof(o->edge_me));
    return OR_OK;
}

/* cut links of body bi in the current geometry, in cell and direction order */
long long or_links(const or_dom *o, int bi, long long cap, long long *cells, int *dirs, double *deltas)
{
    if (!o || bi < 0 || bi >= o->nb) return -1;
    long long cnt = 0;
    for (int z = 0; z < o->n[2]; ++z)
        for (int y = 0; y < o->n[1]; ++y)
            for (int x = 0; x < o->n[0]; ++x) {
                long xc = cell(o, x, y, z);
                if (o->solid[xc] >= 0) continue;
                for (int i = 1; i < o->Q; ++i) {
                    long s = -1;
                    int body;
                    if (classify(o, x, y, z, i, &s, &body) != K_BODY || body != bi) continue;
                    if (cnt < cap) {
                        double X[3], d[3], so, co;
                        pose(&o->b[bi], o->t, X);
                        sincos_cw(orient(&o->b[bi], o->t), &so, &co);
                        disp(o, X, x, y, z, d);
                        if (cells) cells[cnt] = xc;
                        if (dirs) dirs[cnt] = i;
                        if (deltas) deltas[cnt] = link_delta(&o->b[bi], d, o->c[i], co, so);
                    }
                    cnt++;
                }
            }
    return cnt;
}
