/*
 * lbm_oracle.c - plain, slow FP64 CPU reference of the coupled lattice
 * Boltzmann / discrete element hot path of Mutabaruka & Kamrin, "A simulation
 * technique for slurries interacting with moving parts and deformable solids
 * with applications" (arXiv 1703.05158).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header,
 * table or helper with the CUDA library; the D3Q19 tables below are typed
 * from the paper's Table 1 and the weights stated under Eq. (9).
 *
 * One time step n -> n+1, in the order of Sect. 2.5 read with Sect. 2.3:
 *   1. geometry at X^n: owner of every node (fluid or sphere p)
 *   2. refill of nodes uncovered since step n-1 with the equilibrium (Eq. 9)
 *   3. collision, Eqs. (5), (6), (9), (12) with the Smagorinsky relaxation
 *      time of Eq. (18) and a body force (Guo, Zheng & Shi 2002)
 *   4. streaming, Eq. (13), with interpolated bounce-back on cut links,
 *      Eqs. (19) and (21); the z walls are cut links with q = 1/2
 *   5. momentum exchange force and torque on every sphere, Eqs. (25), (26)
 *   6. DEM: linear spring-dashpot normal contact, Eq. (1), integrated by
 *      velocity Verlet (Sect. 2.1) in dem_substeps sub-steps
 *
 * Options (off by default; the paper's own where marked): the tangential
 * spring, dashpot and Coulomb cap of Eqs. (2), (3) (paper's); the ZIEB face
 * of Sect. 2.6, Eqs. (8), (9), after step 5 (paper's); momentum correction
 * of covered / uncovered nodes (Aidun, Lu & Ding 1998); the
 * Galilean-invariant momentum exchange (Wen, Zhang & Fang 2014); an open
 * channel in x with a velocity inlet, a pressure outlet and a fixed plate,
 * the boundaries of the differentiation form, so that its objective (the
 * plate drag) can be evaluated with the spheres free.
 *
 * Arithmetic is FP64, except the geometric decisions (is a node inside a
 * sphere, which sphere owns it, the link fraction q and so which branch of
 * Eq. (19) applies) which are taken in FP32 from FP32 relative positions:
 * the GPU library takes the same decisions with the same FP32 operations, so
 * both sides agree on every node and link.  Build with -ffp-contract=off so
 * that no multiply-add is fused.
 *
 * Readings of passages the paper leaves open are marked "reading:".
 * Parity pins: every function below is pinned by tests in tests/ except the
 * transient of the full coupled moving-sphere trajectory, which has no
 * closed form; its steady state is pinned by Galilean invariance (a free
 * sphere's terminal velocity against the drag in the co-moving frame).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NQ 19

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Table 1: the D3Q19 velocity set, direction i = 0..18. */
static const int CX[NQ] = {0, -1, 0, 0, -1, -1, -1, -1, 0, 0, 1, 0, 0, 1, 1, 1, 1, 0, 0};
static const int CY[NQ] = {0, 0, -1, 0, -1, 1, 0, 0, -1, -1, 0, 1, 0, 1, -1, 0, 0, 1, 1};
static const int CZ[NQ] = {0, 0, 0, -1, 0, 0, -1, 1, -1, 1, 0, 0, 1, 0, 0, 1, -1, 1, -1};

/* Weight of direction i (text under Eq. 9): 1/3 at rest, 1/18 for the six
 * axis directions 1, 2, 3, 10, 11, 12, 1/36 for the twelve diagonals. */
static double weight(int i) {
    if (i == 0) return 1.0 / 3.0;
    if (i == 1 || i == 2 || i == 3 || i == 10 || i == 11 || i == 12) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

/* Opposite direction: the one whose velocity is -c_i, found from the table. */
static int opposite(int i) {
    for (int k = 0; k < NQ; ++k)
        if (CX[k] == -CX[i] && CY[k] == -CY[i] && CZ[k] == -CZ[i]) return k;
    return -1;
}

typedef struct {
    int nx, ny, nz;         /* lattice; x, y periodic; walls at z=-1/2, z=nz-1/2 */
    double tau0;            /* relaxation time, > 1/2 (Eq. 15) */
    double cs;              /* Smagorinsky constant C (Eq. 18) */
    double g[3];            /* body acceleration; force density rho*g */
    double u_lo[3];         /* velocity of the wall at z = -1/2 */
    double u_hi[3];         /* velocity of the wall at z = nz-1/2 */
    double rho_s;           /* sphere density (fluid reference density is 1) */
    double kn;              /* normal contact stiffness (Eq. 1) */
    double restitution;     /* normal restitution coefficient */
    int dem_substeps;       /* DEM sub-steps per lattice step */
    int les;                /* 1: Smagorinsky tau (Eq. 18); 0: plain BGK path */
    int fluid;              /* 0: DEM only, no lattice (hydrodynamic load 0) */
    int periodic_z;         /* 1: z periodic too (no walls) */
    int momentum_correction; /* 1: covered / uncovered nodes exchange their momentum with the sphere */
    double kt;              /* tangential contact stiffness (Eq. 2); friction is on when kt > 0 and mu > 0 */
    double mu;              /* Coulomb friction coefficient mu_s (Eq. 2) */
    double restitution_t;   /* tangential restitution, sets gamma_t (Eq. 2); 1: no tangential damping */
    int zieb;               /* 1: the plane z = 0 is a ZIEB face (Sect. 2.6) onto a virtual cylinder below */
    double zieb_area;       /* piston (and cylinder) cross-section A_p */
    double zieb_volume;     /* cylinder volume V_0 */
    double zieb_vp;         /* piston velocity v_p (H_p advances by v_p per step) */
    int mea;                /* 0: momentum exchange of Eqs. 25, 26; 1: its Galilean-invariant form */
    int channel;            /* 1: open channel in x (differentiation form): inlet plane x = 0, outlet x = nx-1 */
    double u_peak;          /* channel inlet peak velocity */
    int plate_lo[3];        /* channel plate node box, inclusive (no plate when lo[0] > hi[0]) */
    int plate_hi[3];
} orc_params;

#define CT_MAX 64
struct orc_contact {
    int id;
    double d[3];
};

typedef struct {
    orc_params p;
    long N;                 /* nx*ny*nz */
    double w[NQ];
    int opp[NQ];
    double *f;              /* [NQ][N] populations at time n (pre-collision) */
    double *fc;             /* [NQ][N] post-collision populations */
    double *fn;             /* [NQ][N] populations at time n+1 */
    int *owner;             /* sphere owning each node at time n, -1 = fluid */
    int *owner_prev;        /* the same at time n-1 */
    float *key;             /* scratch for the overlap tie-break */
    int np;
    double *X, *V, *Om, *R; /* sphere centre, velocity, angular velocity, radius */
    double *Fh, *Th;        /* hydrodynamic force and torque of the last step */
    double *Fc;             /* contact force at the current position (carried) */
    double *Tc;             /* contact (friction) torque at the current position (carried) */
    struct orc_contact *ct; /* [np][CT_MAX] open sphere contacts of a: partner and delta_t seen from a */
    int *ct_n;              /* [np] number of open contacts */
    int ct_overflow;        /* a sphere had more than CT_MAX contacts (its extra ones lose their state) */
    double *dt_wall;        /* [np][2][3] delta_t against the lower and the upper wall */
    double *Fx, *Tx;        /* external force and torque held over every step */
    double *Fcorr, *Tcorr;  /* momentum of the nodes covered / uncovered this step (correction) */
    unsigned char *fixed;   /* 1: prescribed motion, X += V dt; V, Om constant */
    long step;
    long refilled;          /* nodes refilled in the last step */
    double zrho, zH, zvf;   /* ZIEB: cylinder density rho^n, piston displacement H_p^n, mean inflow v_f^n */
    double plate_drag;      /* channel: x momentum the plate took in the last step (Eq. 25 over its links) */
    int channel_violation;  /* channel: a sphere covered a node of the planes x <= 1 or x >= nx-2 */
} orc_state;

/* ------------------------------------------------------------------ */
/* Geometry                                                            */
/* ------------------------------------------------------------------ */

/* Image of lattice coordinate x (0..n-1) closest to centre coordinate Xc on
 * a periodic axis: b + d with b = floor(Xc) and d the wrapped offset in
 * [-n/2, n/2).  On a wall axis the coordinate itself. */
static int image(int x, double Xc, int n, int periodic) {
    if (!periodic) return x;
    int b = (int)floor(Xc);
    int d = (x - b) % n;
    if (d < 0) d += n;
    if (2 * d >= n) d -= n;
    return b + d;
}

/* FP32 relative coordinate of an (unwrapped) lattice coordinate xi to the
 * centre coordinate Xc: (float)(xi - b) - (float)(Xc - b) with b = floor(Xc).
 * (Xc - b is exact in FP64; it is rounded to FP32 once per sphere.) */
static float rel32(int xi, double Xc) {
    double b = floor(Xc);
    return (float)(xi - (int)b) - (float)(Xc - b);
}

/* Squared FP32 distance, summed x, y, z in that order. */
static float dist2_32(float dx, float dy, float dz) { return dx * dx + dy * dy + dz * dz; }

static int wrap(int x, int n) {
    int r = x % n;
    return r < 0 ? r + n : r;
}

/* Channel option (the differentiation form, Sect. 2.3 applied to an open
 * channel): x is not periodic; the planes x = 0 (velocity inlet) and
 * x = nx - 1 (pressure outlet) are not collided and take an equilibrium
 * after streaming; a plate (node box) is a static solid with halfway
 * bounce-back at rest.  Plate nodes carry the owner index np (one past the
 * spheres), so that every test "owner >= 0" treats them as solid; the
 * sphere-specific steps skip that index. */
static int x_periodic(const orc_state *s) { return !s->p.channel; }

static int is_plate_owner(const orc_state *s, int p) { return s->p.channel && p == s->np; }

static int in_plate(const orc_params *P, int x, int y, int z) {
    return P->channel && x >= P->plate_lo[0] && x <= P->plate_hi[0] && y >= P->plate_lo[1] &&
           y <= P->plate_hi[1] && z >= P->plate_lo[2] && z <= P->plate_hi[2];
}

/* Inlet or outlet node of the channel (never collided). */
static int open_plane(const orc_state *s, int x) { return s->p.channel && (x == 0 || x == s->p.nx - 1); }

/* Step 1.  A node is inside sphere p when |x - X_p|^2 < R_p^2 (strict).
 * reading: a node inside several overlapping spheres belongs to the one with
 * the smallest |x - X_p| - R_p, ties to the smallest p. */
static void geometry(orc_state *s) {
    const orc_params *P = &s->p;
    for (long n = 0; n < s->N; ++n) {
        s->owner[n] = -1;
        s->key[n] = INFINITY;
    }
    if (P->channel)
        for (int z = 0; z < P->nz; ++z)
            for (int y = 0; y < P->ny; ++y)
                for (int x = 0; x < P->nx; ++x)
                    if (in_plate(P, x, y, z)) {
                        long n = x + (long)P->nx * (y + (long)P->ny * z);
                        s->owner[n] = s->np; /* static: no sphere takes a plate node */
                        s->key[n] = -INFINITY;
                    }
    for (int p = 0; p < s->np; ++p) {
        const double *X = s->X + 3 * p;
        float Rf = (float)s->R[p];
        float R2 = Rf * Rf;
        int ext = (int)ceil(s->R[p]) + 1;
        int bx = (int)floor(X[0]), by = (int)floor(X[1]), bz = (int)floor(X[2]);
        for (int oz = -ext; oz <= ext; ++oz) {
            int zi = bz + oz;
            if (!P->periodic_z && (zi < 0 || zi >= P->nz)) continue;
            for (int oy = -ext; oy <= ext; ++oy) {
                int yi = by + oy;
                for (int ox = -ext; ox <= ext; ++ox) {
                    int xi = bx + ox;
                    float dx = rel32(xi, X[0]), dy = rel32(yi, X[1]), dz = rel32(zi, X[2]);
                    float d2 = dist2_32(dx, dy, dz);
                    if (!(d2 < R2)) continue;
                    if (P->channel && (xi <= 1 || xi >= P->nx - 2)) {
                        /* the open planes and the planes they read stay fluid */
                        s->channel_violation = 1;
                        continue;
                    }
                    float key = sqrtf(d2) - Rf;
                    long n = wrap(xi, P->nx) + (long)P->nx * (wrap(yi, P->ny) + (long)P->ny * wrap(zi, P->nz));
                    if (key < s->key[n]) {
                        s->key[n] = key;
                        s->owner[n] = p;
                    }
                }
            }
        }
    }
}

/* Link fraction q of the cut link from fluid node x (unwrapped image xi, yi,
 * zi relative to sphere p) along direction j: the smallest root t of
 * |x + t c_j - X_p| = R_p, i.e. q = |x_b - x_f| / |c_j| (Sect. 2.3).
 * Written in the cancellation-free form q = c0 / (-b + sqrt(b^2 - a c0)) of
 * t^2 a + 2 t b + c0 = 0 with a = |c_j|^2, b = c_j.(x - X), c0 = |x-X|^2 - R^2.
 * FP32, like the inside test, so that q < 1/2 is decided identically on both
 * sides. */
static float link_q(const orc_state *s, int p, int xi, int yi, int zi, int j) {
    const double *X = s->X + 3 * p;
    float Rf = (float)s->R[p];
    float dx = rel32(xi, X[0]), dy = rel32(yi, X[1]), dz = rel32(zi, X[2]);
    float cx = (float)CX[j], cy = (float)CY[j], cz = (float)CZ[j];
    float a = cx * cx + cy * cy + cz * cz;
    float b = cx * dx + cy * dy + cz * dz;
    float c0 = dist2_32(dx, dy, dz) - Rf * Rf;
    float disc = b * b - a * c0;
    if (disc < 0.0f) disc = 0.0f;
    float q = c0 / (-b + sqrtf(disc));
    if (q < 0.0f) q = 0.0f;
    if (q > 1.0f) q = 1.0f;
    return q;
}

/* ------------------------------------------------------------------ */
/* Lattice Boltzmann                                                   */
/* ------------------------------------------------------------------ */

/* Eq. (9) with c_s^2 = 1/3: f_i^eq = rho w_i [1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2]. */
static double feq(const orc_state *s, int i, double rho, const double u[3]) {
    double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return rho * s->w[i] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

/* Density (Eq. 5) and velocity (Eq. 6) of node n; with a body force the
 * velocity is shifted by half the force, u = (sum f c + F/2)/rho, F = rho g. */
static void moments(const orc_state *s, const double *f, long n, double *rho, double u[3]) {
    double r = 0, mx = 0, my = 0, mz = 0;
    for (int i = 0; i < NQ; ++i) {
        double fi = f[(long)i * s->N + n];
        r += fi;
        mx += fi * CX[i];
        my += fi * CY[i];
        mz += fi * CZ[i];
    }
    *rho = r;
    u[0] = mx / r + 0.5 * s->p.g[0];
    u[1] = my / r + 0.5 * s->p.g[1];
    u[2] = mz / r + 0.5 * s->p.g[2];
}

/* Effective relaxation time tau* = tau0 + tau_t at node n (Sect. 2.2).
 * Pi_ab = sum_i c_ia c_ib (f_i - f_i^eq); Q = sqrt(Pi_ab Pi_ab).
 * reading: Eq. (18) is used with its Pi read as Q.  This is the root of
 * tau_t (tau0 + tau_t) = sqrt(2) C^2 Q / (2 rho c_s^4), which follows from
 * eta_t = (C l_x)^2 |S|, |S| = sqrt(2 S_ab S_ab) and S = Pi/(2 rho c_s^2 tau*);
 * with c_s^4 = 1/9 and l_x = dt = 1:
 *   tau_t = 1/2 [ sqrt(tau0^2 + 18 sqrt(2) C^2 Q / rho) - tau0 ]. */
static double tau_eff(const orc_state *s, const double *f, long n, double rho, const double u[3]) {
    double tau0 = s->p.tau0;
    if (!s->p.les) return tau0;
    double Pxx = 0, Pyy = 0, Pzz = 0, Pxy = 0, Pxz = 0, Pyz = 0;
    for (int i = 0; i < NQ; ++i) {
        double ne = f[(long)i * s->N + n] - feq(s, i, rho, u);
        Pxx += CX[i] * CX[i] * ne;
        Pyy += CY[i] * CY[i] * ne;
        Pzz += CZ[i] * CZ[i] * ne;
        Pxy += CX[i] * CY[i] * ne;
        Pxz += CX[i] * CZ[i] * ne;
        Pyz += CY[i] * CZ[i] * ne;
    }
    double Q = sqrt(Pxx * Pxx + Pyy * Pyy + Pzz * Pzz + 2.0 * (Pxy * Pxy + Pxz * Pxz + Pyz * Pyz));
    double C = s->p.cs;
    double tau_t = 0.5 * (sqrt(tau0 * tau0 + 18.0 * sqrt(2.0) * C * C * Q / rho) - tau0);
    return tau0 + tau_t;
}

/* Step 3 at one fluid node: BGK relaxation towards Eq. (9) with tau*
 * (Eq. 12), plus the body-force source of Guo et al. (2002),
 *   S_i = (1 - 1/(2 tau*)) w_i [3 (c_i - u).F + 9 (c_i.u)(c_i.F)],  F = rho g. */
static void collide_node(orc_state *s, long n) {
    double rho, u[3];
    moments(s, s->f, n, &rho, u);
    double tau = tau_eff(s, s->f, n, rho, u);
    double F[3] = {rho * s->p.g[0], rho * s->p.g[1], rho * s->p.g[2]};
    for (int i = 0; i < NQ; ++i) {
        double fi = s->f[(long)i * s->N + n];
        double e = feq(s, i, rho, u);
        double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
        double cF = CX[i] * F[0] + CY[i] * F[1] + CZ[i] * F[2];
        double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
        double src = s->w[i] * (3.0 * (cF - uF) + 9.0 * cu * cF);
        s->fc[(long)i * s->N + n] = fi - (fi - e) / tau + (1.0 - 0.5 / tau) * src;
    }
}

/* Is z a lattice plane (always on a periodic z axis)? */
static int in_z(const orc_state *s, int z) { return s->p.periodic_z || (z >= 0 && z < s->p.nz); }

static long node_of(const orc_state *s, int x, int y, int z) {
    return wrap(x, s->p.nx) + (long)s->p.nx * (wrap(y, s->p.ny) + (long)s->p.ny * wrap(z, s->p.nz));
}

static int is_fluid(const orc_state *s, int x, int y, int z) {
    if (!in_z(s, z)) return 0;
    if (s->p.channel && (x < 0 || x >= s->p.nx)) return 0;
    return s->owner[node_of(s, x, y, z)] < 0;
}

/* Boundary point x_b = x + q c_j relative to the centre of sphere p, with x
 * taken at its image nearest to the centre. */
static void arm(const orc_state *s, int p, int x, int y, int z, int j, double q, double l[3]) {
    const double *X = s->X + 3 * p;
    int xi = image(x, X[0], s->p.nx, x_periodic(s)), yi = image(y, X[1], s->p.ny, 1);
    int zi = image(z, X[2], s->p.nz, s->p.periodic_z);
    l[0] = ((double)xi - X[0]) + q * CX[j];
    l[1] = ((double)yi - X[1]) + q * CY[j];
    l[2] = ((double)zi - X[2]) + q * CZ[j];
}

/* Describe the boundary met by the link from fluid node (x,y,z) along c_j:
 * fraction q and boundary velocity u_b.  Returns the owning sphere, -1 for a
 * z wall (q = 1/2, u_b = wall velocity; the halfway wall of Eq. 19) or the
 * channel's plate (q = 1/2, u_b = 0). */
static int boundary(const orc_state *s, int x, int y, int z, int j, double *q, double ub[3]) {
    int zz = z + CZ[j];
    if (!in_z(s, zz)) {
        const double *uw = zz < 0 ? s->p.u_lo : s->p.u_hi;
        *q = 0.5;
        ub[0] = uw[0];
        ub[1] = uw[1];
        ub[2] = uw[2];
        return -1;
    }
    int p = s->owner[node_of(s, x + CX[j], y + CY[j], zz)];
    if (is_plate_owner(s, p)) { /* the plate: halfway wall at rest */
        *q = 0.5;
        ub[0] = ub[1] = ub[2] = 0.0;
        return -1;
    }
    const double *X = s->X + 3 * p;
    int xi = image(x, X[0], s->p.nx, x_periodic(s)), yi = image(y, X[1], s->p.ny, 1);
    int zi = image(z, X[2], s->p.nz, s->p.periodic_z);
    *q = (double)link_q(s, p, xi, yi, zi, j);
    double l[3];
    arm(s, p, x, y, z, j, *q, l);
    const double *V = s->V + 3 * p, *W = s->Om + 3 * p;
    ub[0] = V[0] + (W[1] * l[2] - W[2] * l[1]);
    ub[1] = V[1] + (W[2] * l[0] - W[0] * l[2]);
    ub[2] = V[2] + (W[0] * l[1] - W[1] * l[0]);
    return p;
}

/* Step 4 for the population k arriving at fluid node (x,y,z) from a solid or
 * wall node along the cut link j = opposite(k) (x + c_j is not fluid).
 * Eq. (19) with the moving-boundary term of Eq. (21):
 *   q <  1/2: f_k = 2q fc_j(x) + (1-2q) fc_j(x - c_j) + 6 w_j (c_k.u_b)
 *   q >= 1/2: f_k = fc_j(x)/(2q) + (2q-1)/(2q) fc_k(x) + (3/q) w_j (c_k.u_b)
 * reading: the sign of Eq. (21) is the one that makes a wall moving towards
 * the fluid add momentum; the density factor is the reference density 1.
 * reading: when q < 1/2 and x - c_j is not fluid, the halfway rule
 * f_k = fc_j(x) + 6 w_j (c_k.u_b) is used. */
static double bounce(const orc_state *s, long n, int x, int y, int z, int k, double q, const double ub[3]) {
    int j = s->opp[k];
    double cku = CX[k] * ub[0] + CY[k] * ub[1] + CZ[k] * ub[2];
    double fcj = s->fc[(long)j * s->N + n];
    if (q < 0.5) {
        double dw = 6.0 * s->w[j] * cku;
        if (is_fluid(s, x - CX[j], y - CY[j], z - CZ[j])) {
            long nb = node_of(s, x - CX[j], y - CY[j], z - CZ[j]);
            return 2.0 * q * fcj + (1.0 - 2.0 * q) * s->fc[(long)j * s->N + nb] + dw;
        }
        return fcj + dw;
    }
    double fck = s->fc[(long)k * s->N + n];
    return fcj / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * fck + 3.0 / q * s->w[j] * cku;
}

/* Step 4: f_k(x, n+1) = fc_k(x - c_k) when x - c_k is fluid (Eq. 13), else
 * the bounce-back value above. */
static void stream(orc_state *s) {
    const orc_params *P = &s->p;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < P->nz; ++z) {
        for (int y = 0; y < P->ny; ++y) {
            for (int x = 0; x < P->nx; ++x) {
                long n = node_of(s, x, y, z);
                if (s->owner[n] >= 0 || open_plane(s, x)) continue;
                for (int k = 0; k < NQ; ++k) {
                    int j = s->opp[k];
                    double v;
                    if (is_fluid(s, x - CX[k], y - CY[k], z - CZ[k])) {
                        v = s->fc[(long)k * s->N + node_of(s, x - CX[k], y - CY[k], z - CZ[k])];
                    } else {
                        double q, ub[3];
                        boundary(s, x, y, z, j, &q, ub);
                        v = bounce(s, n, x, y, z, k, q, ub);
                    }
                    s->fn[(long)k * s->N + n] = v;
                }
            }
        }
    }
}

/* Channel option, after streaming: the inlet node (0, y, z) takes
 * f^eq(rho(1, y, z), u_in(z)) with u_in = u_peak 4 zh (1 - zh) x^,
 * zh = (z + 1/2)/nz, and the outlet node (nx-1, y, z) takes f^eq(1,
 * u(nx-2, y, z)), both moments (Eqs. 5, 6, with the force shift) of the
 * populations just streamed into the neighbouring plane (the readings of
 * the differentiation form's boundaries). */
static void channel_planes(orc_state *s) {
    const orc_params *P = &s->p;
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y) {
            double zh = (z + 0.5) / P->nz;
            double u_in[3] = {P->u_peak * 4.0 * zh * (1.0 - zh), 0.0, 0.0};
            double rho1, u1[3], rho2, u2[3];
            moments(s, s->fn, node_of(s, 1, y, z), &rho1, u1);
            moments(s, s->fn, node_of(s, P->nx - 2, y, z), &rho2, u2);
            long n0 = node_of(s, 0, y, z), n1 = node_of(s, P->nx - 1, y, z);
            for (int i = 0; i < NQ; ++i) {
                s->fn[(long)i * s->N + n0] = feq(s, i, rho1, u_in);
                s->fn[(long)i * s->N + n1] = feq(s, i, 1.0, u2);
            }
        }
}

/* Step 5: momentum exchange (Eqs. 25, 26).  Every cut link from fluid node x
 * along j into sphere p carries fc_j(x) c_j into the solid and takes back
 * f_k(x, n+1) c_k, k = opposite(j); the solid receives
 *   dP = (fc_j(x) + f_k(x, n+1)) c_j,    F_p += dP,   T_p += l x dP,
 * l = x_b - X_p, x_b = x + q c_j (reading of "l" as the arm to the boundary
 * point of the link).  Summed in (node index, j) order.  Channel option:
 * the plate's links give its drag, the x component of the same sum. */
static void momentum_exchange(orc_state *s) {
    const orc_params *P = &s->p;
    memset(s->Fh, 0, sizeof(double) * 3 * s->np);
    memset(s->Th, 0, sizeof(double) * 3 * s->np);
    s->plate_drag = 0.0;
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long n = node_of(s, x, y, z);
                if (s->owner[n] >= 0) continue;
                for (int j = 1; j < NQ; ++j) {
                    int zz = z + CZ[j];
                    if (!in_z(s, zz)) continue;
                    if (P->channel && (x + CX[j] < 0 || x + CX[j] >= P->nx)) continue;
                    int p = s->owner[node_of(s, x + CX[j], y + CY[j], zz)];
                    if (p < 0) continue;
                    int k = s->opp[j];
                    if (is_plate_owner(s, p)) {
                        s->plate_drag += (s->fc[(long)j * s->N + n] + s->fn[(long)k * s->N + n]) * CX[j];
                        continue;
                    }
                    double q, ub[3], l[3];
                    boundary(s, x, y, z, j, &q, ub);
                    arm(s, p, x, y, z, j, q, l);
                    double m = s->fc[(long)j * s->N + n] + s->fn[(long)k * s->N + n];
                    double dP[3] = {m * CX[j], m * CY[j], m * CZ[j]};
                    if (P->mea) {
                        /* Galilean-invariant form (Wen, Zhang & Fang 2014; not in the paper): the
                         * populations carry c - u_b, so dP = fc_j (c_j - u_b) - f_k (c_k - u_b) */
                        double e = s->fc[(long)j * s->N + n] - s->fn[(long)k * s->N + n];
                        for (int a = 0; a < 3; ++a) dP[a] -= e * ub[a];
                    }
                    double *F = s->Fh + 3 * p, *T = s->Th + 3 * p;
                    F[0] += dP[0];
                    F[1] += dP[1];
                    F[2] += dP[2];
                    T[0] += l[1] * dP[2] - l[2] * dP[1];
                    T[1] += l[2] * dP[0] - l[0] * dP[2];
                    T[2] += l[0] * dP[1] - l[1] * dP[0];
                }
            }
}

/* Momentum correction (optional; the paper uses none), after Aidun, Lu &
 * Ding (1998): the populations of a node that becomes solid are dropped and
 * their momentum sum_i c_i f_i is handed to the sphere that covers it; the
 * equilibrium given to a node that becomes fluid (the refill below) is paid
 * by its previous sphere.  Torques with the arm x - X_p (minimum image).
 * The corrections join the momentum exchange of the same step, so the total
 * momentum of fluid and spheres changes only by the body force, contacts
 * and walls.  This part: the nodes covered at step n. */
static void arm_of(const orc_state *s, int p, int x, int y, int z, double l[3]) {
    const double *X = s->X + 3 * p;
    l[0] = (double)image(x, X[0], s->p.nx, x_periodic(s)) - X[0];
    l[1] = (double)image(y, X[1], s->p.ny, 1) - X[1];
    l[2] = (double)image(z, X[2], s->p.nz, s->p.periodic_z) - X[2];
}

static void add_momentum(orc_state *s, int p, const double l[3], const double m[3], double sign) {
    double *F = s->Fcorr + 3 * p, *T = s->Tcorr + 3 * p;
    for (int a = 0; a < 3; ++a) F[a] += sign * m[a];
    T[0] += sign * (l[1] * m[2] - l[2] * m[1]);
    T[1] += sign * (l[2] * m[0] - l[0] * m[2]);
    T[2] += sign * (l[0] * m[1] - l[1] * m[0]);
}

static void node_momentum(const orc_state *s, long n, double m[3]) {
    m[0] = m[1] = m[2] = 0.0;
    for (int i = 0; i < NQ; ++i) {
        double fi = s->f[(long)i * s->N + n];
        m[0] += CX[i] * fi;
        m[1] += CY[i] * fi;
        m[2] += CZ[i] * fi;
    }
}

static void covered_correction(orc_state *s) {
    const orc_params *P = &s->p;
    memset(s->Fcorr, 0, sizeof(double) * 3 * s->np);
    memset(s->Tcorr, 0, sizeof(double) * 3 * s->np);
    if (!P->momentum_correction) return;
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long n = node_of(s, x, y, z);
                int p = s->owner[n];
                if (p < 0 || s->owner_prev[n] >= 0 || is_plate_owner(s, p)) continue;
                double m[3], l[3];
                node_momentum(s, n, m);
                arm_of(s, p, x, y, z, l);
                add_momentum(s, p, l, m, 1.0);
            }
}

/* Step 2.  reading (the paper does not describe it): a node solid at n-1
 * and fluid at n takes the equilibrium (Eq. 9) at the velocity of the
 * surface of its previous owner, u_s = V_p + Om_p x (x - X_p), and at the
 * mean density of its neighbours x + c_i that are fluid at both n-1 and n
 * (1 if there are none).  State of the owner: the one at time n. */
static void refill(orc_state *s) {
    const orc_params *P = &s->p;
    s->refilled = 0;
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long n = node_of(s, x, y, z);
                int p = s->owner_prev[n];
                if (p < 0 || s->owner[n] >= 0 || is_plate_owner(s, p)) continue;
                double sum = 0.0;
                int cnt = 0;
                for (int i = 1; i < NQ; ++i) {
                    int zz = z + CZ[i];
                    if (!in_z(s, zz)) continue;
                    long m = node_of(s, x + CX[i], y + CY[i], zz);
                    if (s->owner_prev[m] >= 0 || s->owner[m] >= 0) continue;
                    double r = 0.0;
                    for (int k = 0; k < NQ; ++k) r += s->f[(long)k * s->N + m];
                    sum += r;
                    ++cnt;
                }
                double rho = cnt > 0 ? sum / cnt : 1.0;
                const double *X = s->X + 3 * p, *V = s->V + 3 * p, *W = s->Om + 3 * p;
                double l[3] = {(double)image(x, X[0], P->nx, x_periodic(s)) - X[0],
                               (double)image(y, X[1], P->ny, 1) - X[1],
                               (double)image(z, X[2], P->nz, P->periodic_z) - X[2]};
                double us[3] = {V[0] + (W[1] * l[2] - W[2] * l[1]), V[1] + (W[2] * l[0] - W[0] * l[2]),
                                V[2] + (W[0] * l[1] - W[1] * l[0])};
                for (int i = 0; i < NQ; ++i) s->f[(long)i * s->N + n] = feq(s, i, rho, us);
                ++s->refilled;
                if (P->momentum_correction) {
                    double m[3];
                    node_momentum(s, n, m);
                    add_momentum(s, p, l, m, -1.0);
                }
            }
}

/* Zoom-in with Effective Boundaries (Sect. 2.6): the plane z = 0 is the
 * first simulated plane x_S next to a virtual cylinder of volume V_0 and
 * cross-section A_p below it, whose piston has moved by H_p^n.  After the
 * streaming of step n (and the momentum exchange):
 *   rho^{n+1} = rho^n exp[(v_p A_p - v_f^n A_p) / (V_0 - A_p H_p^n)]   (Eq. 8)
 * with rho^n the cylinder density and v_f^n the mean inflow velocity over
 * the face at time n; then at every fluid node of the face the five
 * populations that would enter from the cylinder (c_z = +1) are unknown:
 * rho* is the sum of the 14 streamed populations and of the five
 * unknown ones at their post-collision values of time n at the node
 * (reading of "f^n": what the node holds for them after its collision, as
 * nothing streamed in); the one normal to the face takes
 *   f_12 = rho^{n+1} - (rho* - f_12)                                    (Eq. 9)
 * so that the density is rho^{n+1}; u = sum_i f_i c_i / rho^{n+1}; and all 19
 * populations are replaced by f^eq(rho^{n+1}, u) (Eq. 9 of the LBM section).
 * readings: v_f^n is the mean of u_z over the fluid nodes of the face as
 * the previous update left them (0 at the start, fluid at rest), rho^0 = 1,
 * H_p^0 = 0, H_p advances by v_p per step; u carries no force shift; the
 * face replaces the wall z = -1/2 for the fluid only (spheres keep their
 * contact with that plane). */
static void zieb(orc_state *s) {
    const orc_params *P = &s->p;
    const double A = P->zieb_area;
    const double rho1 = s->zrho * exp((P->zieb_vp * A - s->zvf * A) / (P->zieb_volume - A * s->zH));
    double sum_uz = 0.0;
    long count = 0;
    for (int y = 0; y < P->ny; ++y)
        for (int x = 0; x < P->nx; ++x) {
            long n = node_of(s, x, y, 0);
            if (s->owner[n] >= 0) continue;
            double f[NQ], rstar = 0.0;
            for (int i = 0; i < NQ; ++i) {
                f[i] = CZ[i] == 1 ? s->fc[(long)i * s->N + n] : s->fn[(long)i * s->N + n];
                rstar += f[i];
            }
            f[12] = rho1 - (rstar - f[12]);
            double u[3] = {0.0, 0.0, 0.0};
            for (int i = 0; i < NQ; ++i) {
                u[0] += CX[i] * f[i];
                u[1] += CY[i] * f[i];
                u[2] += CZ[i] * f[i];
            }
            for (int a = 0; a < 3; ++a) u[a] /= rho1;
            for (int i = 0; i < NQ; ++i) s->fn[(long)i * s->N + n] = feq(s, i, rho1, u);
            sum_uz += u[2];
            ++count;
        }
    s->zrho = rho1;
    s->zH += P->zieb_vp;
    s->zvf = count ? sum_uz / count : 0.0;
}

/* ------------------------------------------------------------------ */
/* DEM                                                                 */
/* ------------------------------------------------------------------ */

static double sphere_mass(const orc_state *s, int a) {
    double r = s->R[a];
    return s->p.rho_s * (4.0 / 3.0) * M_PI * r * r * r;
}

/* Damping coefficient of Eq. (1).  reading: the paper says only that it
 * depends on the restitution e; the linear spring-dashpot result
 * gamma_n = -2 ln(e) sqrt(m_eff k_n) / sqrt(pi^2 + ln(e)^2) gives a normal
 * restitution of exactly e for an isolated binary collision. */
static double gamma_n(const orc_state *s, double meff) {
    double le = log(s->p.restitution);
    return -2.0 * le * sqrt(meff * s->p.kn) / sqrt(M_PI * M_PI + le * le);
}

static int friction_on(const orc_state *s) { return s->p.kt > 0.0 && s->p.mu > 0.0; }

/* Damping coefficient of the tangential law (Eq. 2).  reading: the paper says
 * only that it depends on the tangential restitution; the same
 * spring-dashpot relation as gamma_n with k_t in place of k_n (and the same
 * m_eff), 0 for restitution_t >= 1. */
static double gamma_t(const orc_state *s, double meff) {
    if (!(s->p.restitution_t < 1.0)) return 0.0;
    double le = log(s->p.restitution_t);
    return -2.0 * le * sqrt(meff * s->p.kt) / sqrt(M_PI * M_PI + le * le);
}

static void cross(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Tangential force of one contact (Eqs. 2, 3).  readings: the force on the
 * sphere opposes its tangential displacement and its tangential relative
 * velocity, f_t = -k_t delta_t - gamma_t v_t (the paper's sliding branch,
 * -mu f^n v_t/|v_t|, fixes this sign convention); delta_t is first turned
 * into the current tangent plane (its normal part removed), then advanced by
 * v_t h; when |f_t| exceeds mu max(f^n, 0) the contact slides,
 * f_t = -mu f^n v_t/|v_t| (along the trial force if v_t = 0), and delta_t is
 * reset to -f_t / k_t.  h = 0 evaluates the force without advancing or
 * storing delta_t. */
static void tangential(const orc_state *s, double *state, const double n[3], const double vt[3], double fn,
                       double gt, double h, double ft[3]) {
    double d[3] = {state[0], state[1], state[2]};
    double dn = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
    for (int c = 0; c < 3; ++c) d[c] -= dn * n[c];
    if (h > 0.0)
        for (int c = 0; c < 3; ++c) d[c] += vt[c] * h;
    double tr[3], t2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        tr[c] = -s->p.kt * d[c] - gt * vt[c];
        t2 += tr[c] * tr[c];
    }
    double cap = s->p.mu * (fn > 0.0 ? fn : 0.0);
    if (t2 > cap * cap) {
        double v = sqrt(vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]);
        double tl = sqrt(t2);
        for (int c = 0; c < 3; ++c) ft[c] = v > 0.0 ? -cap * vt[c] / v : cap * tr[c] / tl;
        for (int c = 0; c < 3; ++c) d[c] = -ft[c] / s->p.kt;
    } else {
        for (int c = 0; c < 3; ++c) ft[c] = tr[c];
    }
    if (h > 0.0)
        for (int c = 0; c < 3; ++c) state[c] = d[c];
}

/* Contact force (and, with friction, torque) on every sphere at positions X,
 * velocities v and spins Om (Eq. 1, reading: f^n = k_n delta - gamma_n v_n
 * with delta > 0 the overlap, unclipped).  Sphere-sphere with the minimum
 * image in x and y; sphere-wall against the planes z = -1/2 and z = nz - 1/2
 * with m_eff = m.  A fixed sphere acts with infinite mass.  With friction
 * (Eqs. 2, 3): reading, the contact point is the middle of the overlap, at
 * R - delta/2 from each centre along the line of centres; the relative
 * velocity there is v^r = v_a - v_b - ((R_a - delta/2) Om_a + (R_b -
 * delta/2) Om_b) x n (n from b to a; a wall moves with its lattice velocity
 * and does not spin), and the torque on a is (-(R_a - delta/2) n) x f_t, so
 * that a pair conserves linear and angular momentum exactly.  The
 * tangential displacement of a contact that opened is reset to 0.  h > 0
 * advances the tangential displacements by one sub-step of length h. */
static void contact_forces(orc_state *s, const double *X, const double *v, const double *Om, double *Fc, double *Tc,
                           double h) {
    const orc_params *P = &s->p;
    const int fric = friction_on(s);
#pragma omp parallel for schedule(static)
    for (int a = 0; a < s->np; ++a) {
        double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
        double ma = sphere_mass(s, a);
        struct orc_contact next[CT_MAX]; /* the contacts of a still open after this evaluation */
        int nnext = 0;
        for (int b = 0; b < s->np; ++b) {
            if (b == a) continue;
            double stv[3] = {0.0, 0.0, 0.0}, *st = stv;
            double d[3] = {X[3 * a] - X[3 * b], X[3 * a + 1] - X[3 * b + 1], X[3 * a + 2] - X[3 * b + 2]};
            if (!P->channel && d[0] > 0.5 * P->nx) d[0] -= P->nx;
            if (!P->channel && d[0] < -0.5 * P->nx) d[0] += P->nx;
            if (d[1] > 0.5 * P->ny) d[1] -= P->ny;
            if (d[1] < -0.5 * P->ny) d[1] += P->ny;
            if (P->periodic_z && d[2] > 0.5 * P->nz) d[2] -= P->nz;
            if (P->periodic_z && d[2] < -0.5 * P->nz) d[2] += P->nz;
            double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double delta = s->R[a] + s->R[b] - dist;
            if (!(delta > 0.0) || dist == 0.0) continue; /* an opened contact is not carried over */
            double nv[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
            double vn = (v[3 * a] - v[3 * b]) * nv[0] + (v[3 * a + 1] - v[3 * b + 1]) * nv[1] +
                        (v[3 * a + 2] - v[3 * b + 2]) * nv[2];
            double mb = sphere_mass(s, b);
            double meff = s->fixed[b] ? ma : (s->fixed[a] ? mb : ma * mb / (ma + mb));
            double fn = P->kn * delta - gamma_n(s, meff) * vn;
            F[0] += fn * nv[0];
            F[1] += fn * nv[1];
            F[2] += fn * nv[2];
            if (fric) {
                const struct orc_contact *old = s->ct + (long)a * CT_MAX;
                for (int k = 0; k < s->ct_n[a]; ++k)
                    if (old[k].id == b) {
                        for (int c = 0; c < 3; ++c) stv[c] = old[k].d[c];
                        break;
                    }
                double la = s->R[a] - 0.5 * delta, lb = s->R[b] - 0.5 * delta;
                double S[3], Sn[3], vt[3], ft[3], r[3], tq[3];
                for (int c = 0; c < 3; ++c) S[c] = la * Om[3 * a + c] + lb * Om[3 * b + c];
                cross(S, nv, Sn);
                double vr[3], vrn = 0.0;
                for (int c = 0; c < 3; ++c) {
                    vr[c] = v[3 * a + c] - v[3 * b + c] - Sn[c];
                    vrn += vr[c] * nv[c];
                }
                for (int c = 0; c < 3; ++c) vt[c] = vr[c] - vrn * nv[c];
                tangential(s, st, nv, vt, fn, gamma_t(s, meff), h, ft);
                for (int c = 0; c < 3; ++c) {
                    F[c] += ft[c];
                    r[c] = -la * nv[c];
                }
                cross(r, ft, tq);
                for (int c = 0; c < 3; ++c) T[c] += tq[c];
                if (h > 0.0) {
                    if (nnext < CT_MAX) {
                        next[nnext].id = b;
                        for (int c = 0; c < 3; ++c) next[nnext].d[c] = stv[c];
                        ++nnext;
                    } else {
                        s->ct_overflow = 1;
                    }
                }
            }
        }
        if (fric && h > 0.0) {
            memcpy(s->ct + (long)a * CT_MAX, next, sizeof(struct orc_contact) * (size_t)nnext);
            s->ct_n[a] = nnext;
        }
        for (int side = 0; side < 2 && !P->periodic_z; ++side) {
            /* side 0: wall z = -1/2, normal +z into the sphere; side 1: z = nz - 1/2, normal -z */
            double pen = side == 0 ? s->R[a] - (X[3 * a + 2] + 0.5) : s->R[a] - ((P->nz - 0.5) - X[3 * a + 2]);
            double *st = fric ? s->dt_wall + 3 * (2L * a + side) : NULL;
            if (!(pen > 0.0)) {
                if (fric && h > 0.0) st[0] = st[1] = st[2] = 0.0;
                continue;
            }
            if (side == 0) F[2] += P->kn * pen - gamma_n(s, ma) * v[3 * a + 2];
            else F[2] -= P->kn * pen - gamma_n(s, ma) * (-v[3 * a + 2]);
            if (fric) {
                double nv[3] = {0.0, 0.0, side == 0 ? 1.0 : -1.0};
                const double *uw = side == 0 ? P->u_lo : P->u_hi;
                double fn = P->kn * pen - gamma_n(s, ma) * (v[3 * a + 2] * nv[2]);
                double la = s->R[a] - 0.5 * pen;
                double S[3], Sn[3], vt[3], ft[3], r[3], tq[3], vr[3], vrn = 0.0;
                for (int c = 0; c < 3; ++c) S[c] = la * Om[3 * a + c];
                cross(S, nv, Sn);
                for (int c = 0; c < 3; ++c) {
                    vr[c] = v[3 * a + c] - uw[c] - Sn[c];
                    vrn += vr[c] * nv[c];
                }
                for (int c = 0; c < 3; ++c) vt[c] = vr[c] - vrn * nv[c];
                tangential(s, st, nv, vt, fn, gamma_t(s, ma), h, ft);
                for (int c = 0; c < 3; ++c) {
                    F[c] += ft[c];
                    r[c] = -la * nv[c];
                }
                cross(r, ft, tq);
                for (int c = 0; c < 3; ++c) T[c] += tq[c];
            }
        }
        if (P->channel && P->plate_lo[0] <= P->plate_hi[0]) {
            /* channel plate: normal contact (Eq. 1, m_eff = m) with its surface,
             * the node box grown by 1/2 (its halfway bounce-back planes), at
             * the closest point of that box to the centre (y minimum image) */
            double d[3], dist2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                double xc = X[3 * a + c];
                if (c == 1) {
                    double mid = 0.5 * (P->plate_lo[1] + P->plate_hi[1]);
                    if (xc - mid > 0.5 * P->ny) xc -= P->ny;
                    if (xc - mid < -0.5 * P->ny) xc += P->ny;
                }
                double lo = P->plate_lo[c] - 0.5, hi = P->plate_hi[c] + 0.5;
                double pc = xc < lo ? lo : (xc > hi ? hi : xc);
                d[c] = xc - pc;
                dist2 += d[c] * d[c];
            }
            double dist = sqrt(dist2), pen = s->R[a] - dist;
            if (pen > 0.0 && dist > 0.0) {
                double nv[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
                double vn = v[3 * a] * nv[0] + v[3 * a + 1] * nv[1] + v[3 * a + 2] * nv[2];
                double fn = P->kn * pen - gamma_n(s, ma) * vn;
                for (int c = 0; c < 3; ++c) F[c] += fn * nv[c];
            }
        }
        for (int c = 0; c < 3; ++c) {
            Fc[3 * a + c] = F[c];
            Tc[3 * a + c] = T[c];
        }
    }
}

/* Step 6: velocity Verlet (Sect. 2.1) with sub-step h = 1/dem_substeps, the
 * hydrodynamic load F_h, T_h and an external load F_x, T_x held over the
 * lattice step, and no body force on spheres:
 *   v += (F_h + F_x + F_c) h/(2m);  X += v h;  F_c = contact(X, v);
 *   v += (F_h + F_x + F_c) h/(2m);  Om += (T_h + T_x) h / I,  I = 2/5 m R^2.
 * With friction the spin takes the same two half kicks as v, with the
 * contact torque T_c of the last contact evaluation added:
 *   Om += (T_h + T_x + T_c) h/(2I) before the drift and after the contacts.
 * A fixed sphere moves with its prescribed velocity: X += V h only.  Centres
 * are wrapped into [0, n) on periodic axes after every drift. */
static void dem(orc_state *s) {
    const orc_params *P = &s->p;
    const int fric = friction_on(s);
    int ns = P->dem_substeps > 0 ? P->dem_substeps : 1;
    double h = 1.0 / ns;
    for (int it = 0; it < ns; ++it) {
        for (int a = 0; a < s->np; ++a) {
            double m = sphere_mass(s, a);
            double I = 0.4 * m * s->R[a] * s->R[a];
            for (int c = 0; c < 3; ++c) {
                if (!s->fixed[a]) {
                    s->V[3 * a + c] += (s->Fh[3 * a + c] + s->Fx[3 * a + c] + s->Fc[3 * a + c]) * h / (2.0 * m);
                    if (fric) s->Om[3 * a + c] += (s->Th[3 * a + c] + s->Tx[3 * a + c] + s->Tc[3 * a + c]) * h / (2.0 * I);
                }
                s->X[3 * a + c] += s->V[3 * a + c] * h;
            }
            if (!P->channel && s->X[3 * a] >= P->nx) s->X[3 * a] -= P->nx;
            if (!P->channel && s->X[3 * a] < 0.0) s->X[3 * a] += P->nx;
            if (s->X[3 * a + 1] >= P->ny) s->X[3 * a + 1] -= P->ny;
            if (s->X[3 * a + 1] < 0.0) s->X[3 * a + 1] += P->ny;
            if (P->periodic_z && s->X[3 * a + 2] >= P->nz) s->X[3 * a + 2] -= P->nz;
            if (P->periodic_z && s->X[3 * a + 2] < 0.0) s->X[3 * a + 2] += P->nz;
        }
        contact_forces(s, s->X, s->V, s->Om, s->Fc, s->Tc, h);
        for (int a = 0; a < s->np; ++a) {
            if (s->fixed[a]) continue;
            double m = sphere_mass(s, a);
            double I = 0.4 * m * s->R[a] * s->R[a];
            for (int c = 0; c < 3; ++c) {
                s->V[3 * a + c] += (s->Fh[3 * a + c] + s->Fx[3 * a + c] + s->Fc[3 * a + c]) * h / (2.0 * m);
                if (fric) s->Om[3 * a + c] += (s->Th[3 * a + c] + s->Tx[3 * a + c] + s->Tc[3 * a + c]) * h / (2.0 * I);
                else s->Om[3 * a + c] += (s->Th[3 * a + c] + s->Tx[3 * a + c]) * h / I;
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Interface (ctypes)                                                  */
/* ------------------------------------------------------------------ */

static void *xcalloc(size_t n, size_t sz) { return n ? calloc(n, sz) : NULL; }

void orc_destroy(orc_state *s);

orc_state *orc_create(const orc_params *p) {
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return NULL;
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    s->p = *p;
    s->N = p->fluid ? (long)p->nx * p->ny * p->nz : 0;
    for (int i = 0; i < NQ; ++i) {
        s->w[i] = weight(i);
        s->opp[i] = opposite(i);
    }
    if (s->N) {
        s->f = (double *)xcalloc((size_t)NQ * s->N, sizeof(double));
        s->fc = (double *)xcalloc((size_t)NQ * s->N, sizeof(double));
        s->fn = (double *)xcalloc((size_t)NQ * s->N, sizeof(double));
        s->owner = (int *)xcalloc((size_t)s->N, sizeof(int));
        s->owner_prev = (int *)xcalloc((size_t)s->N, sizeof(int));
        s->key = (float *)xcalloc((size_t)s->N, sizeof(float));
        if (!s->f || !s->fc || !s->fn || !s->owner || !s->owner_prev || !s->key) {
            orc_destroy(s);
            return NULL;
        }
        for (int i = 0; i < NQ; ++i)
            for (long n = 0; n < s->N; ++n) s->f[(long)i * s->N + n] = s->w[i];
        for (long n = 0; n < s->N; ++n) s->owner[n] = s->owner_prev[n] = -1;
    }
    s->zrho = 1.0;
    return s;
}

void orc_destroy(orc_state *s) {
    if (!s) return;
    free(s->f); free(s->fc); free(s->fn); free(s->owner); free(s->owner_prev); free(s->key);
    free(s->X); free(s->V); free(s->Om); free(s->R); free(s->Fh); free(s->Th); free(s->Fc); free(s->fixed);
    free(s->Fx); free(s->Tx); free(s->Fcorr); free(s->Tcorr); free(s->Tc); free(s->ct); free(s->ct_n); free(s->dt_wall);
    free(s);
}

/* Place n spheres and reset the fluid to rest (f = w, rho = 1, u = 0). */
int orc_set_particles(orc_state *s, int n, const double *X, const double *V, const double *Om,
                      const double *R, const unsigned char *fixed) {
    free(s->X); free(s->V); free(s->Om); free(s->R); free(s->Fh); free(s->Th); free(s->Fc); free(s->fixed);
    free(s->Fx); free(s->Tx); free(s->Fcorr); free(s->Tcorr); free(s->Tc); free(s->ct); free(s->ct_n);
    free(s->dt_wall);
    s->ct = NULL;
    s->ct_n = NULL;
    s->dt_wall = NULL;
    s->ct_overflow = 0;
    s->np = n;
    s->Tc = (double *)xcalloc(3 * (size_t)n, sizeof(double));
    if (friction_on(s)) {
        s->ct = (struct orc_contact *)xcalloc((size_t)n * CT_MAX, sizeof(struct orc_contact));
        s->ct_n = (int *)xcalloc((size_t)n, sizeof(int));
        s->dt_wall = (double *)xcalloc(6 * (size_t)n, sizeof(double));
        if (n && (!s->ct || !s->ct_n || !s->dt_wall)) return -1;
    }
    s->Fcorr = (double *)xcalloc(3 * (size_t)n, sizeof(double));
    s->Tcorr = (double *)xcalloc(3 * (size_t)n, sizeof(double));
    s->Fx = (double *)xcalloc(3 * (size_t)n, sizeof(double));
    s->Tx = (double *)xcalloc(3 * (size_t)n, sizeof(double));
    s->X = (double *)xcalloc(3 * (size_t)n, sizeof(double));
    s->V = (double *)xcalloc(3 * (size_t)n, sizeof(double));
    s->Om = (double *)xcalloc(3 * (size_t)n, sizeof(double));
    s->R = (double *)xcalloc((size_t)n, sizeof(double));
    s->Fh = (double *)xcalloc(3 * (size_t)n, sizeof(double));
    s->Th = (double *)xcalloc(3 * (size_t)n, sizeof(double));
    s->Fc = (double *)xcalloc(3 * (size_t)n, sizeof(double));
    s->fixed = (unsigned char *)xcalloc((size_t)n, 1);
    if (n) {
        memcpy(s->X, X, sizeof(double) * 3 * n);
        memcpy(s->V, V, sizeof(double) * 3 * n);
        memcpy(s->Om, Om, sizeof(double) * 3 * n);
        memcpy(s->R, R, sizeof(double) * n);
        if (fixed) memcpy(s->fixed, fixed, n);
    }
    if (s->N) {
        for (int i = 0; i < NQ; ++i)
            for (long m = 0; m < s->N; ++m) s->f[(long)i * s->N + m] = s->w[i];
        geometry(s);
        memcpy(s->owner_prev, s->owner, sizeof(int) * s->N);
    }
    contact_forces(s, s->X, s->V, s->Om, s->Fc, s->Tc, 0.0);
    s->step = 0;
    s->zrho = 1.0;
    s->zH = 0.0;
    s->zvf = 0.0;
    s->refilled = 0;
    return 0;
}

/* External force and torque per sphere, [n][3] each (NULL = zero). */
void orc_set_load(orc_state *s, const double *F, const double *T) {
    for (int m = 0; m < 3 * s->np; ++m) {
        s->Fx[m] = F ? F[m] : 0.0;
        s->Tx[m] = T ? T[m] : 0.0;
    }
}

/* Pre-collision populations in natural layout [19][N]; solid nodes ignored. */
void orc_set_populations(orc_state *s, const double *f) {
    for (long m = 0; m < (long)NQ * s->N; ++m)
        if (s->owner[m % s->N] < 0) s->f[m] = f[m];
}

void orc_get_populations(const orc_state *s, double *f) {
    for (long m = 0; m < (long)NQ * s->N; ++m) f[m] = s->owner[m % s->N] < 0 ? s->f[m] : 0.0;
}

void orc_step(orc_state *s, int nsteps) {
    for (int it = 0; it < nsteps; ++it) {
        if (s->N) {
            memcpy(s->owner_prev, s->owner, sizeof(int) * s->N);
            geometry(s);
            covered_correction(s);
            refill(s);
#pragma omp parallel for schedule(static)
            for (long n = 0; n < s->N; ++n) {
                if (s->owner[n] >= 0) continue;
                if (open_plane(s, (int)(n % s->p.nx))) /* channel inlet / outlet: not collided */
                    for (int i = 0; i < NQ; ++i) s->fc[(long)i * s->N + n] = s->f[(long)i * s->N + n];
                else
                    collide_node(s, n);
            }
            stream(s);
            if (s->p.channel) channel_planes(s);
            momentum_exchange(s);
            for (long k = 0; k < 3 * (long)s->np; ++k) {
                s->Fh[k] += s->Fcorr[k];
                s->Th[k] += s->Tcorr[k];
            }
            if (s->p.zieb) zieb(s);
            double *t = s->f;
            s->f = s->fn;
            s->fn = t;
        }
        dem(s);
        ++s->step;
    }
}

void orc_forces(const orc_state *s, double *F, double *T) {
    memcpy(F, s->Fh, sizeof(double) * 3 * s->np);
    memcpy(T, s->Th, sizeof(double) * 3 * s->np);
}

void orc_contact_forces(const orc_state *s, double *Fc) { memcpy(Fc, s->Fc, sizeof(double) * 3 * s->np); }

void orc_contact_torques(const orc_state *s, double *Tc) { memcpy(Tc, s->Tc, sizeof(double) * 3 * s->np); }

int orc_contact_overflow(const orc_state *s) { return s->ct_overflow; }

/* ZIEB state: cylinder density, piston displacement, mean inflow velocity. */
void orc_zieb_state(const orc_state *s, double *out) {
    out[0] = s->zrho;
    out[1] = s->zH;
    out[2] = s->zvf;
}

void orc_zieb_set_piston(orc_state *s, double vp) { s->p.zieb_vp = vp; }

void orc_particles(const orc_state *s, double *X, double *V, double *Om) {
    memcpy(X, s->X, sizeof(double) * 3 * s->np);
    memcpy(V, s->V, sizeof(double) * 3 * s->np);
    memcpy(Om, s->Om, sizeof(double) * 3 * s->np);
}

/* Density and velocity (Eqs. 5, 6 with the force shift) of the current
 * pre-collision state; u is [3][N]; solid nodes give rho = 0, u = 0. */
void orc_fields(const orc_state *s, double *rho, double *u) {
    for (long n = 0; n < s->N; ++n) {
        if (s->owner[n] >= 0) {
            rho[n] = 0.0;
            u[n] = u[s->N + n] = u[2 * s->N + n] = 0.0;
            continue;
        }
        double r, v[3];
        moments(s, s->f, n, &r, v);
        rho[n] = r;
        u[n] = v[0];
        u[s->N + n] = v[1];
        u[2 * s->N + n] = v[2];
    }
}

/* tau* of the collision the next step would apply at each fluid node. */
void orc_tau_eff(const orc_state *s, double *tau) {
    for (long n = 0; n < s->N; ++n) {
        if (s->owner[n] >= 0) {
            tau[n] = 0.0;
            continue;
        }
        double r, v[3];
        moments(s, s->f, n, &r, v);
        tau[n] = tau_eff(s, s->f, n, r, v);
    }
}

void orc_owner(const orc_state *s, int *owner) { memcpy(owner, s->owner, sizeof(int) * s->N); }

/* Cut sphere links of the current geometry in (node, j) order; returns the
 * count and fills up to cap entries. */
long orc_links(const orc_state *s, long cap, long *node, int *dir, float *q, int *pid) {
    const orc_params *P = &s->p;
    long cnt = 0;
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long n = node_of(s, x, y, z);
                if (s->owner[n] >= 0) continue;
                for (int j = 1; j < NQ; ++j) {
                    int zz = z + CZ[j];
                    if (!in_z(s, zz)) continue;
                    int p = s->owner[node_of(s, x + CX[j], y + CY[j], zz)];
                    if (p < 0 || is_plate_owner(s, p)) continue;
                    if (cnt < cap) {
                        const double *X = s->X + 3 * p;
                        node[cnt] = n;
                        dir[cnt] = j;
                        q[cnt] = link_q(s, p, image(x, X[0], P->nx, x_periodic(s)), image(y, X[1], P->ny, 1),
                                        image(z, X[2], P->nz, P->periodic_z), j);
                        pid[cnt] = p;
                    }
                    ++cnt;
                }
            }
    return cnt;
}

long orc_refilled(const orc_state *s) { return s->refilled; }

/* Channel option: the plate drag of the last step and the violation flag. */
double orc_plate_drag(const orc_state *s) { return s->plate_drag; }
int orc_channel_violation(const orc_state *s) { return s->channel_violation; }
long orc_step_count(const orc_state *s) { return s->step; }

/* ------------------------------------------------------------------ */
/* Test hooks                                                          */
/* ------------------------------------------------------------------ */

/* The velocity set and weights as the oracle uses them. */
void orc_tables(int *cx, int *cy, int *cz, double *w, int *opp) {
    for (int i = 0; i < NQ; ++i) {
        cx[i] = CX[i];
        cy[i] = CY[i];
        cz[i] = CZ[i];
        w[i] = weight(i);
        opp[i] = opposite(i);
    }
}

/* Eq. (9) for one (rho, u): out[19]. */
void orc_feq(double rho, const double *u, double *out) {
    orc_state tmp;
    for (int i = 0; i < NQ; ++i) tmp.w[i] = weight(i);
    for (int i = 0; i < NQ; ++i) out[i] = feq(&tmp, i, rho, u);
}

/* Steps 1 and 2 of the next time step only (geometry and refill); the
 * following orc_step then finds the geometry unchanged and refills nothing. */
void orc_refill_only(orc_state *s) {
    if (!s->N) return;
    memcpy(s->owner_prev, s->owner, sizeof(int) * s->N);
    geometry(s);
    refill(s);
}
