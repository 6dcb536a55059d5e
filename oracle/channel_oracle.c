/*
 * channel_oracle.c - plain, slow FP64 CPU reference of the differentiation
 * form: a D3Q19 channel with a velocity inlet, a pressure outlet, a fixed
 * plate obstacle and fixed spheres, run for S steps; the objective is the
 * mean plate drag J over steps [avg_from, S], and its tangent-linear
 * derivative along a parameter direction of (inlet peak velocity, body
 * force, Smagorinsky constant).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the scripts that write stored
 * expected values under tests/golden/ and the CPU baseline leg of the
 * benchmark load this file.  It shares no code, header, table or helper with
 * the CUDA library.
 *
 * Every quantity is a dual number (value, derivative along dtheta): the
 * tangent-linear pass is the same arithmetic carried on duals, so the value
 * part is the plain FP64 run and the derivative part is its exact forward
 * derivative.  The derivative of sqrt at 0 is taken as 0 (Q = 0 in Eq. 18).
 *
 * The lattice step (Sects. 2.2, 2.3) on this geometry, step s = 1 .. S:
 *   1. streaming (Eq. 13) of the post-collision populations G^{s-1} into
 *      f^s at every interior fluid node, with bounce-back on cut links: the
 *      z walls (at -1/2, nz - 1/2) and the plate are halfway walls, q = 1/2;
 *      sphere links take Bouzidi's rule (Eq. 19) with q the smallest root of
 *      |x + q c_j - X| = R; everything is at rest (no Eq. 21 term);
 *   2. inlet nodes (x = 0): f^s = f^eq(rho_1, u_in(z)) (Eq. 9), rho_1 the
 *      density of f^s at (1, y, z), u_in = u_peak 4 zh (1 - zh) x^,
 *      zh = (z + 1/2) / nz; outlet nodes (x = nx - 1): f^s = f^eq(1, u_2),
 *      u_2 the velocity (Eq. 6 with the force shift) of f^s at (nx-2, y, z);
 *   3. collision (Eqs. 5, 6, 9, 12, 18 and the Guo source, as in
 *      lbm_oracle.c) at interior fluid nodes; inlet and outlet nodes keep
 *      G^s = f^s;
 *   4. plate drag D^s = sum over links (x, j) with x + c_j in the plate of
 *      (G_j^s(x) + f_k^{s+1}(x)) c_j,x = 2 G_j^s(x) c_j,x (halfway wall at
 *      rest, Eqs. 25 with k = opp(j)).
 * Initially f^0 = w everywhere (rest, rho = 1) and G^0 = collide(f^0).
 * y is periodic; x is periodic instead of open when periodic_x = 1 (then
 * there are no inlet / outlet nodes), which the tests use to compare this
 * file with lbm_oracle.c.
 *
 * Geometry decisions are FP64: a node is inside a sphere when
 * |x - X|^2 < R^2 (y minimum image), in the plate when inside its node box;
 * plate before spheres.  Build with -ffp-contract=off.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NQ 19

/* Table 1: the D3Q19 velocity set. */
static const int CX[NQ] = {0, -1, 0, 0, -1, -1, -1, -1, 0, 0, 1, 0, 0, 1, 1, 1, 1, 0, 0};
static const int CY[NQ] = {0, 0, -1, 0, -1, 1, 0, 0, -1, -1, 0, 1, 0, 1, -1, 0, 0, 1, 1};
static const int CZ[NQ] = {0, 0, 0, -1, 0, 0, -1, 1, -1, 1, 0, 0, 1, 0, 0, 1, -1, 1, -1};

static double weight(int i) {
    if (i == 0) return 1.0 / 3.0;
    if (i == 1 || i == 2 || i == 3 || i == 10 || i == 11 || i == 12) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

static int opposite(int i) {
    for (int k = 0; k < NQ; ++k)
        if (CX[k] == -CX[i] && CY[k] == -CY[i] && CZ[k] == -CZ[i]) return k;
    return -1;
}

/* ---- dual numbers: (value, derivative) ---------------------------------- */

typedef struct {
    double v, d;
} dual;

static dual dc(double v) {
    dual r = {v, 0.0};
    return r;
}
static dual dadd(dual a, dual b) {
    dual r = {a.v + b.v, a.d + b.d};
    return r;
}
static dual dsub(dual a, dual b) {
    dual r = {a.v - b.v, a.d - b.d};
    return r;
}
static dual dmul(dual a, dual b) {
    dual r = {a.v * b.v, a.d * b.v + a.v * b.d};
    return r;
}
static dual dscale(dual a, double c) {
    dual r = {a.v * c, a.d * c};
    return r;
}
static dual ddiv(dual a, dual b) {
    dual r = {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
    return r;
}
static dual dsqrt(dual a) {
    double s = sqrt(a.v);
    dual r = {s, s > 0.0 ? a.d / (2.0 * s) : 0.0};
    return r;
}

/* ---- problem ------------------------------------------------------------ */

typedef struct {
    int nx, ny, nz;
    double tau0;        /* relaxation time (Eq. 15) */
    double cs;          /* Smagorinsky constant C (Eq. 18) */
    double gx;          /* body acceleration along x */
    double u_peak;      /* inlet peak velocity */
    int plate_lo[3];    /* plate node box, inclusive */
    int plate_hi[3];
    int steps;          /* S */
    int avg_from;       /* first step of the drag average */
    int periodic_x;     /* 1: x periodic, no inlet / outlet */
} chan_params;

enum { FLUID = 0, SOLID = 1, INLET = 2, OUTLET = 3, PLATE = 4 };

typedef struct {
    chan_params p;
    long N;
    unsigned char *type; /* per node */
    double *q;           /* [NQ][N]: fraction of the cut link x -> x + c_j, -1 if not cut */
    unsigned char *plate_link; /* [NQ][N]: link x -> x + c_j ends in the plate */
    dual *f, *G;
    dual theta[3];       /* (u_peak, gx, cs) with their tangent directions */
} chan_state;

static int wrap(int x, int n) {
    int r = x % n;
    return r < 0 ? r + n : r;
}

static long node(const chan_state *s, int x, int y, int z) {
    return (long)wrap(x, s->p.nx) + (long)s->p.nx * ((long)wrap(y, s->p.ny) + (long)s->p.ny * z);
}

static int in_plate(const chan_params *p, int x, int y, int z) {
    return x >= p->plate_lo[0] && x <= p->plate_hi[0] && y >= p->plate_lo[1] && y <= p->plate_hi[1] &&
           z >= p->plate_lo[2] && z <= p->plate_hi[2];
}

/* y-minimum-image offset of coordinate y from centre Y (x is not periodic
 * unless periodic_x, z never). */
static double offset(double xi, double Xc, int n, int periodic) {
    double d = xi - Xc;
    if (periodic) {
        if (d > 0.5 * n) d -= n;
        if (d < -0.5 * n) d += n;
    }
    return d;
}

static void build_geometry(chan_state *s, int np, const double *X, const double *R) {
    const chan_params *P = &s->p;
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long n = node(s, x, y, z);
                unsigned char t = FLUID;
                if (!P->periodic_x && x == 0) t = INLET;
                else if (!P->periodic_x && x == P->nx - 1) t = OUTLET;
                else if (in_plate(P, x, y, z)) t = PLATE;
                else
                    for (int a = 0; a < np && t == FLUID; ++a) {
                        double dx = offset(x, X[3 * a], P->nx, P->periodic_x);
                        double dy = offset(y, X[3 * a + 1], P->ny, 1);
                        double dz = z - X[3 * a + 2];
                        if (dx * dx + dy * dy + dz * dz < R[a] * R[a]) t = SOLID;
                    }
                s->type[n] = t;
            }
    /* cut links of fluid nodes (interior, inlet, outlet) */
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long n = node(s, x, y, z);
                if (s->type[n] == SOLID || s->type[n] == PLATE) continue;
                for (int j = 1; j < NQ; ++j) {
                    int xx = x + CX[j], yy = y + CY[j], zz = z + CZ[j];
                    double q = -1.0;
                    int plate = 0;
                    if (zz < 0 || zz >= P->nz) {
                        q = 0.5; /* z wall */
                    } else if (!P->periodic_x && (xx < 0 || xx >= P->nx)) {
                        q = -1.0; /* leaves through the open ends: never read */
                    } else {
                        long m = node(s, xx, yy, zz);
                        if (s->type[m] == PLATE) {
                            q = 0.5;
                            plate = 1;
                        } else if (s->type[m] == SOLID) {
                            /* smallest root t of |x + t c_j - X_a|^2 = R_a^2 over the
                             * spheres containing x + c_j: written as
                             * t = c0 / (-b + sqrt(b^2 - a c0)), a = |c_j|^2,
                             * b = c_j.(x - X), c0 = |x - X|^2 - R^2 */
                            double best = 2.0;
                            for (int a2 = 0; a2 < np; ++a2) {
                                double dx = offset(x, X[3 * a2], P->nx, P->periodic_x);
                                double dy = offset(y, X[3 * a2 + 1], P->ny, 1);
                                double dz = z - X[3 * a2 + 2];
                                double ex = dx + CX[j], ey = dy + CY[j], ez = dz + CZ[j];
                                if (!(ex * ex + ey * ey + ez * ez < R[a2] * R[a2])) continue;
                                double aa = (double)(CX[j] * CX[j] + CY[j] * CY[j] + CZ[j] * CZ[j]);
                                double b = CX[j] * dx + CY[j] * dy + CZ[j] * dz;
                                double c0 = dx * dx + dy * dy + dz * dz - R[a2] * R[a2];
                                double disc = b * b - aa * c0;
                                if (disc < 0.0) disc = 0.0;
                                double t = c0 / (-b + sqrt(disc));
                                if (t < best) best = t;
                            }
                            if (best > 1.0) best = 1.0;
                            if (best < 0.0) best = 0.0;
                            q = best;
                        }
                    }
                    s->q[(long)j * s->N + n] = q;
                    s->plate_link[(long)j * s->N + n] = (unsigned char)plate;
                }
            }
}

/* f^eq_i(rho, u) of Eq. (9) with c_s^2 = 1/3, on duals. */
static dual feq(int i, dual rho, const dual u[3]) {
    dual cu = dadd(dadd(dscale(u[0], CX[i]), dscale(u[1], CY[i])), dscale(u[2], CZ[i]));
    dual uu = dadd(dadd(dmul(u[0], u[0]), dmul(u[1], u[1])), dmul(u[2], u[2]));
    dual br = dadd(dadd(dc(1.0), dscale(cu, 3.0)), dsub(dscale(dmul(cu, cu), 4.5), dscale(uu, 1.5)));
    return dmul(dscale(rho, weight(i)), br);
}

/* Density (Eq. 5) and force-shifted velocity (Eq. 6) of 19 populations. */
static void moments(const chan_state *s, const dual *f, long n, dual *rho, dual u[3]) {
    dual r = dc(0), mx = dc(0), my = dc(0), mz = dc(0);
    for (int i = 0; i < NQ; ++i) {
        dual fi = f[(long)i * s->N + n];
        r = dadd(r, fi);
        mx = dadd(mx, dscale(fi, CX[i]));
        my = dadd(my, dscale(fi, CY[i]));
        mz = dadd(mz, dscale(fi, CZ[i]));
    }
    *rho = r;
    dual hg = dscale(s->theta[1], 0.5);
    u[0] = dadd(ddiv(mx, r), hg);
    u[1] = ddiv(my, r);
    u[2] = ddiv(mz, r);
}

/* Collision at interior fluid node n: BGK towards Eq. (9) with the
 * Smagorinsky tau* of Eq. (18) (Q = sqrt(Pi:Pi), Pi = sum c c (f - f^eq))
 * plus the Guo source (1 - 1/(2 tau*)) w_i [3 (c_i - u).F + 9 (c_i.u)(c_i.F)],
 * F = rho g. */
static void collide(chan_state *s, long n) {
    dual rho, u[3];
    moments(s, s->f, n, &rho, u);
    dual fe[NQ];
    for (int i = 0; i < NQ; ++i) fe[i] = feq(i, rho, u);
    dual P[6] = {dc(0), dc(0), dc(0), dc(0), dc(0), dc(0)};
    for (int i = 0; i < NQ; ++i) {
        dual ne = dsub(s->f[(long)i * s->N + n], fe[i]);
        P[0] = dadd(P[0], dscale(ne, CX[i] * CX[i]));
        P[1] = dadd(P[1], dscale(ne, CY[i] * CY[i]));
        P[2] = dadd(P[2], dscale(ne, CZ[i] * CZ[i]));
        P[3] = dadd(P[3], dscale(ne, CX[i] * CY[i]));
        P[4] = dadd(P[4], dscale(ne, CX[i] * CZ[i]));
        P[5] = dadd(P[5], dscale(ne, CY[i] * CZ[i]));
    }
    dual QQ = dadd(dadd(dmul(P[0], P[0]), dmul(P[1], P[1])), dmul(P[2], P[2]));
    QQ = dadd(QQ, dscale(dadd(dadd(dmul(P[3], P[3]), dmul(P[4], P[4])), dmul(P[5], P[5])), 2.0));
    dual Q = dsqrt(QQ);
    dual C = s->theta[2];
    dual tau0 = dc(s->p.tau0);
    dual K = dscale(dmul(C, C), 18.0 * sqrt(2.0));
    dual tau_t = dscale(dsub(dsqrt(dadd(dmul(tau0, tau0), ddiv(dmul(K, Q), rho))), tau0), 0.5);
    dual tau = dadd(tau0, tau_t);
    dual F0 = dmul(rho, s->theta[1]); /* F = rho g, g along x */
    dual uF = dmul(u[0], F0);
    dual om = ddiv(dc(1.0), tau);
    dual sk = dsub(dc(1.0), dscale(om, 0.5));
    for (int i = 0; i < NQ; ++i) {
        dual fi = s->f[(long)i * s->N + n];
        dual cu = dadd(dadd(dscale(u[0], CX[i]), dscale(u[1], CY[i])), dscale(u[2], CZ[i]));
        dual cF = dscale(F0, CX[i]);
        dual src = dscale(dadd(dscale(dsub(cF, uF), 3.0), dscale(dmul(cu, cF), 9.0)), weight(i));
        s->G[(long)i * s->N + n] = dadd(dsub(fi, dmul(dsub(fi, fe[i]), om)), dmul(sk, src));
    }
}

/* Streaming into interior fluid node (x, y, z) for direction i, from G. */
static dual pull(const chan_state *s, const dual *G, int x, int y, int z, int i, const int *opp) {
    long n = node(s, x, y, z);
    int j = opp[i];
    double q = s->q[(long)j * s->N + n];
    if (q < 0.0) return G[(long)i * s->N + node(s, x - CX[i], y - CY[i], z - CZ[i])];
    dual gj = G[(long)j * s->N + n];
    if (q < 0.5) {
        int x2 = x - CX[j], y2 = y - CY[j], z2 = z - CZ[j];
        int fluid2 = z2 >= 0 && z2 < s->p.nz && (s->p.periodic_x || (x2 >= 0 && x2 < s->p.nx));
        if (fluid2) {
            unsigned char t2 = s->type[node(s, x2, y2, z2)];
            fluid2 = t2 != SOLID && t2 != PLATE;
        }
        if (fluid2) {
            dual g2 = G[(long)j * s->N + node(s, x2, y2, z2)];
            return dadd(dscale(gj, 2.0 * q), dscale(g2, 1.0 - 2.0 * q));
        }
        return gj;
    }
    dual gi = G[(long)i * s->N + n];
    return dadd(dscale(gj, 1.0 / (2.0 * q)), dscale(gi, (2.0 * q - 1.0) / (2.0 * q)));
}

static void step(chan_state *s, const int *opp) {
    const chan_params *P = &s->p;
    /* 1. streaming into interior fluid nodes */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long n = node(s, x, y, z);
                if (s->type[n] != FLUID) continue;
                for (int i = 0; i < NQ; ++i) s->f[(long)i * s->N + n] = pull(s, s->G, x, y, z, i, opp);
            }
    /* 2. inlet and outlet nodes */
    if (!P->periodic_x)
#pragma omp parallel for schedule(static)
        for (int z = 0; z < P->nz; ++z)
            for (int y = 0; y < P->ny; ++y) {
                double zh = (z + 0.5) / P->nz;
                dual u_in[3] = {dscale(s->theta[0], 4.0 * zh * (1.0 - zh)), dc(0), dc(0)};
                dual rho1, u1[3];
                moments(s, s->f, node(s, 1, y, z), &rho1, u1);
                long n0 = node(s, 0, y, z);
                for (int i = 0; i < NQ; ++i) s->f[(long)i * s->N + n0] = feq(i, rho1, u_in);
                dual rho2, u2[3];
                moments(s, s->f, node(s, P->nx - 2, y, z), &rho2, u2);
                long n1 = node(s, P->nx - 1, y, z);
                for (int i = 0; i < NQ; ++i) s->f[(long)i * s->N + n1] = feq(i, dc(1.0), u2);
            }
    /* 3. collision */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long n = node(s, x, y, z);
                unsigned char t = s->type[n];
                if (t == FLUID) collide(s, n);
                else if (t == INLET || t == OUTLET)
                    for (int i = 0; i < NQ; ++i) s->G[(long)i * s->N + n] = s->f[(long)i * s->N + n];
            }
}

/* 4. plate drag of the current G (x component), summed in (node, j) order. */
static dual drag(const chan_state *s) {
    dual D = dc(0);
    for (long n = 0; n < s->N; ++n) {
        unsigned char t = s->type[n];
        if (t == SOLID || t == PLATE) continue;
        for (int j = 1; j < NQ; ++j)
            if (s->plate_link[(long)j * s->N + n] && CX[j] != 0)
                D = dadd(D, dscale(s->G[(long)j * s->N + n], 2.0 * CX[j]));
    }
    return D;
}

/* Run the problem.  dtheta: tangent direction of (u_peak, gx, cs).  Outputs:
 * J and dJ (its derivative along dtheta); drag_out[S] the per-step drag
 * values (may be NULL); f_out[NQ][N] the final f^S values (may be NULL);
 * type_out[N] the node classes (may be NULL).  Returns 0, or -1 on bad
 * input or allocation failure. */
int chan_run(const chan_params *p, int np, const double *X, const double *R, const double *dtheta, double *J,
             double *dJ, double *drag_out, double *f_out, unsigned char *type_out) {
    if (p->nx < 4 || p->ny < 1 || p->nz < 1 || p->steps < 0 || !(p->tau0 > 0.5)) return -1;
    chan_state s;
    memset(&s, 0, sizeof(s));
    s.p = *p;
    s.N = (long)p->nx * p->ny * p->nz;
    s.type = calloc((size_t)s.N, 1);
    s.q = calloc((size_t)s.N * NQ, sizeof(double));
    s.plate_link = calloc((size_t)s.N * NQ, 1);
    s.f = calloc((size_t)s.N * NQ, sizeof(dual));
    s.G = calloc((size_t)s.N * NQ, sizeof(dual));
    int rc = 0;
    if (!s.type || !s.q || !s.plate_link || !s.f || !s.G) rc = -1;
    int opp[NQ];
    for (int i = 0; i < NQ; ++i) opp[i] = opposite(i);
    if (!rc)
        for (long k = 0; k < s.N * NQ; ++k) s.q[k] = -1.0;
    if (!rc) {
        s.theta[0].v = p->u_peak;
        s.theta[1].v = p->gx;
        s.theta[2].v = p->cs;
        for (int k = 0; k < 3; ++k) s.theta[k].d = dtheta ? dtheta[k] : 0.0;
        build_geometry(&s, np, X, R);
        /* f^0 = w, G^0 = collide(f^0) */
        for (long n = 0; n < s.N; ++n)
            for (int i = 0; i < NQ; ++i) s.f[(long)i * s.N + n] = dc(weight(i));
        for (long n = 0; n < s.N; ++n) {
            unsigned char t = s.type[n];
            if (t == FLUID) collide(&s, n);
            else
                for (int i = 0; i < NQ; ++i) s.G[(long)i * s.N + n] = s.f[(long)i * s.N + n];
        }
        dual Jsum = dc(0);
        int cnt = 0;
        for (int st = 1; st <= p->steps; ++st) {
            step(&s, opp);
            dual D = drag(&s);
            if (drag_out) drag_out[st - 1] = D.v;
            if (st >= p->avg_from) {
                Jsum = dadd(Jsum, D);
                ++cnt;
            }
        }
        if (J) *J = cnt ? Jsum.v / cnt : 0.0;
        if (dJ) *dJ = cnt ? Jsum.d / cnt : 0.0;
        if (f_out)
            for (long k = 0; k < s.N * NQ; ++k) f_out[k] = s.f[k].v;
        if (type_out) memcpy(type_out, s.type, (size_t)s.N);
    }
    free(s.type);
    free(s.q);
    free(s.plate_link);
    free(s.f);
    free(s.G);
    return rc;
}
