// Differentiation form: the mean plate drag of a channel flow and its
// gradient by a hand-written adjoint (reverse) of the stream-collide step
// with bounce-back, with checkpoint and recompute.
//
// Problem (lattice units).  D3Q19, x from an inlet plane (x = 0) to an
// outlet plane (x = nx - 1), y periodic, halfway walls at z = -1/2 and
// nz - 1/2, a fixed plate (node box) and fixed spheres.  Step s = 1 .. S:
//   f^s = P(G^{s-1}):  streaming (Eq. 13) into interior fluid nodes, with
//        bounce-back on cut links: walls and plate q = 1/2, spheres Bouzidi
//        (Eq. 19) with q the smallest root of |x + q c_j - X| = R, all at
//        rest; inlet nodes f = f^eq(rho(1, y, z), u_in(z)), u_in = u_peak
//        4 zh (1 - zh) x^, zh = (z + 1/2)/nz; outlet nodes f = f^eq(1,
//        u(nx - 2, y, z)) with u the force-shifted velocity of Eq. (6);
//   G^s = C(f^s):  the collision of the production kernels (collide_node:
//        BGK, Smagorinsky tau of Eq. 18, Guo source) at interior fluid
//        nodes; G = f at inlet and outlet nodes;
//   D^s = sum over plate links (x, j) of (G_j^s(x) + f_opp(j)^{s+1}(x)) c_j,x
//        = 2 G_j^s(x) c_j,x (momentum exchange, Eq. 25, on a halfway wall).
// f^0 = w (rest), J = mean of D^s over s in [avg_from, S], and the gradient
// is taken with respect to theta = (u_peak, g_x, C).
//
// Populations are stored as FP32 deviations from w, like the production
// path; the pull rules are affine with weights summing to 1 and w_opp(j) =
// w_j, so they apply to deviations unchanged.  Geometry (node classes and
// link fractions) is decided once in FP64 with round-to-nearest intrinsics
// in the order the FP64 oracle uses, so both classify every node alike.
//
// Reverse.  With lambda^s = dJ/df^s and gbar^s = dJ/dG^s:
//   gbar^s = (dD^s/dG^s) [s in the window] / n + P'(G^s)^T lambda^{s+1}
//   lambda^s = C'(f^s)^T gbar^s  (identity at inlet and outlet nodes)
//   dJ/dtheta = sum_s gbar^s . dC/dtheta + lambda^{s+1} . dP/dtheta
// P^T is a gather: the entry G_i(x) is read by the regular pull of
// x + c_i, by the bounce-back of x's own cut links and by the Bouzidi rule
// of the fluid node x + c_i whose link along c_i is cut with q < 1/2; the
// inlet and outlet rows add the adjoint of rho(1, y, z) and u(nx-2, y, z)
// to the nodes they read (k_chan_bc_adj).  C^T is the analytic
// vector-Jacobian product of collide_node (chan_collide_vjp).  The forward
// run keeps f^s every K steps; the reverse sweep recomputes each K-step
// segment from its checkpoint, keeping its f^s, and runs the segment
// backwards.  Parameter gradients are summed per block in FP64 and added
// with FP64 atomics.
#include <cmath>
#include <vector>

#include "lbm_collide_node.cuh"

namespace lbm {
namespace {

enum : uint8_t { CH_FLUID = 0, CH_SOLID = 1, CH_INLET = 2, CH_OUTLET = 3, CH_PLATE = 4 };

struct ChanGeo {
    int nx, ny, nz, N;
    const uint8_t *type;    // [N]
    const uint8_t *cut;     // [N]: 1 if some link x -> x + c_j is cut (then q is read)
    const float *q;         // [Q][N]: fraction of the cut link x -> x + c_j, -1 if not cut
    const uint32_t *plate;  // [N]: bit j set if x -> x + c_j ends in the plate
    // neighbour masks (static geometry, for the reverse gather): bit i set if
    // x + c_i is in the box and is an interior fluid node (mfl), also has a
    // cut link (mcut), or is any fluid class, inlet / outlet included (many)
    const uint32_t *mfl, *mcut, *many;
};

__device__ __forceinline__ int wrapy(int y, int ny) { return y < 0 ? y + ny : (y >= ny ? y - ny : y); }

__device__ __forceinline__ bool is_fluid_type(uint8_t t) { return t != CH_SOLID && t != CH_PLATE; }

// Node index of (x, y, z) + c, or -1 outside the box in x or z.
__device__ __forceinline__ int nbr(const ChanGeo &G, int x, int y, int z, int cxv, int cyv, int czv) {
    const int xx = x + cxv, zz = z + czv;
    if (xx < 0 || xx >= G.nx || zz < 0 || zz >= G.nz) return -1;
    return xx + G.nx * (wrapy(y + cyv, G.ny) + G.ny * zz);
}

// ---- geometry ---------------------------------------------------------------

__device__ __forceinline__ double offs(double xi, double Xc, int n, bool periodic) {
    double d = __dsub_rn(xi, Xc);
    if (periodic) {
        if (d > 0.5 * n) d = __dsub_rn(d, (double)n);
        if (d < -0.5 * n) d = __dadd_rn(d, (double)n);
    }
    return d;
}

__device__ __forceinline__ double sq3(double a, double b, double c) {
    return __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c));
}

__device__ __forceinline__ bool in_box(const int *lo, const int *hi, int x, int y, int z) {
    return x >= lo[0] && x <= hi[0] && y >= lo[1] && y <= hi[1] && z >= lo[2] && z <= hi[2];
}

struct PlateBox {
    int lo[3], hi[3];
};

__device__ uint8_t node_type(int nx, int ny, int x, int y, int z, const PlateBox &pb, int np, const double *X,
                             const double *R) {
    if (x == 0) return CH_INLET;
    if (x == nx - 1) return CH_OUTLET;
    if (in_box(pb.lo, pb.hi, x, y, z)) return CH_PLATE;
    for (int a = 0; a < np; ++a) {
        const double dx = offs(x, X[3 * a], nx, false), dy = offs(y, X[3 * a + 1], ny, true);
        const double dz = __dsub_rn((double)z, X[3 * a + 2]);
        if (sq3(dx, dy, dz) < __dmul_rn(R[a], R[a])) return CH_SOLID;
    }
    return CH_FLUID;
}

__global__ void k_chan_types(const int nx, const int ny, const int nz, const PlateBox pb, const int np,
                             const double *__restrict__ X, const double *__restrict__ R, uint8_t *__restrict__ type) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nx * ny * nz) return;
    const int x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
    type[n] = node_type(nx, ny, x, y, z, pb, np, X, R);
}

// Cut links of every fluid node (the branch q < 1/2 is decided in FP64 and
// kept when q is rounded to FP32).
__global__ void k_chan_links(const int nx, const int ny, const int nz, const int np, const double *__restrict__ X,
                             const double *__restrict__ R, const uint8_t *__restrict__ type, float *__restrict__ qout,
                             uint32_t *__restrict__ plate, uint8_t *__restrict__ cut) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = nx * ny * nz;
    if (n >= N) return;
    const int x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
    uint32_t pm = 0;
    bool any = false;
    qout[n] = -1.f;  // j = 0
    for (int j = 1; j < Q; ++j) {
        float qf = -1.f;
        if (is_fluid_type(type[n])) {
            const int xx = x + rcx(j), zz = z + rcz(j);
            if (zz < 0 || zz >= nz) {
                qf = 0.5f;
            } else if (xx >= 0 && xx < nx) {
                const int m = xx + nx * (wrapy(y + rcy(j), ny) + ny * zz);
                if (type[m] == CH_PLATE) {
                    qf = 0.5f;
                    pm |= 1u << j;
                } else if (type[m] == CH_SOLID) {
                    double best = 2.0;
                    for (int a = 0; a < np; ++a) {
                        const double dx = offs(x, X[3 * a], nx, false), dy = offs(y, X[3 * a + 1], ny, true);
                        const double dz = __dsub_rn((double)z, X[3 * a + 2]);
                        const double ex = __dadd_rn(dx, (double)rcx(j)), ey = __dadd_rn(dy, (double)rcy(j));
                        const double ez = __dadd_rn(dz, (double)rcz(j));
                        if (!(sq3(ex, ey, ez) < __dmul_rn(R[a], R[a]))) continue;
                        const double aa = (double)(rcx(j) * rcx(j) + rcy(j) * rcy(j) + rcz(j) * rcz(j));
                        const double b = __dadd_rn(__dadd_rn(rcx(j) * dx, rcy(j) * dy), rcz(j) * dz);
                        const double c0 = __dsub_rn(sq3(dx, dy, dz), __dmul_rn(R[a], R[a]));
                        double disc = __dsub_rn(__dmul_rn(b, b), __dmul_rn(aa, c0));
                        if (disc < 0.0) disc = 0.0;
                        const double t = __ddiv_rn(c0, __dadd_rn(-b, __dsqrt_rn(disc)));
                        if (t < best) best = t;
                    }
                    if (best > 1.0) best = 1.0;
                    if (best < 0.0) best = 0.0;
                    qf = (float)best;
                    if (best < 0.5 && !(qf < 0.5f)) qf = 0.49999997f;  // keep the FP64 branch
                }
            }
        }
        qout[(size_t)j * N + n] = qf;
        any |= qf >= 0.f;
    }
    plate[n] = pm;
    cut[n] = any ? 1 : 0;
}

// Neighbour masks of every node (see ChanGeo).
__global__ void k_chan_masks(const ChanGeo G, uint32_t *__restrict__ mfl, uint32_t *__restrict__ mcut,
                             uint32_t *__restrict__ many) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= G.N) return;
    const int x = n % G.nx, y = (n / G.nx) % G.ny, z = n / (G.nx * G.ny);
    uint32_t a = 0u, b = 0u, c = 0u;
    for (int i = 0; i < Q; ++i) {
        const int tn = nbr(G, x, y, z, rcx(i), rcy(i), rcz(i));
        if (tn < 0) continue;
        const uint8_t t = G.type[tn];
        if (t == CH_FLUID) {
            a |= 1u << i;
            if (G.cut[tn]) b |= 1u << i;
        }
        if (is_fluid_type(t)) c |= 1u << i;
    }
    mfl[n] = a;
    mcut[n] = b;
    many[n] = c;
}

// ---- forward -----------------------------------------------------------------

// Incoming population i at interior fluid node (x, y, z), index n, from G
// (cut: whether any link of the node is cut).
__device__ __forceinline__ float pull(const ChanGeo &G, const float *__restrict__ Gin, int x, int y, int z, int n,
                                      int i, bool cut) {
    const int j = ropp(i);
    const float q = cut ? G.q[(size_t)j * G.N + n] : -1.f;
    if (q < 0.f) return Gin[(size_t)i * G.N + nbr(G, x, y, z, -rcx(i), -rcy(i), -rcz(i))];
    const float gj = Gin[(size_t)j * G.N + n];
    if (q < 0.5f) {
        const int n2 = nbr(G, x, y, z, -rcx(j), -rcy(j), -rcz(j));
        if (n2 >= 0 && is_fluid_type(G.type[n2])) return 2.f * q * gj + (1.f - 2.f * q) * Gin[(size_t)j * G.N + n2];
        return gj;
    }
    return gj / (2.f * q) + (2.f * q - 1.f) / (2.f * q) * Gin[(size_t)i * G.N + n];
}

// Deviation of f^eq_i(rho, u) (Eq. 9) from w_i.
__device__ __forceinline__ float feq_dev(int i, float rho, float ux, float uy, float uz) {
    const float cu = rcx(i) * ux + rcy(i) * uy + rcz(i) * uz, uu = ux * ux + uy * uy + uz * uz;
    const float w = (float)rw36(i) / 36.f;
    return w * (rho * (1.f + 3.f * cu + 4.5f * cu * cu - 1.5f * uu) - 1.f);
}

__device__ __forceinline__ void moments(const float *d, float &rho, float &jx, float &jy, float &jz) {
    rho = 1.f;
    jx = jy = jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rho += d[i];
        jx += rcx(i) * d[i];
        jy += rcy(i) * d[i];
        jz += rcz(i) * d[i];
    }
}

__device__ __forceinline__ void block_add(double v, double *dst) {
    __shared__ double part[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) part[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += part[k];
        if (s != 0.0) atomicAdd(dst, s);
    }
}

// Warp sum of a plate-drag contribution, one FP64 atomic per warp that has
// any (most warps have none).
__device__ __forceinline__ void warp_add(double v, double *dst) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(dst, v);
}

// One step at the interior fluid nodes (PULL: f^s pulled from G^{s-1}) or at
// every fluid node (!PULL: f^s = fin, the stored state): record f^s in frec
// (may be null), G^s = C(f^s) into Gout (G = f at inlet and outlet nodes),
// plate drag of G^s added to *drag (may be null).  With PULL the inlet and
// outlet planes are k_chan_bc_step's.
template <bool PULL>
__global__ void __launch_bounds__(256, 4) k_chan_step(const ChanGeo G, const Phys ph, const float *__restrict__ Gin,
                                                   const float *__restrict__ fin, float *__restrict__ frec,
                                                   float *__restrict__ Gout, double *__restrict__ drag,
                                                   int *__restrict__ status) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    double D = 0.0;
    if (n < G.N) {
        const uint8_t t = G.type[n];
        if (PULL ? t == CH_FLUID : is_fluid_type(t)) {
            float d[Q];
            if (!PULL) {
#pragma unroll
                for (int i = 0; i < Q; ++i) d[i] = fin[(size_t)i * G.N + n];
            } else {
                const int x = n % G.nx, y = (n / G.nx) % G.ny, z = n / (G.nx * G.ny);
                const bool cut = G.cut[n] != 0;
                if (!cut) {
                    // no cut link: every x - c_i is in the box (walls and the plate
                    // cut the links that would leave it; x is interior), plain pull
                    // with y periodic
                    const int ym = y == 0 ? G.nx * (G.ny - 1) : -G.nx;
                    const int yp = y == G.ny - 1 ? -G.nx * (G.ny - 1) : G.nx;
                    const int zp = G.nx * G.ny;
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        const int off = -rcx(i) + (rcy(i) > 0 ? ym : (rcy(i) < 0 ? yp : 0)) - rcz(i) * zp;
                        d[i] = Gin[(size_t)i * G.N + n + off];
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < Q; ++i) d[i] = pull(G, Gin, x, y, z, n, i, cut);
                }
            }
            if (frec)
#pragma unroll
                for (int i = 0; i < Q; ++i) frec[(size_t)i * G.N + n] = d[i];
            if (t == CH_FLUID) collide_node(ph, d, status);
#pragma unroll
            for (int i = 0; i < Q; ++i) Gout[(size_t)i * G.N + n] = d[i];
            const uint32_t pm = G.plate[n];
            if (pm)
#pragma unroll
                for (int j = 1; j < Q; ++j)
                    if (((pm >> j) & 1u) && rcx(j) != 0)
                        D += 2.0 * rcx(j) * ((double)d[j] + (double)rw36(j) / 36.0);
        }
    }
    if (drag) warp_add(D, drag);
}

// Inlet (x = 0) and outlet (x = nx - 1) planes of a pulled step, one thread
// per (y, z, side): the equilibrium of Eq. (9) from the populations pulled at
// the neighbour plane; G = f there (not collided).
__global__ void __launch_bounds__(128) k_chan_bc_step(const ChanGeo G, const Phys ph, const float u_peak,
                                                      const float *__restrict__ Gin, float *__restrict__ frec,
                                                      float *__restrict__ Gout) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int P = G.ny * G.nz;
    if (k >= 2 * P) return;
    const bool inlet = k < P;
    const int yz = inlet ? k : k - P, y = yz % G.ny, z = yz / G.ny;
    const int xs = inlet ? 1 : G.nx - 2, ns = xs + G.nx * yz, n = (inlet ? 0 : G.nx - 1) + G.nx * yz;
    float e[Q], d[Q];
    const bool cut = G.cut[ns] != 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) e[i] = pull(G, Gin, xs, y, z, ns, i, cut);
    float rho, jx, jy, jz;
    moments(e, rho, jx, jy, jz);
    if (inlet) {
        const float zh = (z + 0.5f) / G.nz;
        const float ux = u_peak * 4.f * zh * (1.f - zh);
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = feq_dev(i, rho, ux, 0.f, 0.f);
    } else {
        const float ux = jx / rho + 0.5f * ph.g[0], uy = jy / rho + 0.5f * ph.g[1], uz = jz / rho + 0.5f * ph.g[2];
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = feq_dev(i, 1.f, ux, uy, uz);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (frec) frec[(size_t)i * G.N + n] = d[i];
        Gout[(size_t)i * G.N + n] = d[i];
    }
}

// ---- reverse -----------------------------------------------------------------

// Adjoint of the inlet and outlet rows of P at step s + 1, one thread per
// (y, z):  rho_bar(y, z) is added to the adjoint of every population pulled
// at (1, y, z), ext[k](y, z) to that of population k pulled at (nx-2, y, z);
// the u_peak and g_x terms go to grad.
__global__ void __launch_bounds__(128) k_chan_bc_adj(const ChanGeo G, const Phys ph, const float u_peak,
                                                     const float *__restrict__ lam1, const float *__restrict__ f1,
                                                     float *__restrict__ rho_bar, float *__restrict__ ext,
                                                     double *__restrict__ grad) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;  // y + ny z
    const int P = G.ny * G.nz;
    double gu = 0.0, gg = 0.0;
    if (k < P) {
        const int y = k % G.ny, z = k / G.ny;
        const int n0 = G.nx * k, n1 = 1 + G.nx * k, n2 = G.nx - 2 + G.nx * k, nl = G.nx - 1 + G.nx * k;
        (void)y;
        // inlet: f_i(0) = rho_1 fe_i(1, u_in)
        const float zh = (z + 0.5f) / G.nz, sh = 4.f * zh * (1.f - zh), ux = u_peak * sh;
        float e[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) e[i] = f1[(size_t)i * G.N + n1];
        float rho1, jx, jy, jz;
        moments(e, rho1, jx, jy, jz);
        float rb = 0.f, ub = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float w = (float)rw36(i) / 36.f, cu = rcx(i) * ux, l = lam1[(size_t)i * G.N + n0];
            rb += l * w * (1.f + 3.f * cu + 4.5f * cu * cu - 1.5f * ux * ux);
            ub += l * w * (3.f * rcx(i) + 9.f * cu * rcx(i) - 3.f * ux);
        }
        rho_bar[k] = rb;
        gu = (double)ub * rho1 * sh;
        // outlet: f_i(nx-1) = f^eq_i(1, u(nx-2)), u = j / rho + g / 2
#pragma unroll
        for (int i = 0; i < Q; ++i) e[i] = f1[(size_t)i * G.N + n2];
        float rho2;
        moments(e, rho2, jx, jy, jz);
        const float ir = 1.f / rho2;
        const float u[3] = {jx * ir + 0.5f * ph.g[0], jy * ir + 0.5f * ph.g[1], jz * ir + 0.5f * ph.g[2]};
        float uba[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float w = (float)rw36(i) / 36.f, l = lam1[(size_t)i * G.N + nl];
            const float cu = rcx(i) * u[0] + rcy(i) * u[1] + rcz(i) * u[2];
            uba[0] += l * w * (3.f * rcx(i) + 9.f * cu * rcx(i) - 3.f * u[0]);
            uba[1] += l * w * (3.f * rcy(i) + 9.f * cu * rcy(i) - 3.f * u[1]);
            uba[2] += l * w * (3.f * rcz(i) + 9.f * cu * rcz(i) - 3.f * u[2]);
        }
        const float v[3] = {jx * ir, jy * ir, jz * ir};
#pragma unroll
        for (int i = 0; i < Q; ++i)
            ext[(size_t)i * P + k] = ir * (uba[0] * (rcx(i) - v[0]) + uba[1] * (rcy(i) - v[1]) + uba[2] * (rcz(i) - v[2]));
        gg = 0.5 * (double)uba[0];
    }
    block_add(gu, grad + 0);
    block_add(gg, grad + 1);
}

// Vector-Jacobian product of collide_node at deviations d: lam = C'(d)^T gb,
// and the products with dC/dg_x and dC/dsmag (smag = 18 sqrt(2) C^2).
__device__ __forceinline__ void chan_collide_vjp(const Phys &ph, const float (&d)[Q], const float (&gb)[Q],
                                                 float (&lam)[Q], float &gx_bar, float &smag_bar) {
    // forward intermediates
    float drho = 0.f, j[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += d[i];
        j[0] += rcx(i) * d[i];
        j[1] += rcy(i) * d[i];
        j[2] += rcz(i) * d[i];
    }
    const float rho = 1.f + drho, ir = 1.f / rho;
    const float u[3] = {j[0] * ir + 0.5f * ph.g[0], j[1] * ir + 0.5f * ph.g[1], j[2] * ir + 0.5f * ph.g[2]};
    const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    float m[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // xx yy zz xy xz yz
    float P6[6], Qn = 0.f, inner = ph.tau0 * ph.tau0, tau = ph.tau0;
    const bool les = ph.smag > 0.f;
    if (les) {
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            m[0] += rcx(i) * rcx(i) * d[i];
            m[1] += rcy(i) * rcy(i) * d[i];
            m[2] += rcz(i) * rcz(i) * d[i];
            m[3] += rcx(i) * rcy(i) * d[i];
            m[4] += rcx(i) * rcz(i) * d[i];
            m[5] += rcy(i) * rcz(i) * d[i];
        }
        const float t3 = drho / 3.f;
        P6[0] = m[0] - t3 - rho * u[0] * u[0];
        P6[1] = m[1] - t3 - rho * u[1] * u[1];
        P6[2] = m[2] - t3 - rho * u[2] * u[2];
        P6[3] = m[3] - rho * u[0] * u[1];
        P6[4] = m[4] - rho * u[0] * u[2];
        P6[5] = m[5] - rho * u[1] * u[2];
        const float q2 = P6[0] * P6[0] + P6[1] * P6[1] + P6[2] * P6[2] +
                         2.f * (P6[3] * P6[3] + P6[4] * P6[4] + P6[5] * P6[5]);
        Qn = sqrtf(q2);
        inner = ph.smag * Qn * ir + ph.tau0 * ph.tau0;
        tau = ph.tau0 + 0.5f * (sqrtf(inner) - ph.tau0);
    }
    const float om = 1.f / tau, sk = 1.f - 0.5f * om, gx = ph.g[0];
    // g_i = (1 - om) d_i + om E_i + sk S_i,
    // E_i = w_i (drho - 1.5 rho uu + 4.5 rho cu^2 + 3 rho cu),
    // S_i = w_i rho g_x (3 c_ix - 3 u_x + 9 cu c_ix)
    float om_bar = 0.f, drho_bar = 0.f, rho_bar = 0.f, ub[3] = {0.f, 0.f, 0.f};
    gx_bar = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float w = (float)rw36(i) / 36.f;
        const float cu = rcx(i) * u[0] + rcy(i) * u[1] + rcz(i) * u[2];
        const float E = w * (drho - 1.5f * rho * uu + 4.5f * rho * cu * cu + 3.f * rho * cu);
        const float sb = w * rho * (3.f * rcx(i) - 3.f * u[0] + 9.f * cu * rcx(i));  // S_i / g_x
        const float S = sb * gx;
        lam[i] = (1.f - om) * gb[i];
        om_bar += gb[i] * (E - d[i] - 0.5f * S);
        const float Eb = om * gb[i], Sb = sk * gb[i];
        drho_bar += Eb * w;
        rho_bar += Eb * w * (-1.5f * uu + 4.5f * cu * cu + 3.f * cu) + Sb * sb * gx * ir;
        const float ke = Eb * w * rho, ks = Sb * w * rho * gx;
        ub[0] += ke * (-3.f * u[0] + 9.f * cu * rcx(i) + 3.f * rcx(i)) + ks * (-3.f + 9.f * rcx(i) * rcx(i));
        ub[1] += ke * (-3.f * u[1] + 9.f * cu * rcy(i) + 3.f * rcy(i)) + ks * (9.f * rcx(i) * rcy(i));
        ub[2] += ke * (-3.f * u[2] + 9.f * cu * rcz(i) + 3.f * rcz(i)) + ks * (9.f * rcx(i) * rcz(i));
        gx_bar += Sb * sb;
    }
    // om = 1 / tau, tau = tau0 + (sqrt(inner) - tau0) / 2, inner = smag Q / rho + tau0^2
    float ir_bar = 0.f, mb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    smag_bar = 0.f;
    if (les) {
        const float tau_bar = -om_bar * om * om;
        const float in_bar = tau_bar * 0.25f / sqrtf(inner);
        smag_bar = in_bar * Qn * ir;
        ir_bar += in_bar * ph.smag * Qn;
        const float Q_bar = in_bar * ph.smag * ir;
        const float q2_bar = Qn > 0.f ? Q_bar / (2.f * Qn) : 0.f;
        float Pb[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) Pb[k] = 2.f * P6[k] * q2_bar;
#pragma unroll
        for (int k = 3; k < 6; ++k) Pb[k] = 4.f * P6[k] * q2_bar;
#pragma unroll
        for (int k = 0; k < 6; ++k) mb[k] = Pb[k];
        drho_bar -= (Pb[0] + Pb[1] + Pb[2]) / 3.f;
        rho_bar -= Pb[0] * u[0] * u[0] + Pb[1] * u[1] * u[1] + Pb[2] * u[2] * u[2] + Pb[3] * u[0] * u[1] +
                   Pb[4] * u[0] * u[2] + Pb[5] * u[1] * u[2];
        ub[0] -= rho * (2.f * Pb[0] * u[0] + Pb[3] * u[1] + Pb[4] * u[2]);
        ub[1] -= rho * (2.f * Pb[1] * u[1] + Pb[3] * u[0] + Pb[5] * u[2]);
        ub[2] -= rho * (2.f * Pb[2] * u[2] + Pb[4] * u[0] + Pb[5] * u[1]);
    }
    // u = j / rho + g / 2
    const float jb[3] = {ub[0] * ir, ub[1] * ir, ub[2] * ir};
    ir_bar += ub[0] * j[0] + ub[1] * j[1] + ub[2] * j[2];
    gx_bar += 0.5f * ub[0];
    rho_bar -= ir_bar * ir * ir;
    const float dtot = drho_bar + rho_bar;  // rho = 1 + drho
#pragma unroll
    for (int i = 0; i < Q; ++i)
        lam[i] += dtot + jb[0] * rcx(i) + jb[1] * rcy(i) + jb[2] * rcz(i) + mb[0] * rcx(i) * rcx(i) +
                  mb[1] * rcy(i) * rcy(i) + mb[2] * rcz(i) * rcz(i) + mb[3] * rcx(i) * rcy(i) +
                  mb[4] * rcx(i) * rcz(i) + mb[5] * rcy(i) * rcz(i);
}

// Adjoint of the population pulled as k at interior fluid node t (at x = xt,
// row yz = y + ny z), with the inlet / outlet rows folded in.
__device__ __forceinline__ float eff(const ChanGeo &G, const float *__restrict__ lam1, const float *__restrict__ rho_bar,
                                     const float *__restrict__ ext, int t, int xt, int yz, int k) {
    float v = lam1[(size_t)k * G.N + t];
    if (xt == 1) v += rho_bar[yz];
    if (xt == G.nx - 2) v += ext[(size_t)k * (G.ny * G.nz) + yz];
    return v;
}

// Reverse step s: lambda^s from lambda^{s+1} (lam1) and f^s (fs; null for
// the rest state f^0 = w), weight wd of D^s in J (0 outside the window).
__global__ void __launch_bounds__(256, 3) k_chan_adj(const ChanGeo G, const Phys ph, const float *__restrict__ lam1,
                                                  const float *__restrict__ fs, const float *__restrict__ rho_bar,
                                                  const float *__restrict__ ext, const float wd,
                                                  float *__restrict__ lam0, double *__restrict__ grad) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    double ggx = 0.0, gsm = 0.0;
    if (n < G.N) {
        const int x = n % G.nx, y = (n / G.nx) % G.ny, z = n / (G.nx * G.ny);
        const uint8_t t = G.type[n];
        if (!is_fluid_type(t)) {
#pragma unroll
            for (int i = 0; i < Q; ++i) lam0[(size_t)i * G.N + n] = 0.f;
        } else {
            float gb[Q];
            const uint32_t pm = G.plate[n];
            const bool cut = G.cut[n] != 0;
            const int yz0 = y + G.ny * z;
            const uint32_t mf = G.mfl[n], mc = G.mcut[n], ma = G.many[n];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                float v = 0.f;
                if ((mf >> i) & 1u) {  // x + c_i is an interior fluid node
                    const int tn = nbr(G, x, y, z, rcx(i), rcy(i), rcz(i));
                    const int xt = x + rcx(i), yzt = wrapy(y + rcy(i), G.ny) + G.ny * (z + rcz(i));
                    v += eff(G, lam1, rho_bar, ext, tn, xt, yzt, i);  // regular pull of x + c_i
                    const float qt = ((mc >> i) & 1u) ? G.q[(size_t)i * G.N + tn] : -1.f;
                    if (qt >= 0.f && qt < 0.5f)
                        v += (1.f - 2.f * qt) * eff(G, lam1, rho_bar, ext, tn, xt, yzt, ropp(i));
                }
                if (t == CH_FLUID && cut) {
                    const float qi = G.q[(size_t)i * G.N + n];  // own link along c_i
                    if (qi >= 0.f) {
                        float a;
                        if (qi < 0.5f) {
                            a = ((ma >> ropp(i)) & 1u) ? 2.f * qi : 1.f;  // x - c_i fluid
                        } else {
                            a = 1.f / (2.f * qi);
                        }
                        v += a * eff(G, lam1, rho_bar, ext, n, x, yz0, ropp(i));
                    }
                    const float qo = G.q[(size_t)ropp(i) * G.N + n];  // own link along -c_i
                    if (qo >= 0.5f) v += (2.f * qo - 1.f) / (2.f * qo) * eff(G, lam1, rho_bar, ext, n, x, yz0, i);
                }
                if (wd != 0.f && ((pm >> i) & 1u)) v += wd * 2.f * rcx(i);
                gb[i] = v;
            }
            if (t == CH_FLUID) {
                float d[Q], lam[Q], gxb, smb;
#pragma unroll
                for (int i = 0; i < Q; ++i) d[i] = fs ? fs[(size_t)i * G.N + n] : 0.f;
                chan_collide_vjp(ph, d, gb, lam, gxb, smb);
#pragma unroll
                for (int i = 0; i < Q; ++i) lam0[(size_t)i * G.N + n] = lam[i];
                ggx = gxb;
                gsm = smb;
            } else {
#pragma unroll
                for (int i = 0; i < Q; ++i) lam0[(size_t)i * G.N + n] = gb[i];
            }
        }
    }
    block_add(ggx, grad + 1);
    block_add(gsm, grad + 2);
}

}  // namespace
}  // namespace lbm

using namespace lbm;

struct lbm_channel_s {
    lbm_channel_params p;
    int N = 0, np = 0, K = 0, nck = 0;
    uint8_t *type = nullptr, *cut = nullptr;
    float *q = nullptr;
    uint32_t *plate = nullptr;
    uint32_t *mfl = nullptr, *mcut = nullptr, *many = nullptr;
    double *X = nullptr, *R = nullptr;
    float *G[2] = {nullptr, nullptr}, *lam[2] = {nullptr, nullptr};
    float *seg = nullptr;   // K states f^s of a segment
    float *ckpt = nullptr;  // f^s at s = 0, K, 2K, ...
    float *fend = nullptr;  // f^S of the last forward
    float *rho_bar = nullptr, *ext = nullptr;
    double *drag = nullptr, *grad = nullptr;
    int *status = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Phys ph{};
    double theta[3] = {0.0, 0.0, 0.0};
    bool have_forward = false;
    size_t bytes = 0;
};

namespace {

ChanGeo geo_of(const lbm_channel_s *c) {
    ChanGeo g;
    g.nx = c->p.nx;
    g.ny = c->p.ny;
    g.nz = c->p.nz;
    g.N = c->N;
    g.type = c->type;
    g.cut = c->cut;
    g.q = c->q;
    g.plate = c->plate;
    g.mfl = c->mfl;
    g.mcut = c->mcut;
    g.many = c->many;
    return g;
}

void set_phys(lbm_channel_s *c) {
    c->ph = Phys{};
    c->ph.tau0 = (float)c->p.tau0;
    c->ph.smag = (float)(18.0 * std::sqrt(2.0) * c->theta[2] * c->theta[2]);
    c->ph.g[0] = (float)c->theta[1];
}

template <typename T>
int calloc_dev(lbm_channel_s *c, T **p, size_t n) {
    *p = nullptr;
    if (n == 0) return LBM_OK;
    if (cudaMalloc((void **)p, n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return LBM_ERR_NOMEM;
    }
    c->bytes += n * sizeof(T);
    return cudaMemsetAsync(*p, 0, n * sizeof(T), c->stream) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

void chan_release(lbm_channel_s *c) {
    void *ptrs[] = {c->type, c->cut, c->q, c->plate, c->mfl, c->mcut, c->many, c->X, c->R, c->G[0], c->G[1], c->lam[0], c->lam[1], c->seg, c->ckpt,
                    c->fend, c->rho_bar, c->ext, c->drag, c->grad, c->status};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

int chan_check(lbm_channel_s *c, int rc) {
    if (rc) {
        cudaGetLastError();
        return rc;
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    int st = 0;
    if (cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    return (st & ST_DIVERGED) ? LBM_ERR_DIVERGED : LBM_OK;
}

int launch_ok() { return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA; }

// Forward from f^{s0} (fin) over steps s0 + 1 .. s1: f^s recorded into
// rec(s) when it returns non-null; drag of G^s into drag[s - 1] when
// with_drag.
template <typename Rec>
int chan_run(lbm_channel_s *c, const float *fin, int s0, int s1, Rec rec, bool with_drag) {
    const ChanGeo g = geo_of(c);
    const int blocks = (c->N + 255) / 256, bblocks = (2 * c->p.ny * c->p.nz + 127) / 128;
    const float up = (float)c->theta[0];
    k_chan_step<false><<<blocks, 256, 0, c->stream>>>(g, c->ph, nullptr, fin, nullptr, c->G[s0 & 1],
                                                      with_drag && s0 >= 1 ? c->drag + (s0 - 1) : nullptr, c->status);
    int rc = launch_ok();
    for (int s = s0 + 1; s <= s1 && !rc; ++s) {
        float *fr = rec(s);
        k_chan_step<true><<<blocks, 256, 0, c->stream>>>(g, c->ph, c->G[(s - 1) & 1], nullptr, fr, c->G[s & 1],
                                                         with_drag ? c->drag + (s - 1) : nullptr, c->status);
        rc = launch_ok();
        if (!rc) k_chan_bc_step<<<bblocks, 128, 0, c->stream>>>(g, c->ph, up, c->G[(s - 1) & 1], fr, c->G[s & 1]);
        if (!rc) rc = launch_ok();
    }
    return rc;
}

}  // namespace

extern "C" {

int lbm_channel_create(const lbm_channel_params *prm, int32_t n, const double *pos, const double *radius,
                       lbm_channel *out) {
    if (!prm || !out || n < 0 || (n > 0 && (!pos || !radius))) return LBM_ERR_ARG;
    *out = nullptr;
    const lbm_channel_params &p = *prm;
    if (p.nx < 8 || p.ny < 1 || p.nz < 2 || !(p.tau0 > 0.5) || !(p.cs_smag >= 0.0)) return LBM_ERR_ARG;
    if (!std::isfinite(p.tau0) || !std::isfinite(p.cs_smag) || !std::isfinite(p.inlet_peak) ||
        !std::isfinite(p.body_accel_x))
        return LBM_ERR_ARG;
    if (p.steps < 1 || p.avg_from < 1 || p.avg_from > p.steps || p.checkpoint_every < 1) return LBM_ERR_ARG;
    if ((long long)p.nx * p.ny * p.nz * Q >= (1ll << 31)) return LBM_ERR_UNSUPPORTED;
    // obstacles stay clear of the inlet / outlet planes and their neighbours
    const bool plate = p.plate_lo[0] <= p.plate_hi[0] && p.plate_lo[1] <= p.plate_hi[1] && p.plate_lo[2] <= p.plate_hi[2];
    if (plate && (p.plate_lo[0] < 2 || p.plate_hi[0] > p.nx - 3)) return LBM_ERR_ARG;
    for (int a = 0; a < n; ++a) {
        const double *X = pos + 3 * a;
        if (!(radius[a] > 0.0) || !(X[0] - radius[a] > 1.0) || !(X[0] + radius[a] < p.nx - 2.0) ||
            !std::isfinite(X[1]) || !std::isfinite(X[2]))
            return LBM_ERR_ARG;
    }
    lbm_channel_s *c = new (std::nothrow) lbm_channel_s();
    if (!c) return LBM_ERR_NOMEM;
    c->p = p;
    c->N = p.nx * p.ny * p.nz;
    c->np = n;
    c->K = p.checkpoint_every;
    c->nck = p.steps / c->K + 1;
    c->theta[0] = p.inlet_peak;
    c->theta[1] = p.body_accel_x;
    c->theta[2] = p.cs_smag;
    set_phys(c);
    DeviceScope ds(p.device);
    int rc = cudaSetDevice(p.device) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
    if (!rc) {
        if (p.cuda_stream) {
            c->stream = (cudaStream_t)p.cuda_stream;
        } else if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) == cudaSuccess) {
            c->own_stream = true;
        } else {
            rc = LBM_ERR_CUDA;
        }
    }
    const size_t NQs = (size_t)c->N * Q, P = (size_t)p.ny * p.nz;
    if (!rc) rc = calloc_dev(c, &c->type, (size_t)c->N);
    if (!rc) rc = calloc_dev(c, &c->cut, (size_t)c->N);
    if (!rc) rc = calloc_dev(c, &c->q, NQs);
    if (!rc) rc = calloc_dev(c, &c->plate, (size_t)c->N);
    if (!rc) rc = calloc_dev(c, &c->mfl, (size_t)c->N);
    if (!rc) rc = calloc_dev(c, &c->mcut, (size_t)c->N);
    if (!rc) rc = calloc_dev(c, &c->many, (size_t)c->N);
    if (!rc) rc = calloc_dev(c, &c->X, 3 * (size_t)n);
    if (!rc) rc = calloc_dev(c, &c->R, (size_t)n);
    for (int k = 0; k < 2 && !rc; ++k) {
        rc = calloc_dev(c, &c->G[k], NQs);
        if (!rc) rc = calloc_dev(c, &c->lam[k], NQs);
    }
    if (!rc) rc = calloc_dev(c, &c->seg, NQs * c->K);
    if (!rc) rc = calloc_dev(c, &c->ckpt, NQs * c->nck);
    if (!rc) rc = calloc_dev(c, &c->fend, NQs);
    if (!rc) rc = calloc_dev(c, &c->rho_bar, P);
    if (!rc) rc = calloc_dev(c, &c->ext, P * Q);
    if (!rc) rc = calloc_dev(c, &c->drag, (size_t)p.steps);
    if (!rc) rc = calloc_dev(c, &c->grad, 3);
    if (!rc) rc = calloc_dev(c, &c->status, 1);
    if (!rc && n > 0 &&
        (cudaMemcpyAsync(c->X, pos, 3 * sizeof(double) * n, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
         cudaMemcpyAsync(c->R, radius, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream) != cudaSuccess))
        rc = LBM_ERR_CUDA;
    if (!rc) {
        PlateBox pb;
        for (int k = 0; k < 3; ++k) {
            pb.lo[k] = p.plate_lo[k];
            pb.hi[k] = p.plate_hi[k];
        }
        const int blocks = (c->N + 255) / 256;
        k_chan_types<<<blocks, 256, 0, c->stream>>>(p.nx, p.ny, p.nz, pb, n, c->X, c->R, c->type);
        rc = launch_ok();
        if (!rc)
            k_chan_links<<<blocks, 256, 0, c->stream>>>(p.nx, p.ny, p.nz, n, c->X, c->R, c->type, c->q, c->plate,
                                                        c->cut);
        if (!rc) rc = launch_ok();
        if (!rc) {
            k_chan_masks<<<blocks, 256, 0, c->stream>>>(geo_of(c), c->mfl, c->mcut, c->many);
            rc = launch_ok();
        }
    }
    rc = chan_check(c, rc);
    if (rc) {
        chan_release(c);
        delete c;
        return rc;
    }
    *out = c;
    return LBM_OK;
}

int lbm_channel_destroy(lbm_channel c) {
    if (!c) return LBM_ERR_ARG;
    DeviceScope ds(c->p.device);
    cudaStreamSynchronize(c->stream);
    chan_release(c);
    delete c;
    return LBM_OK;
}

int lbm_channel_set_theta(lbm_channel c, const double *theta) {
    if (!c || !theta || !std::isfinite(theta[0]) || !std::isfinite(theta[1]) || !(theta[2] >= 0.0) ||
        !std::isfinite(theta[2]))
        return LBM_ERR_ARG;
    for (int k = 0; k < 3; ++k) c->theta[k] = theta[k];
    set_phys(c);
    c->have_forward = false;
    return LBM_OK;
}

int lbm_channel_forward(lbm_channel c, double *J) {
    if (!c) return LBM_ERR_ARG;
    DeviceScope ds(c->p.device);
    const size_t NQs = (size_t)c->N * Q;
    const int S = c->p.steps, K = c->K;
    int rc = cudaMemsetAsync(c->drag, 0, sizeof(double) * S, c->stream) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
    if (!rc && cudaMemsetAsync(c->ckpt, 0, sizeof(float) * NQs, c->stream) != cudaSuccess) rc = LBM_ERR_CUDA;  // f^0 = w
    auto rec = [&](int s) -> float * {
        if (s == S) return c->fend;
        return s % K == 0 ? c->ckpt + NQs * (s / K) : nullptr;
    };
    if (!rc) rc = chan_run(c, c->ckpt, 0, S, rec, true);
    if (!rc && S % K == 0 &&
        cudaMemcpyAsync(c->ckpt + NQs * (S / K), c->fend, sizeof(float) * NQs, cudaMemcpyDeviceToDevice, c->stream) !=
            cudaSuccess)
        rc = LBM_ERR_CUDA;
    std::vector<double> d((size_t)S);
    if (!rc &&
        cudaMemcpyAsync(d.data(), c->drag, sizeof(double) * S, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        rc = LBM_ERR_CUDA;
    rc = chan_check(c, rc);
    if (rc) return rc;
    double sum = 0.0;
    for (int s = c->p.avg_from; s <= S; ++s) sum += d[s - 1];
    if (J) *J = sum / (S - c->p.avg_from + 1);
    c->have_forward = true;
    return LBM_OK;
}

int lbm_channel_backward(lbm_channel c, double *grad) {
    if (!c || !grad) return LBM_ERR_ARG;
    if (!c->have_forward) return LBM_ERR_ARG;  // the checkpoints belong to another theta
    DeviceScope ds(c->p.device);
    const size_t NQs = (size_t)c->N * Q, P = (size_t)c->p.ny * c->p.nz;
    const int S = c->p.steps, K = c->K, blocks = (c->N + 255) / 256, pblocks = (int)((P + 127) / 128);
    const ChanGeo g = geo_of(c);
    const float up = (float)c->theta[0];
    const float wd = (float)(1.0 / (S - c->p.avg_from + 1));
    int rc = cudaMemsetAsync(c->grad, 0, 3 * sizeof(double), c->stream) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
    if (!rc && cudaMemsetAsync(c->lam[(S + 1) & 1], 0, sizeof(float) * NQs, c->stream) != cudaSuccess)
        rc = LBM_ERR_CUDA;  // lambda^{S+1} = 0
    for (int seg = S / K; seg >= 0 && !rc; --seg) {
        const int s0 = seg * K, s1 = std::min(s0 + K - 1, S);  // reverse steps s1 .. s0
        const float *f0 = c->ckpt + NQs * seg;                   // f^{s0}
        // f^{s0+1} .. f^{min(s1+1, S)} into seg slots 0 .. K-1 (drag not needed again)
        const int last = std::min(s1 + 1, S);
        auto rec = [&](int s) -> float * { return c->seg + NQs * (size_t)(s - s0 - 1); };
        rc = chan_run(c, f0, s0, last, rec, false);
        for (int s = s1; s >= s0 && !rc; --s) {
            const float *fs = s == s0 ? f0 : c->seg + NQs * (size_t)(s - s0 - 1);
            const float *lam1 = c->lam[(s + 1) & 1];
            float *lam0 = c->lam[s & 1];
            if (s < S) {
                const float *f1 = c->seg + NQs * (size_t)(s - s0);  // f^{s+1}
                k_chan_bc_adj<<<pblocks, 128, 0, c->stream>>>(g, c->ph, up, lam1, f1, c->rho_bar, c->ext, c->grad);
            } else {
                if (cudaMemsetAsync(c->rho_bar, 0, sizeof(float) * P, c->stream) != cudaSuccess ||
                    cudaMemsetAsync(c->ext, 0, sizeof(float) * P * Q, c->stream) != cudaSuccess)
                    rc = LBM_ERR_CUDA;
            }
            if (!rc) rc = launch_ok();
            const float w = (s >= c->p.avg_from && s >= 1) ? wd : 0.f;
            if (!rc)
                k_chan_adj<<<blocks, 256, 0, c->stream>>>(g, c->ph, lam1, s == 0 ? nullptr : fs, c->rho_bar, c->ext, w,
                                                          lam0, c->grad);
            if (!rc) rc = launch_ok();
        }
    }
    double gr[3] = {0.0, 0.0, 0.0};
    if (!rc && cudaMemcpyAsync(gr, c->grad, sizeof(gr), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        rc = LBM_ERR_CUDA;
    rc = chan_check(c, rc);
    if (rc) return rc;
    grad[0] = gr[0];
    grad[1] = gr[1];
    grad[2] = gr[2] * 36.0 * std::sqrt(2.0) * c->theta[2];  // d smag / d C
    return LBM_OK;
}

int lbm_channel_drag(lbm_channel c, double *drag) {
    if (!c || !drag || !c->have_forward) return LBM_ERR_ARG;
    DeviceScope ds(c->p.device);
    int rc = cudaMemcpyAsync(drag, c->drag, sizeof(double) * c->p.steps, cudaMemcpyDeviceToHost, c->stream) ==
                     cudaSuccess
                 ? LBM_OK
                 : LBM_ERR_CUDA;
    return chan_check(c, rc);
}

int lbm_channel_populations(lbm_channel c, double *f) {
    if (!c || !f || !c->have_forward) return LBM_ERR_ARG;
    DeviceScope ds(c->p.device);
    std::vector<float> h((size_t)c->N * Q);
    int rc = cudaMemcpyAsync(h.data(), c->fend, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, c->stream) ==
                     cudaSuccess
                 ? LBM_OK
                 : LBM_ERR_CUDA;
    rc = chan_check(c, rc);
    if (rc) return rc;
    for (int i = 0; i < Q; ++i)
        for (int n = 0; n < c->N; ++n) f[(size_t)i * c->N + n] = (double)h[(size_t)i * c->N + n] + w36(i) / 36.0;
    return LBM_OK;
}

int lbm_channel_geometry(lbm_channel c, uint8_t *type) {
    if (!c || !type) return LBM_ERR_ARG;
    DeviceScope ds(c->p.device);
    int rc = cudaMemcpyAsync(type, c->type, (size_t)c->N, cudaMemcpyDeviceToHost, c->stream) == cudaSuccess
                 ? LBM_OK
                 : LBM_ERR_CUDA;
    return chan_check(c, rc);
}

}  // extern "C"
