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
// to the nodes they read (bc_adj_row).  C^T is the analytic vector-Jacobian
// product of collide_node (chan_collide_vjp).  The forward run keeps f^s
// every K steps; the reverse sweep recomputes each K-step segment from its
// checkpoint, keeping its f^s, and runs the segment backwards, one launch
// per step.  The boundary planes ride in extra blocks of the same launches:
// the inlet / outlet equilibria of a forward step, and the inlet / outlet
// adjoint that the next reverse step needs (it depends only on the step's
// inputs, lambda^{s+1} and f^s).  Parameter gradients are summed per block
// in FP64 into the block's own slots and added up once at the end of the
// sweep.
#include <cmath>
#include <vector>

#include "lbm_collide_node.cuh"

namespace lbm {
namespace {

enum : uint8_t { CH_FLUID = 0, CH_SOLID = 1, CH_INLET = 2, CH_OUTLET = 3, CH_PLATE = 4 };

struct ChanGeo {
    int nx, ny, nz, N;
    const uint8_t *type;    // [N]
    const uint32_t *cutm;   // [N]: bit j set if the link x -> x + c_j is cut (q is read only then)
    const float *q;         // [Q][N]: fraction of the cut link x -> x + c_j, -1 if not cut
    const uint32_t *plate;  // [N]: bit j set if x -> x + c_j ends in the plate
    // neighbour masks (static geometry): bit i set if x + c_i is in the box
    // and is an interior fluid node (mfl), is an interior fluid node whose
    // link along c_i is cut with q < 1/2 (mbq: the Bouzidi rule there reads
    // x), or is any fluid class, inlet / outlet included (many)
    const uint32_t *mfl, *mbq, *many;
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
                             uint32_t *__restrict__ plate, uint32_t *__restrict__ cutm) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = nx * ny * nz;
    if (n >= N) return;
    const int x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
    uint32_t pm = 0, cm = 0;
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
        if (qf >= 0.f) cm |= 1u << j;
    }
    plate[n] = pm;
    cutm[n] = cm;
}

// Neighbour masks of every node (see ChanGeo).
__global__ void k_chan_masks(const ChanGeo G, uint32_t *__restrict__ mfl, uint32_t *__restrict__ mbq,
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
            if (((G.cutm[tn] >> i) & 1u) && G.q[(size_t)i * G.N + tn] < 0.5f) b |= 1u << i;
        }
        if (is_fluid_type(t)) c |= 1u << i;
    }
    mfl[n] = a;
    mbq[n] = b;
    many[n] = c;
}

// ---- forward -----------------------------------------------------------------

// Incoming population i at interior fluid node (x, y, z), index n, from G
// (cut: whether any link of the node is cut).
__device__ __forceinline__ float pull(const ChanGeo &G, const float *__restrict__ Gin, int x, int y, int z, int n,
                                      int i, bool cut) {
    const int j = ropp(i);
    const float q = cut ? G.q[j * G.N + n] : -1.f;
    if (q < 0.f) return Gin[i * G.N + nbr(G, x, y, z, -rcx(i), -rcy(i), -rcz(i))];
    const float gj = Gin[j * G.N + n];
    if (q < 0.5f) {
        const int n2 = nbr(G, x, y, z, -rcx(j), -rcy(j), -rcz(j));
        if (n2 >= 0 && is_fluid_type(G.type[n2])) return 2.f * q * gj + (1.f - 2.f * q) * Gin[j * G.N + n2];
        return gj;
    }
    return gj / (2.f * q) + (2.f * q - 1.f) / (2.f * q) * Gin[i * G.N + n];
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

// Warp sums of three values added to the warp's own slots dst[0..2] (the
// same warp of the same block adds to them every reverse step, on one
// stream; no block barrier).
__device__ __forceinline__ void warp_part(double a, double b, double c, double *dst) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        dst[0] += a;
        dst[1] += b;
        dst[2] += c;
    }
}

// Warp sum of a plate-drag contribution, one FP64 atomic per warp that has
// any (most warps have none).
__device__ __forceinline__ void warp_add(double v, double *dst) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(dst, v);
}

// Launch shape of the per-node kernels: a block covers kChanTx consecutive
// nodes of one x row; grid (ceil(nx / kChanTx), ny, nz), so that (x, y, z)
// come from the block and thread indices without integer division.
constexpr int kChanTx = 128;
// Resident blocks per SM of k_chan_adj: 10 (48 registers, a few hundred
// bytes of spills to L1) waits out more of its latency than 8 at 64
// registers without spills (reverse sweep 87.7 against 89.1 ms per gradient
// of 500 steps; 12 blocks at 40 registers 88.2).
#ifndef LBM_CHAN_ADJ_MINB
#define LBM_CHAN_ADJ_MINB 10
#endif
// Resident blocks per SM of k_chan_step (the forward and the reverse
// sweep's recompute): 12 at 40 registers, 110.6 ms per gradient against
// 112.1 at 8 (64 registers) and 111.3 at 10; 16 (32 registers) spills
// heavily and took 129 ms.
#ifndef LBM_CHAN_STEP_MINB
#define LBM_CHAN_STEP_MINB 12
#endif

// Row neighbours of (y, z): y periodic; z - 1 and z + 1 clamped into the
// box (a pull from outside the box is replaced by the bounce-back of the cut
// wall link, so the clamped value is never used).
struct RowNb {
    int ym, yp, zm, zp;
    __device__ __forceinline__ RowNb(const ChanGeo &G, int y, int z) {
        ym = y == 0 ? G.ny - 1 : y - 1;
        yp = y == G.ny - 1 ? 0 : y + 1;
        zm = z == 0 ? 0 : z - 1;
        zp = z == G.nz - 1 ? z : z + 1;
    }
    // row index y' + ny z' of (y, z) + s (c_iy, c_iz), s = +1 or -1
    __device__ __forceinline__ int row(const ChanGeo &G, int y, int z, int i, int s) const {
        const int dy = s * rcy(i), dz = s * rcz(i);
        const int yy = dy > 0 ? yp : (dy < 0 ? ym : y), zz = dz > 0 ? zp : (dz < 0 ? zm : z);
        return yy + G.ny * zz;
    }
    // node index of (x, y, z) + s c_i (x + s c_ix must be in the box)
    __device__ __forceinline__ int at(const ChanGeo &G, int x, int y, int z, int i, int s) const {
        return x + s * rcx(i) + G.nx * row(G, y, z, i, s);
    }
};

// Inlet (x = 0) and outlet (x = nx - 1) planes of a pulled step, one thread
// per (y, z, side), k in [0, 2 ny nz): the equilibrium of Eq. (9) from the
// populations pulled at the neighbour plane; G = f there (not collided).
__device__ __noinline__ void bc_step_body(const ChanGeo G, const Phys ph, const float u_peak,
                                          const float *__restrict__ Gin, float *__restrict__ frec,
                                          float *__restrict__ Gout, const int k) {
    const int P = G.ny * G.nz;
    const bool inlet = k < P;
    const int yz = inlet ? k : k - P, y = yz % G.ny, z = yz / G.ny;
    const int xs = inlet ? 1 : G.nx - 2, ns = xs + G.nx * yz, n = (inlet ? 0 : G.nx - 1) + G.nx * yz;
    float e[Q], d[Q];
    const bool cut = G.cutm[ns] != 0;
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
        if (frec) frec[i * G.N + n] = d[i];
        Gout[i * G.N + n] = d[i];
    }
}

// Index of a thread of the blocks beyond the lattice (blockIdx.z >= nz: the
// slabs of extra blocks that a launch carries for the boundary planes).
__device__ __forceinline__ int extra_index(const ChanGeo &G) {
    return (((blockIdx.z - G.nz) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * kChanTx + threadIdx.x;
}

// One step at the interior fluid nodes (PULL: f^s pulled from G^{s-1}) or at
// every fluid node (!PULL: f^s = fin, the stored state): record f^s in frec
// (may be null), G^s = C(f^s) into Gout (G = f at inlet and outlet nodes),
// plate drag of G^s added to *drag (may be null).  With PULL the inlet and
// outlet planes are computed by the launch's extra blocks (blockIdx.z >= nz,
// bc_step_body).  The pull reads x - c_i for every direction, then replaces
// the populations of the node's cut links (bounce-back; Eq. 19 with q from
// the geometry, walls and plate q = 1/2).
template <bool PULL>
__global__ void __launch_bounds__(kChanTx, LBM_CHAN_STEP_MINB) k_chan_step(const ChanGeo G, const Phys ph, const float u_peak,
                                                       const float *__restrict__ Gin, const float *__restrict__ fin,
                                                       float *__restrict__ frec, float *__restrict__ Gout,
                                                       double *__restrict__ drag, int *__restrict__ status) {
    if (PULL && (int)blockIdx.z >= G.nz) {  // the inlet and outlet planes (independent of the other blocks)
        const int k = extra_index(G);
        if (k < 2 * G.ny * G.nz) bc_step_body(G, ph, u_peak, Gin, frec, Gout, k);
        return;
    }
    const int x = blockIdx.x * kChanTx + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    const int n = x + G.nx * (y + G.ny * z);
    double D = 0.0;
    if (x < G.nx) {
        const uint8_t t = G.type[n];
        if (PULL ? t == CH_FLUID : is_fluid_type(t)) {
            float d[Q];
            if (!PULL) {
#pragma unroll
                for (int i = 0; i < Q; ++i) d[i] = fin[i * G.N + n];
            } else {
                const RowNb nb(G, y, z);
#pragma unroll
                for (int i = 0; i < Q; ++i) d[i] = Gin[i * G.N + nb.at(G, x, y, z, i, -1)];
                const uint32_t cm = G.cutm[n];
                if (cm) {
                    const uint32_t ma = G.many[n];
#pragma unroll
                    for (int i = 1; i < Q; ++i) {
                        const int j = ropp(i);  // population i arrives from the cut link along c_j
                        if ((cm >> j) & 1u) {
                            const float q = G.q[j * G.N + n], gj = Gin[j * G.N + n];
                            if (q < 0.5f) {
                                // x - c_j = x + c_i: the second point of the rule, if it is fluid
                                d[i] = ((ma >> i) & 1u)
                                           ? 2.f * q * gj + (1.f - 2.f * q) * Gin[j * G.N + nb.at(G, x, y, z, i, 1)]
                                           : gj;
                            } else {
                                d[i] = gj / (2.f * q) + (2.f * q - 1.f) / (2.f * q) * Gin[i * G.N + n];
                            }
                        }
                    }
                }
            }
            if (frec)
#pragma unroll
                for (int i = 0; i < Q; ++i) frec[i * G.N + n] = d[i];
            if (t == CH_FLUID) collide_node(ph, d, status);
#pragma unroll
            for (int i = 0; i < Q; ++i) Gout[i * G.N + n] = d[i];
            const uint32_t pm = G.plate[n];
            if (pm)
#pragma unroll
                for (int j = 1; j < Q; ++j)
                    if (((pm >> j) & 1u) && rcx(j) != 0)
                        D += 2.0 * rcx(j) * ((double)d[j] + (double)rw36(j) / 36.0);
        }
    }
    if (drag && __any_sync(0xffffffffu, D != 0.0)) warp_add(D, drag);
}

// ---- reverse -----------------------------------------------------------------

// Adjoint of the inlet and outlet rows of P at step s + 1 for one row
// k = y + ny z, given lambda^{s+1} at the row's inlet node (li; bc_adj_inlet)
// or outlet node (lo; bc_adj_outlet) and f^{s+1} (f1):  rho_bar(y, z) is
// added to the adjoint of every population pulled at (1, y, z), ext[i](y, z)
// to that of population i pulled at (nx-2, y, z); gu and gg are the row's
// parts of dJ/du_peak and dJ/dg_x.
__device__ __forceinline__ void bc_adj_inlet(const ChanGeo &G, const float u_peak, const float (&li)[Q],
                                             const float *__restrict__ f1, const int k, float *__restrict__ rho_bar,
                                             double &gu) {
    const int z = k / G.ny, n1 = 1 + G.nx * k;
    // inlet: f_i(0) = rho_1 fe_i(1, u_in)
    const float zh = (z + 0.5f) / G.nz, sh = 4.f * zh * (1.f - zh), ux = u_peak * sh;
    float e[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) e[i] = f1[i * G.N + n1];
    float rho1, jx, jy, jz;
    moments(e, rho1, jx, jy, jz);
    float rb = 0.f, ub = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float w = (float)rw36(i) / 36.f, cu = rcx(i) * ux, l = li[i];
        rb += l * w * (1.f + 3.f * cu + 4.5f * cu * cu - 1.5f * ux * ux);
        ub += l * w * (3.f * rcx(i) + 9.f * cu * rcx(i) - 3.f * ux);
    }
    rho_bar[k] = rb;
    gu = (double)ub * rho1 * sh;
}

__device__ __forceinline__ void bc_adj_outlet(const ChanGeo &G, const Phys &ph, const float (&lo)[Q],
                                              const float *__restrict__ f1, const int k, float *__restrict__ ext,
                                              double &gg) {
    const int P = G.ny * G.nz, n2 = G.nx - 2 + G.nx * k;
    // outlet: f_i(nx-1) = f^eq_i(1, u(nx-2)), u = j / rho + g / 2
    float e[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) e[i] = f1[i * G.N + n2];
    float rho2, jx, jy, jz;
    moments(e, rho2, jx, jy, jz);
    const float ir = 1.f / rho2;
    const float u[3] = {jx * ir + 0.5f * ph.g[0], jy * ir + 0.5f * ph.g[1], jz * ir + 0.5f * ph.g[2]};
    float uba[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float w = (float)rw36(i) / 36.f, l = lo[i];
        const float cu = rcx(i) * u[0] + rcy(i) * u[1] + rcz(i) * u[2];
        uba[0] += l * w * (3.f * rcx(i) + 9.f * cu * rcx(i) - 3.f * u[0]);
        uba[1] += l * w * (3.f * rcy(i) + 9.f * cu * rcy(i) - 3.f * u[1]);
        uba[2] += l * w * (3.f * rcz(i) + 9.f * cu * rcz(i) - 3.f * u[2]);
    }
    const float v[3] = {jx * ir, jy * ir, jz * ir};
#pragma unroll
    for (int i = 0; i < Q; ++i)
        ext[i * P + k] = ir * (uba[0] * (rcx(i) - v[0]) + uba[1] * (rcy(i) - v[1]) + uba[2] * (rcz(i) - v[2]));
    gg = 0.5 * (double)uba[0];
}

// Vector-Jacobian product of collide_node at deviations d: lam = C'(d)^T gb,
// and the products with dC/dg_x and dC/dsmag (smag = 18 sqrt(2) C^2).
//
// The collision is g_k = (1 - om) d_k + om E_k + sk S_k with
//   E_k = w_k (drho - 1.5 rho u.u + 4.5 rho (c_k.u)^2 + 3 rho c_k.u),
//   S_k = w_k rho g_x (3 c_kx - 3 u_x + 9 (c_k.u) c_kx),  sk = 1 - om/2,
// and E, S and om depend on d only through drho, j and Pi.  So every sum
// over k that the chain rule needs is a moment of gb: with
//   N0 = sum w_k gb_k,  N1 = sum w_k gb_k c_k,  N2 = sum w_k gb_k c_k c_k,
// sum w gb (c.u) = u.N1, sum w gb (c.u)^2 = u.N2.u, sum w gb (c.u) c = N2 u.
// The result is lam_i = (1 - om) gb_i + A + B.c_i + M:c_i c_i, taken by
// opposite pairs (i, i + 9) like the forward collision.  Divisions and
// square roots use the hardware approximations (a few ulp): the adjoint
// only has to carry the gradient to well within its 1e-3 tolerance.  The deviations are
// read pair by pair from f (node n of [Q][N] arrays; null: the rest state)
// and the result is written to lam (same layout), so that only gb is held
// whole.
__device__ __forceinline__ void chan_collide_vjp(const Phys &ph, const float *__restrict__ f, const int n,
                                                 const int N, const float (&gb)[Q], float *__restrict__ lam,
                                                 float &gx_bar, float &smag_bar) {
    // forward intermediates (the moments of d, by opposite pairs)
    const float d0 = f ? f[n] : 0.f;
    float drho = d0, j[3] = {0.f, 0.f, 0.f}, m[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // m: xx yy zz xy xz yz
    float N0 = wf(0) * gb[0], N1[3] = {0.f, 0.f, 0.f}, N2[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, gd = gb[0] * d0;
#pragma unroll
    for (int i = 1; i <= 9; ++i) {
        const int k = i + 9;  // opp(i)
        const float di = f ? f[i * N + n] : 0.f, dk = f ? f[k * N + n] : 0.f;
        const float sp = di + dk, dm = di - dk;
        const float gs = wf(i) * (gb[i] + gb[k]), gm = wf(i) * (gb[i] - gb[k]);
        drho += sp;
        N0 += gs;
        gd += gb[i] * di + gb[k] * dk;
        if (cx(i)) { j[0] += cx(i) * dm; N1[0] += cx(i) * gm; m[0] += sp; N2[0] += gs; }
        if (cy(i)) { j[1] += cy(i) * dm; N1[1] += cy(i) * gm; m[1] += sp; N2[1] += gs; }
        if (cz(i)) { j[2] += cz(i) * dm; N1[2] += cz(i) * gm; m[2] += sp; N2[2] += gs; }
        if (cx(i) * cy(i)) { m[3] += cx(i) * cy(i) * sp; N2[3] += cx(i) * cy(i) * gs; }
        if (cx(i) * cz(i)) { m[4] += cx(i) * cz(i) * sp; N2[4] += cx(i) * cz(i) * gs; }
        if (cy(i) * cz(i)) { m[5] += cy(i) * cz(i) * sp; N2[5] += cy(i) * cz(i) * gs; }
    }
    const float rho = 1.f + drho, ir = __fdividef(1.f, rho);
    const float u[3] = {j[0] * ir + 0.5f * ph.g[0], j[1] * ir + 0.5f * ph.g[1], j[2] * ir + 0.5f * ph.g[2]};
    const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    float P6[6], Qn = 0.f, inner = ph.tau0 * ph.tau0, tau = ph.tau0;
    const bool les = ph.smag > 0.f;
    if (les) {
        const float t3 = drho * (1.f / 3.f);
        P6[0] = m[0] - t3 - rho * u[0] * u[0];
        P6[1] = m[1] - t3 - rho * u[1] * u[1];
        P6[2] = m[2] - t3 - rho * u[2] * u[2];
        P6[3] = m[3] - rho * u[0] * u[1];
        P6[4] = m[4] - rho * u[0] * u[2];
        P6[5] = m[5] - rho * u[1] * u[2];
        const float q2 = P6[0] * P6[0] + P6[1] * P6[1] + P6[2] * P6[2] +
                         2.f * (P6[3] * P6[3] + P6[4] * P6[4] + P6[5] * P6[5]);
        Qn = q2 > 0.f ? q2 * rsqrtf(q2) : 0.f;
        inner = ph.smag * Qn * ir + ph.tau0 * ph.tau0;
        tau = ph.tau0 + 0.5f * (inner * rsqrtf(inner) - ph.tau0);
    }
    const float om = __fdividef(1.f, tau), sk = 1.f - 0.5f * om, gx = ph.g[0];
    // moments of gb contracted with u
    const float N2u[3] = {N2[0] * u[0] + N2[3] * u[1] + N2[4] * u[2], N2[3] * u[0] + N2[1] * u[1] + N2[5] * u[2],
                          N2[4] * u[0] + N2[5] * u[1] + N2[2] * u[2]};
    const float uN1 = u[0] * N1[0] + u[1] * N1[1] + u[2] * N1[2];
    const float uN2u = u[0] * N2u[0] + u[1] * N2u[1] + u[2] * N2u[2];
    const float eq = -1.5f * uu * N0 + 4.5f * uN2u + 3.f * uN1;  // sum w gb (E/w - drho)/rho
    const float sx = 3.f * N1[0] - 3.f * u[0] * N0 + 9.f * N2u[0];  // sum gb S / (rho g_x)
    // om_bar = sum gb (E - d - S/2)
    const float om_bar = drho * N0 + rho * eq - gd - 0.5f * rho * gx * sx;
    float drho_bar = om * N0;
    float rho_bar = om * eq + sk * gx * sx;
    float ub[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) ub[a] = om * rho * (-3.f * u[a] * N0 + 9.f * N2u[a] + 3.f * N1[a]);
    const float ks = sk * rho * gx;
    ub[0] += ks * (-3.f * N0 + 9.f * N2[0]);
    ub[1] += ks * 9.f * N2[3];
    ub[2] += ks * 9.f * N2[4];
    gx_bar = sk * rho * sx;
    // om = 1 / tau, tau = tau0 + (sqrt(inner) - tau0) / 2, inner = smag Q / rho + tau0^2
    float ir_bar = 0.f, mb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    smag_bar = 0.f;
    if (les) {
        const float tau_bar = -om_bar * om * om;
        const float in_bar = tau_bar * 0.25f * rsqrtf(inner);
        smag_bar = in_bar * Qn * ir;
        ir_bar += in_bar * ph.smag * Qn;
        const float Q_bar = in_bar * ph.smag * ir;
        const float q2_bar = Qn > 0.f ? __fdividef(Q_bar, 2.f * Qn) : 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) mb[k] = 2.f * P6[k] * q2_bar;
#pragma unroll
        for (int k = 3; k < 6; ++k) mb[k] = 4.f * P6[k] * q2_bar;
        drho_bar -= (mb[0] + mb[1] + mb[2]) * (1.f / 3.f);
        rho_bar -= mb[0] * u[0] * u[0] + mb[1] * u[1] * u[1] + mb[2] * u[2] * u[2] + mb[3] * u[0] * u[1] +
                   mb[4] * u[0] * u[2] + mb[5] * u[1] * u[2];
        ub[0] -= rho * (2.f * mb[0] * u[0] + mb[3] * u[1] + mb[4] * u[2]);
        ub[1] -= rho * (2.f * mb[1] * u[1] + mb[3] * u[0] + mb[5] * u[2]);
        ub[2] -= rho * (2.f * mb[2] * u[2] + mb[4] * u[0] + mb[5] * u[1]);
    }
    // u = j / rho + g / 2
    const float jb[3] = {ub[0] * ir, ub[1] * ir, ub[2] * ir};
    ir_bar += ub[0] * j[0] + ub[1] * j[1] + ub[2] * j[2];
    gx_bar += 0.5f * ub[0];
    rho_bar -= ir_bar * ir * ir;
    const float dtot = drho_bar + rho_bar;  // rho = 1 + drho
    const float keep = 1.f - om;
    lam[n] = keep * gb[0] + dtot;
#pragma unroll
    for (int i = 1; i <= 9; ++i) {
        const int k = i + 9;
        float even = dtot, odd = 0.f;
        if (cx(i)) { even += mb[0]; odd += cx(i) * jb[0]; }
        if (cy(i)) { even += mb[1]; odd += cy(i) * jb[1]; }
        if (cz(i)) { even += mb[2]; odd += cz(i) * jb[2]; }
        if (cx(i) * cy(i)) even += cx(i) * cy(i) * mb[3];
        if (cx(i) * cz(i)) even += cx(i) * cz(i) * mb[4];
        if (cy(i) * cz(i)) even += cy(i) * cz(i) * mb[5];
        lam[i * N + n] = keep * gb[i] + even + odd;
        lam[k * N + n] = keep * gb[k] + even - odd;
    }
}

// The inlet / outlet part of the adjoint of the population pulled as k at
// interior fluid node t at x = xt (row yz): the inlet and outlet rows of P
// read the pulls at x = 1 and x = nx - 2.
__device__ __forceinline__ float edge_adj(const ChanGeo &G, const float *__restrict__ rho_bar,
                                          const float *__restrict__ ext, int xt, int yz, int k) {
    float v = 0.f;
    if (xt == 1) v += rho_bar[yz];
    if (xt == G.nx - 2) v += ext[k * (G.ny * G.nz) + yz];
    return v;
}

// Adjoint of the population pulled as k at interior fluid node t (at x = xt,
// row yz), with the inlet / outlet rows folded in.
__device__ __forceinline__ float eff(const ChanGeo &G, const float *__restrict__ lam1, const float *__restrict__ rho_bar,
                                     const float *__restrict__ ext, int t, int xt, int yz, int k) {
    return lam1[k * G.N + t] + edge_adj(G, rho_bar, ext, xt, yz, k);
}

// The adjoint gb of G^s at fluid-class node (x, y, z), index n, that the
// pulls of step s + 1 at the neighbours give: the regular pull of x + c_i
// (an interior fluid node) and the Bouzidi rule of x + c_i whose link along
// c_i is cut with q < 1/2 (it reads x).
__device__ __forceinline__ void gather_adj(const ChanGeo &G, const float *__restrict__ lam1,
                                           const float *__restrict__ rho_bar, const float *__restrict__ ext, int x,
                                           int y, int z, int n, float (&gb)[Q]) {
    const RowNb nb(G, y, z);
    const uint32_t mf = G.mfl[n], mb = G.mbq[n];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float v = 0.f;
        if ((mf >> i) & 1u) {
            const int xt = x + rcx(i), yzt = nb.row(G, y, z, i, 1), tn = xt + G.nx * yzt;
            v = eff(G, lam1, rho_bar, ext, tn, xt, yzt, i);
            if ((mb >> i) & 1u)
                v += (1.f - 2.f * G.q[i * G.N + tn]) * eff(G, lam1, rho_bar, ext, tn, xt, yzt, ropp(i));
        }
        gb[i] = v;
    }
}

// The inlet / outlet adjoint of step s - 1 for row k (k_chan_adj's extra
// blocks): lambda^s at the row's inlet and outlet nodes is their gathered gb.
// Not inlined, so that the node kernel's instruction stream stays short.
__device__ __noinline__ void adj_extra_row(const ChanGeo G, const Phys ph, const float u_peak,
                                           const float *__restrict__ lam1, const float *__restrict__ fs,
                                           const float *__restrict__ rho_bar, const float *__restrict__ ext,
                                           float *__restrict__ rho_nx, float *__restrict__ ext_nx, const int k,
                                           double &gup, double &ggx) {
    const int y = k % G.ny, z = k / G.ny;
    float l[Q];
    gather_adj(G, lam1, rho_bar, ext, 0, y, z, G.nx * k, l);
    bc_adj_inlet(G, u_peak, l, fs, k, rho_nx, gup);
    gather_adj(G, lam1, rho_bar, ext, G.nx - 1, y, z, G.nx - 1 + G.nx * k, l);
    bc_adj_outlet(G, ph, l, fs, k, ext_nx, ggx);
}

// Reverse step s: lambda^s from lambda^{s+1} (lam1) and f^s (fs; null for
// the rest state f^0 = w), weight wd of D^s in J (0 outside the window),
// with the inlet / outlet adjoint of step s + 1 in rho_bar and ext.  The
// parts of dJ/d(u_peak, g_x, smag) of each warp are added to its own slots
// of gpart (3 per warp, summed over the steps; no atomics).  The launch's
// extra blocks (blockIdx.z >= nz, present when rho_nx is not null) compute
// the inlet / outlet adjoint of step s that the next reverse step reads
// (rho_nx, ext_nx; from lambda^s at the inlet and outlet nodes, where it is
// the gathered gb, and f^s), independently of the other blocks.
__global__ void __launch_bounds__(kChanTx, LBM_CHAN_ADJ_MINB) k_chan_adj(
    const ChanGeo G, const Phys ph, const float u_peak, const float *__restrict__ lam1, const float *__restrict__ fs,
    const float *__restrict__ rho_bar, const float *__restrict__ ext, const float wd, float *__restrict__ lam0,
    float *__restrict__ rho_nx, float *__restrict__ ext_nx, double *__restrict__ gpart) {
    double gup = 0.0, ggx = 0.0, gsm = 0.0;
    if ((int)blockIdx.z >= G.nz) {
        const int k = extra_index(G);  // row y + ny z
        if (k < G.ny * G.nz) adj_extra_row(G, ph, u_peak, lam1, fs, rho_bar, ext, rho_nx, ext_nx, k, gup, ggx);
    } else {
        const int x = blockIdx.x * kChanTx + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
        const int n = x + G.nx * (y + G.ny * z);
        if (x < G.nx) {
            const uint8_t t = G.type[n];
            if (!is_fluid_type(t)) {
#pragma unroll
                for (int i = 0; i < Q; ++i) lam0[i * G.N + n] = 0.f;
            } else {
                float gb[Q];
                gather_adj(G, lam1, rho_bar, ext, x, y, z, n, gb);
                const int yz0 = y + G.ny * z;
                // the node's own cut links (the adjoint of the populations it pulls itself)
                const uint32_t cm = t == CH_FLUID ? G.cutm[n] : 0u;
                if (cm) {
                    const uint32_t ma = G.many[n];
#pragma unroll
                    for (int i = 1; i < Q; ++i) {
                        if ((cm >> i) & 1u) {  // link along c_i: population opp(i) reads G_i(x)
                            const float qi = G.q[i * G.N + n];
                            const float a = qi < 0.5f ? (((ma >> ropp(i)) & 1u) ? 2.f * qi : 1.f) : 1.f / (2.f * qi);
                            gb[i] += a * eff(G, lam1, rho_bar, ext, n, x, yz0, ropp(i));
                        }
                        if ((cm >> ropp(i)) & 1u) {  // link along -c_i with q >= 1/2: population i reads G_i(x)
                            const float qo = G.q[ropp(i) * G.N + n];
                            if (qo >= 0.5f) gb[i] += (2.f * qo - 1.f) / (2.f * qo) * eff(G, lam1, rho_bar, ext, n, x, yz0, i);
                        }
                    }
                }
                const uint32_t pm = G.plate[n];
                if (wd != 0.f && pm)
#pragma unroll
                    for (int i = 0; i < Q; ++i)
                        if ((pm >> i) & 1u) gb[i] += wd * 2.f * rcx(i);
                if (t == CH_FLUID) {
                    float gxb, smb;
                    chan_collide_vjp(ph, fs, n, G.N, gb, lam0, gxb, smb);
                    ggx = gxb;
                    gsm = smb;
                } else {
#pragma unroll
                    for (int i = 0; i < Q; ++i) lam0[i * G.N + n] = gb[i];
                }
            }
        }
    }
    const int warp = (blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)) * (kChanTx / 32) + (threadIdx.x >> 5);
    warp_part(gup, ggx, gsm, gpart + 3 * warp);
}

// grad[0..2] += the sum of the nb warps' parts.
__global__ void __launch_bounds__(256) k_chan_gsum(const double *__restrict__ gpart, int nb, double *__restrict__ grad) {
    double a[3] = {0.0, 0.0, 0.0};
    for (int k = threadIdx.x; k < nb; k += blockDim.x)
#pragma unroll
        for (int c = 0; c < 3; ++c) a[c] += gpart[3 * k + c];
    __shared__ double sh[3][8];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a[c] += __shfl_xor_sync(0xffffffffu, a[c], o);
        if ((threadIdx.x & 31) == 0) sh[c][threadIdx.x >> 5] = a[c];
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) a[c] += sh[c][w];
            grad[c] += a[c];
        }
}

}  // namespace
}  // namespace lbm

using namespace lbm;

struct lbm_channel_s {
    lbm_channel_params p;
    int N = 0, np = 0, K = 0, nck = 0;
    uint8_t *type = nullptr;
    uint32_t *cutm = nullptr;
    float *q = nullptr;
    uint32_t *plate = nullptr;
    uint32_t *mfl = nullptr, *mbq = nullptr, *many = nullptr;
    double *gpart = nullptr;  // per-warp parts of dJ/d(u_peak, g_x, smag) (k_chan_adj)
    double *X = nullptr, *R = nullptr;
    float *G[2] = {nullptr, nullptr}, *lam[2] = {nullptr, nullptr};
    float *seg = nullptr;   // K states f^s of a segment
    float *ckpt = nullptr;  // f^s at s = 0, K, 2K, ...
    float *fend = nullptr;  // f^S of the last forward
    float *rho_bar[2] = {nullptr, nullptr}, *ext[2] = {nullptr, nullptr};  // inlet / outlet adjoint, by step parity
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
    g.cutm = c->cutm;
    g.q = c->q;
    g.plate = c->plate;
    g.mfl = c->mfl;
    g.mbq = c->mbq;
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
    void *ptrs[] = {c->type, c->cutm, c->q, c->plate, c->mfl, c->mbq, c->many, c->gpart, c->X, c->R, c->G[0], c->G[1], c->lam[0], c->lam[1], c->seg, c->ckpt,
                    c->fend, c->rho_bar[0], c->rho_bar[1], c->ext[0], c->ext[1], c->drag, c->grad, c->status};
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

// Grid of the per-node kernels (see kChanTx) with extra slabs of blocks for
// `extra` more threads (the boundary-plane work), and its block count.
dim3 chan_grid(const lbm_channel_params &p, long long extra) {
    const long long gx = (p.nx + kChanTx - 1) / kChanTx, per_slab = gx * p.ny * kChanTx;
    return dim3((unsigned)gx, p.ny, p.nz + (unsigned)((extra + per_slab - 1) / per_slab));
}
int chan_warps(const lbm_channel_params &p, long long extra) {
    const dim3 g = chan_grid(p, extra);
    return (int)(g.x * g.y * g.z) * (kChanTx / 32);
}

// Forward from f^{s0} (fin) over steps s0 + 1 .. s1: f^s recorded into
// rec(s) when it returns non-null; drag of G^s into drag[s - 1] when
// with_drag.
template <typename Rec>
int chan_run(lbm_channel_s *c, const float *fin, int s0, int s1, Rec rec, bool with_drag) {
    const ChanGeo g = geo_of(c);
    const dim3 grid = chan_grid(c->p, 0), grid_bc = chan_grid(c->p, 2ll * c->p.ny * c->p.nz);
    const float up = (float)c->theta[0];
    k_chan_step<false><<<grid, kChanTx, 0, c->stream>>>(g, c->ph, up, nullptr, fin, nullptr, c->G[s0 & 1],
                                                      with_drag && s0 >= 1 ? c->drag + (s0 - 1) : nullptr, c->status);
    int rc = launch_ok();
    for (int s = s0 + 1; s <= s1 && !rc; ++s) {
        float *fr = rec(s);
        k_chan_step<true><<<grid_bc, kChanTx, 0, c->stream>>>(g, c->ph, up, c->G[(s - 1) & 1], nullptr, fr,
                                                              c->G[s & 1], with_drag ? c->drag + (s - 1) : nullptr,
                                                              c->status);
        rc = launch_ok();
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
    if ((long long)p.nx * p.ny * p.nz * Q >= (1ll << 31)) return LBM_ERR_UNSUPPORTED;  // kernels index [Q][N] in int
    // grid rows (y, z) of the per-node kernels, plus at most nz / 64 + 1 slabs of extra blocks in z
    if (p.ny > 65535 || p.nz > 64000) return LBM_ERR_UNSUPPORTED;
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
    if (!rc) rc = calloc_dev(c, &c->cutm, (size_t)c->N);
    if (!rc) rc = calloc_dev(c, &c->q, NQs);
    if (!rc) rc = calloc_dev(c, &c->plate, (size_t)c->N);
    if (!rc) rc = calloc_dev(c, &c->mfl, (size_t)c->N);
    if (!rc) rc = calloc_dev(c, &c->mbq, (size_t)c->N);
    if (!rc) rc = calloc_dev(c, &c->gpart, 3 * (size_t)chan_warps(p, (long long)p.ny * p.nz));
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
    for (int k = 0; k < 2 && !rc; ++k) {
        rc = calloc_dev(c, &c->rho_bar[k], P);
        if (!rc) rc = calloc_dev(c, &c->ext[k], P * Q);
    }
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
                                                        c->cutm);
        if (!rc) rc = launch_ok();
        if (!rc) {
            k_chan_masks<<<blocks, 256, 0, c->stream>>>(geo_of(c), c->mfl, c->mbq, c->many);
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
    const int S = c->p.steps, K = c->K;
    const dim3 grid = chan_grid(c->p, 0), grid_bc = chan_grid(c->p, (long long)P);
    const int nwarps = chan_warps(c->p, (long long)P);
    const ChanGeo g = geo_of(c);
    const float up = (float)c->theta[0];
    const float wd = (float)(1.0 / (S - c->p.avg_from + 1));
    int rc = cudaMemsetAsync(c->grad, 0, 3 * sizeof(double), c->stream) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
    if (!rc && cudaMemsetAsync(c->gpart, 0, 3 * sizeof(double) * nwarps, c->stream) != cudaSuccess)
        rc = LBM_ERR_CUDA;
    if (!rc && cudaMemsetAsync(c->lam[(S + 1) & 1], 0, sizeof(float) * NQs, c->stream) != cudaSuccess)
        rc = LBM_ERR_CUDA;  // lambda^{S+1} = 0
    // lambda^{S+1} = 0: no inlet / outlet adjoint enters reverse step S
    if (!rc && (cudaMemsetAsync(c->rho_bar[S & 1], 0, sizeof(float) * P, c->stream) != cudaSuccess ||
                cudaMemsetAsync(c->ext[S & 1], 0, sizeof(float) * P * Q, c->stream) != cudaSuccess))
        rc = LBM_ERR_CUDA;
    for (int seg = S / K; seg >= 0 && !rc; --seg) {
        const int s0 = seg * K, s1 = std::min(s0 + K - 1, S);  // reverse steps s1 .. s0
        const float *f0 = c->ckpt + NQs * seg;                   // f^{s0}
        // f^{s0+1} .. f^{s1} into seg slots 0 .. K-2 (drag not needed again)
        auto rec = [&](int s) -> float * { return c->seg + NQs * (size_t)(s - s0 - 1); };
        if (s1 > s0) rc = chan_run(c, f0, s0, s1, rec, false);
        for (int s = s1; s >= s0 && !rc; --s) {
            const float *fs = s == s0 ? f0 : c->seg + NQs * (size_t)(s - s0 - 1);
            const float w = (s >= c->p.avg_from && s >= 1) ? wd : 0.f;
            // the extra blocks of reverse step s > 0 prepare the inlet / outlet adjoint of step s - 1
            const bool nxt = s > 0;
            k_chan_adj<<<nxt ? grid_bc : grid, kChanTx, 0, c->stream>>>(
                g, c->ph, up, c->lam[(s + 1) & 1], s == 0 ? nullptr : fs, c->rho_bar[s & 1], c->ext[s & 1], w,
                c->lam[s & 1], nxt ? c->rho_bar[(s - 1) & 1] : nullptr, nxt ? c->ext[(s - 1) & 1] : nullptr,
                c->gpart);
            rc = launch_ok();
        }
    }
    if (!rc) {
        k_chan_gsum<<<1, 256, 0, c->stream>>>(c->gpart, nwarps, c->grad);
        rc = launch_ok();
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
