// Sphere DEM (Sect. 2.1): linear spring-dashpot normal contact (Eq. 1) between
// spheres and with the z walls, velocity Verlet in dem_substeps sub-steps per
// lattice step with the hydrodynamic (and external) load held constant.
//
// Reading of Eq. (1): f^n = k_n delta - gamma_n v_n for an overlap delta > 0
// (unclipped), gamma_n = -2 ln(e) sqrt(m_eff k_n) / sqrt(pi^2 + ln(e)^2), which
// gives a normal restitution of exactly e.  A fixed sphere moves with its
// prescribed velocity and acts with infinite mass.
//
// Precision.  Centres and velocities are FP64 and are updated once per
// lattice step, x <- x0 + dx, v <- v0 + dv, so their drift is FP64.  Within
// the step the sub-steps advance only the displacement dx and the velocity
// change dv, which are small, in FP32 (FP64 throughput on this GPU is ~1/64
// of FP32).  The overlap of a listed pair is evaluated without cancellation
// from FP64 start-of-step data: with d0 = x0_a - x0_b and
// c0 = (R_a + R_b)^2 - |d0|^2 (both FP64, once per step),
//   c = c0 - 2 d0.D - D.D,  D = dx_a - dx_b,   delta = c / (R_a + R_b + |d0 + D|),
// so delta keeps ~1e-8 absolute accuracy although |d0| ~ 2R.  Contact
// forces are summed in FP32 per sub-step; the spin is advanced once per step
// (the torque is constant over it).
//
// Sub-steps need every sphere's displacement of the previous sub-step.  One
// thread-block cluster runs all of them: each thread keeps its spheres in
// registers, publishes (dx, dv) in its CTA's shared memory (double-buffered by
// sub-step parity) and reads neighbours' through distributed shared memory;
// a hardware cluster barrier (release / acquire) separates drift and force.
// More spheres than one cluster holds fall back to a cooperative launch with
// a bounded software grid barrier.
//
// Neighbour lists (pairs within R_a + R_b + skin, FP32 search) are rebuilt
// only when a sphere has moved more than skin/2 - max_step since the last
// build; every sphere moving less than max_step per step (else the geometry
// error is raised) keeps every pair that can touch within a step in the list.
#include <cooperative_groups.h>

#include <vector>

#include "lbm_internal.cuh"

namespace lbm {

constexpr double kPi = 3.14159265358979323846;
constexpr int kDemKmax = 4;       // spheres per thread held in registers
constexpr int kDemThreads = 256;  // threads per CTA of the cluster kernel

__device__ __forceinline__ double sphere_mass(const Parts &pt, int a) {
    const double r = pt.R[a];
    return pt.rho_s * (4.0 / 3.0) * kPi * r * r * r;
}

__device__ __forceinline__ void min_image(const Lat &L, double d[3]) {
    if (d[0] > 0.5 * L.nx) d[0] -= L.nx;
    if (d[0] < -0.5 * L.nx) d[0] += L.nx;
    if (d[1] > 0.5 * L.ny) d[1] -= L.ny;
    if (d[1] < -0.5 * L.ny) d[1] += L.ny;
}

// One warp per sphere, step parity sp.  If a rebuild is due (or forced),
// list every b != a
// with |X_a - X_b| < R_a + R_b + skin in increasing b (centres staged through
// shared memory); then compute the pair constants of every list entry for
// the current centres and velocities:
//   pairA = (d0, c0),  d0 = X_a - X_b (minimum image), c0 = (R_a+R_b)^2 - |d0|^2
//   pairB = (V_a - V_b, gamma_n)
constexpr int kNbrTile = 1024;

__device__ __forceinline__ void neighbours_body(const Lat &L, const Parts &pt, const int sp, const int force,
                                                int *__restrict__ status) {
    __shared__ float4 tile[kNbrTile];
    const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const bool live = a < pt.np;
    const bool rebuild = force || *(volatile int *)(pt.rebuild + sp) != 0;
    if (rebuild) {
        float4 me = live ? pt.Xf[a] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float ra = me.w + (float)pt.skin;
        const float hx = 0.5f * L.nx, hy = 0.5f * L.ny;
        int cnt = 0;
        for (int t0 = 0; t0 < pt.np; t0 += kNbrTile) {
            const int tn = min(kNbrTile, pt.np - t0);
            __syncthreads();
            for (int i = threadIdx.x; i < tn; i += blockDim.x) tile[i] = pt.Xf[t0 + i];
            __syncthreads();
            if (!live) continue;
            for (int base = 0; base < tn; base += 32) {
                const int i = base + lane, b = t0 + i;
                bool ok = false;
                if (i < tn && b != a) {
                    const float4 o = tile[i];
                    float dx = me.x - o.x, dy = me.y - o.y;
                    const float dz = me.z - o.z;
                    if (dx > hx) dx -= L.nx;
                    if (dx < -hx) dx += L.nx;
                    if (dy > hy) dy -= L.ny;
                    if (dy < -hy) dy += L.ny;
                    const float cut = ra + o.w;
                    ok = dx * dx + dy * dy + dz * dz < cut * cut;
                }
                const unsigned m = __ballot_sync(0xffffffffu, ok);
                if (ok) {
                    const int pos = cnt + __popc(m & ((1u << lane) - 1u));
                    if (pos < pt.max_nbr) pt.nbr[(long long)a * pt.max_nbr + pos] = b;
                }
                cnt += __popc(m);
            }
        }
        if (live && lane == 0) {
            pt.nbr_cnt[a] = min(cnt, pt.max_nbr);
            if (cnt > pt.max_nbr) atomicOr(status, ST_NBR_OVERFLOW);
        }
        if (live && lane < 3) pt.Xbuild[3 * a + lane] = pt.X[3 * a + lane];
        __syncwarp();
    }
    if (!live) return;
    const int cnt = pt.nbr_cnt[a];
    for (int m = lane; m < cnt; m += 32) {
        const int b = pt.nbr[(long long)a * pt.max_nbr + m];
        double d[3] = {pt.X[3 * a] - pt.X[3 * b], pt.X[3 * a + 1] - pt.X[3 * b + 1], pt.X[3 * a + 2] - pt.X[3 * b + 2]};
        min_image(L, d);
        const double Rs = pt.R[a] + pt.R[b];
        const double c0 = Rs * Rs - (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const double ma = sphere_mass(pt, a), mb = sphere_mass(pt, b);
        const double meff = pt.fixed[b] ? ma : (pt.fixed[a] ? mb : ma * mb / (ma + mb));
        const float gam = (float)pt.ce * sqrtf((float)(meff * pt.kn));
        const long long e = (long long)a * pt.max_nbr + m;
        pt.pairA[e] = make_float4((float)d[0], (float)d[1], (float)d[2], (float)c0);
        pt.pairB[e] = make_float4((float)(pt.V[3 * a] - pt.V[3 * b]), (float)(pt.V[3 * a + 1] - pt.V[3 * b + 1]),
                                  (float)(pt.V[3 * a + 2] - pt.V[3 * b + 2]), gam);
    }
}

// Contact force on sphere a at centre xa, velocity va, given the centres Xs
// and velocities Vs of all spheres (FP64 throughout; used for the initial
// contact force and by the cooperative fallback).
__device__ void contact_force(const Lat &L, const Parts &pt, int a, const double xa[3], const double va[3],
                              const double *Xs, const double *Vs, double F[3]) {
    F[0] = F[1] = F[2] = 0.0;
    const double ma = sphere_mass(pt, a);
    const double Ra = pt.R[a];
    const float kn = (float)pt.kn, ce = (float)pt.ce;
    const int cnt = pt.nbr_cnt[a];
    for (int m = 0; m < cnt; ++m) {
        const int b = pt.nbr[(long long)a * pt.max_nbr + m];
        double d[3] = {xa[0] - Xs[3 * b], xa[1] - Xs[3 * b + 1], xa[2] - Xs[3 * b + 2]};
        min_image(L, d);
        const double Rs = Ra + pt.R[b];
        const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (!(d2 < Rs * Rs)) continue;
        const double dist = sqrt(d2);
        const double delta = Rs - dist;
        if (!(delta > 0.0) || dist == 0.0) continue;
        const float id = (float)(1.0 / dist);
        const float nx = (float)d[0] * id, ny = (float)d[1] * id, nz = (float)d[2] * id;
        const float vn = (float)(va[0] - Vs[3 * b]) * nx + (float)(va[1] - Vs[3 * b + 1]) * ny +
                         (float)(va[2] - Vs[3 * b + 2]) * nz;
        const double mb = sphere_mass(pt, b);
        const double meff = pt.fixed[b] ? ma : (pt.fixed[a] ? mb : ma * mb / (ma + mb));
        const float fn = kn * (float)delta - ce * sqrtf((float)meff * kn) * vn;
        F[0] += (double)(fn * nx);
        F[1] += (double)(fn * ny);
        F[2] += (double)(fn * nz);
    }
    const float gw = ce * sqrtf((float)ma * kn);
    const float vz = (float)va[2];
    const double lo = Ra - (xa[2] + 0.5);
    if (lo > 0.0) F[2] += (double)(kn * (float)lo - gw * vz);
    const double hi = Ra - ((L.nz - 0.5) - xa[2]);
    if (hi > 0.0) F[2] -= (double)(kn * (float)hi + gw * vz);
}

__global__ void k_contact(const Lat L, const Parts pt) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= pt.np) return;
    double F[3];
    contact_force(L, pt, a, pt.X + 3 * a, pt.V + 3 * a, pt.X, pt.V, F);
    for (int c = 0; c < 3; ++c) pt.Fc[3 * a + c] = F[c];
}

__device__ __forceinline__ void wrap_pos(const Lat &L, double *x) {
    if (x[0] >= L.nx) x[0] -= L.nx;
    if (x[0] < 0.0) x[0] += L.nx;
    if (x[1] >= L.ny) x[1] -= L.ny;
    if (x[1] < 0.0) x[1] += L.ny;
}

__device__ __forceinline__ SFrame make_frame(const double x[3], double R, const double v[3], const double w[3]) {
    SFrame F;
    for (int c = 0; c < 3; ++c) {
        const double b = floor(x[c]);
        F.b[c] = (int)b;
        F.fr[c] = __double2float_rn(x[c] - b);
        F.V[c] = (float)v[c];
        F.W[c] = (float)w[c];
    }
    F.R = __double2float_rn(R);
    F.R2 = __fmul_rn(F.R, F.R);
    F.pad[0] = F.pad[1] = 0.f;
    return F;
}

// End of a step (parity sp) for sphere a: store the new state and its frame,
// flag a sphere that moved max_step in the step (or left the box), and ask
// the next step's neighbour pass for a list rebuild when it drifted
// skin/2 - max_step from where the lists were built.
__device__ __forceinline__ void commit(const Lat &L, const Parts &pt, SFrame *fnext, int a, const double x[3],
                                       const double v[3], const double w[3], const double fc[3], double moved2,
                                       int sp, int *status) {
    double b2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        double dd = x[c] - pt.Xbuild[3 * a + c];
        if (c == 0 && dd > 0.5 * L.nx) dd -= L.nx;
        if (c == 0 && dd < -0.5 * L.nx) dd += L.nx;
        if (c == 1 && dd > 0.5 * L.ny) dd -= L.ny;
        if (c == 1 && dd < -0.5 * L.ny) dd += L.ny;
        b2 += dd * dd;
        pt.X[3 * a + c] = x[c];
        pt.V[3 * a + c] = v[c];
        pt.W[3 * a + c] = w[c];
        pt.Fc[3 * a + c] = fc[c];
    }
    pt.Xf[a] = make_float4((float)x[0], (float)x[1], (float)x[2], (float)pt.R[a]);
    fnext[a] = make_frame(x, pt.R[a], v, w);
    if (!(moved2 < pt.max_step * pt.max_step) || !(x[2] > -0.5 && x[2] < L.nz - 0.5)) atomicOr(status, ST_FAST);
    const double lim = 0.5 * pt.skin - pt.max_step;
    if (!(b2 < lim * lim)) pt.rebuild[sp ^ 1] = 1;
}

__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// All sub-steps of the lattice step of parity sp in one cluster (gridDim.x
// CTAs).  Thread t of CTA c owns spheres a = c T + t + q G (q < kDemKmax,
// G = cluster threads).  The step's neighbour pass has read rebuild[sp], so
// it is cleared here; the commits may set rebuild[sp ^ 1].
__device__ __forceinline__ void dem_cluster_body(const Lat &L, const Parts &pt, SFrame *fnext, const int sp,
                                                 int *status) {
    extern __shared__ float4 dsm[];  // [2][kDemKmax * T][2]: (dx, -), (dv, -)
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int T = blockDim.x, G = gridDim.x * T, cap = kDemKmax * T;
    const int g0 = blockIdx.x * T + threadIdx.x;
    if (g0 == 0) pt.rebuild[sp] = 0;
    const int ns = pt.substeps;
    const float h = 1.f / ns, h2 = 0.5f * h;
    const float kn = (float)pt.kn, ce = (float)pt.ce;
    float3 dx[kDemKmax], dv[kDemKmax], v0[kDemKmax], fa[kDemKmax], fc[kDemKmax];
    float im[kDemKmax], Rf[kDemKmax], Llo[kDemKmax], Lhi[kDemKmax], gw[kDemKmax];
    int nc[kDemKmax];
    bool fx[kDemKmax];
#pragma unroll
    for (int q = 0; q < kDemKmax; ++q) {
        const int a = g0 + q * G;
        if (a >= pt.np) break;
        const double m = sphere_mass(pt, a), R = pt.R[a], z0 = pt.X[3 * a + 2];
        fx[q] = pt.fixed[a] != 0;
        const double ia = 1.0 / m;
        im[q] = (float)ia;
        Rf[q] = (float)R;
        fa[q] = make_float3((float)((pt.Fh[3 * a] + pt.Fx[3 * a]) * ia), (float)((pt.Fh[3 * a + 1] + pt.Fx[3 * a + 1]) * ia),
                            (float)((pt.Fh[3 * a + 2] + pt.Fx[3 * a + 2]) * ia));
        fc[q] = make_float3((float)pt.Fc[3 * a], (float)pt.Fc[3 * a + 1], (float)pt.Fc[3 * a + 2]);
        v0[q] = make_float3((float)pt.V[3 * a], (float)pt.V[3 * a + 1], (float)pt.V[3 * a + 2]);
        Llo[q] = (float)(R - (z0 + 0.5));
        Lhi[q] = (float)(R - ((L.nz - 0.5) - z0));
        gw[q] = ce * sqrtf((float)m * kn);
        nc[q] = pt.nbr_cnt[a];
        dx[q] = make_float3(0.f, 0.f, 0.f);
        dv[q] = make_float3(0.f, 0.f, 0.f);
    }
    cluster_barrier();  // every CTA of the cluster is running before shared memory is shared
    for (int s = 0; s < ns; ++s) {
        float4 *buf = dsm + (size_t)((s + 1) & 1) * cap * 2;
#pragma unroll
        for (int q = 0; q < kDemKmax; ++q) {
            const int a = g0 + q * G;
            if (a >= pt.np) break;
            if (!fx[q]) {  // half kick
                dv[q].x += (fa[q].x + fc[q].x * im[q]) * h2;
                dv[q].y += (fa[q].y + fc[q].y * im[q]) * h2;
                dv[q].z += (fa[q].z + fc[q].z * im[q]) * h2;
            }
            dx[q].x += (v0[q].x + dv[q].x) * h;
            dx[q].y += (v0[q].y + dv[q].y) * h;
            dx[q].z += (v0[q].z + dv[q].z) * h;
            float4 *me = buf + (size_t)(q * T + threadIdx.x) * 2;
            me[0] = make_float4(dx[q].x, dx[q].y, dx[q].z, 0.f);
            me[1] = make_float4(dv[q].x, dv[q].y, dv[q].z, 0.f);
        }
        cluster_barrier();
#pragma unroll
        for (int q = 0; q < kDemKmax; ++q) {
            const int a = g0 + q * G;
            if (a >= pt.np) break;
            if (fx[q]) continue;
            float3 F = make_float3(0.f, 0.f, 0.f);
            // neighbours in groups of kNbrGroup: every load of a group is
            // issued before any of its arithmetic; the sum keeps list order
            constexpr int kNbrGroup = 4;
            for (int m0 = 0; m0 < nc[q]; m0 += kNbrGroup) {
                float4 A[kNbrGroup], Bv[kNbrGroup], ox[kNbrGroup], ov[kNbrGroup];
                float Rb[kNbrGroup];
#pragma unroll
                for (int u = 0; u < kNbrGroup; ++u) {
                    if (m0 + u >= nc[q]) break;
                    const long long e = (long long)a * pt.max_nbr + m0 + u;
                    const int b = __ldg(pt.nbr + e);
                    A[u] = __ldg(pt.pairA + e);
                    Bv[u] = __ldg(pt.pairB + e);
                    Rb[u] = __ldg(&pt.Xf[b].w);
                    const int qb = b / G, rb = b - qb * G, cb = rb / T, tb = rb - cb * T;
                    const float4 *o = cluster.map_shared_rank(buf + (size_t)(qb * T + tb) * 2, cb);
                    ox[u] = o[0];
                    ov[u] = o[1];
                }
#pragma unroll
                for (int u = 0; u < kNbrGroup; ++u) {
                    if (m0 + u >= nc[q]) break;
                    const float Dx = dx[q].x - ox[u].x, Dy = dx[q].y - ox[u].y, Dz = dx[q].z - ox[u].z;
                    const float c =
                        A[u].w - 2.f * (A[u].x * Dx + A[u].y * Dy + A[u].z * Dz) - (Dx * Dx + Dy * Dy + Dz * Dz);
                    if (!(c > 0.f)) continue;
                    const float ex = A[u].x + Dx, ey = A[u].y + Dy, ez = A[u].z + Dz;
                    const float dist = sqrtf(ex * ex + ey * ey + ez * ez);
                    const float Rs = Rf[q] + Rb[u];
                    const float delta = c / (Rs + dist);
                    const float id = 1.f / dist;
                    const float nx = ex * id, ny = ey * id, nz = ez * id;
                    const float vn = (Bv[u].x + dv[q].x - ov[u].x) * nx + (Bv[u].y + dv[q].y - ov[u].y) * ny +
                                     (Bv[u].z + dv[q].z - ov[u].z) * nz;
                    const float fn = kn * delta - Bv[u].w * vn;
                    F.x += fn * nx;
                    F.y += fn * ny;
                    F.z += fn * nz;
                }
            }
            const float vz = v0[q].z + dv[q].z;
            const float lo = Llo[q] - dx[q].z;
            if (lo > 0.f) F.z += kn * lo - gw[q] * vz;
            const float hi = Lhi[q] + dx[q].z;
            if (hi > 0.f) F.z -= kn * hi + gw[q] * vz;
            fc[q] = F;
            dv[q].x += (fa[q].x + F.x * im[q]) * h2;
            dv[q].y += (fa[q].y + F.y * im[q]) * h2;
            dv[q].z += (fa[q].z + F.z * im[q]) * h2;
        }
    }
    cluster_barrier();  // no CTA leaves while another may still read its shared memory
#pragma unroll
    for (int q = 0; q < kDemKmax; ++q) {
        const int a = g0 + q * G;
        if (a >= pt.np) break;
        double x[3] = {pt.X[3 * a] + (double)dx[q].x, pt.X[3 * a + 1] + (double)dx[q].y, pt.X[3 * a + 2] + (double)dx[q].z};
        wrap_pos(L, x);
        double v[3] = {pt.V[3 * a], pt.V[3 * a + 1], pt.V[3 * a + 2]};
        double w[3] = {pt.W[3 * a], pt.W[3 * a + 1], pt.W[3 * a + 2]};
        if (!fx[q]) {
            const double m = sphere_mass(pt, a);
            const double iI = 1.0 / (0.4 * m * pt.R[a] * pt.R[a]);
            v[0] += (double)dv[q].x;
            v[1] += (double)dv[q].y;
            v[2] += (double)dv[q].z;
            for (int c = 0; c < 3; ++c) w[c] += (pt.Th[3 * a + c] + pt.Tx[3 * a + c]) * iI;
        }
        const double f3[3] = {(double)fc[q].x, (double)fc[q].y, (double)fc[q].z};
        const double moved2 = (double)(dx[q].x * dx[q].x + dx[q].y * dx[q].y + dx[q].z * dx[q].z);
        commit(L, pt, fnext, a, x, v, w, f3, moved2, sp, status);
    }
}

__global__ void __launch_bounds__(256) k_neighbours(const Lat L, const Parts pt, const int sp, const int force,
                                                    int *__restrict__ status) {
    neighbours_body(L, pt, sp, force, status);
}

__global__ void __launch_bounds__(kDemThreads, 1) k_dem_cluster(const Lat L, const Parts pt, SFrame *fnext,
                                                                const int sp, int *status) {
    dem_cluster_body(L, pt, fnext, sp, status);
}

// Batched forms: instance blockIdx.y.
__global__ void __launch_bounds__(256) k_neighbours_b(const Inst *__restrict__ I, const int sp) {
    const Inst &a = I[blockIdx.y];
    if ((int)(blockIdx.x * (blockDim.x >> 5)) >= a.pt.np) return;
    neighbours_body(a.L, a.pt, sp, 0, a.status);
}

__global__ void __launch_bounds__(kDemThreads, 1) k_dem_cluster_b(const Inst *__restrict__ I, const int sp) {
    const Inst &a = I[blockIdx.y];
    if (a.pt.np == 0) return;  // the whole cluster (one instance) leaves together
    dem_cluster_body(a.L, a.pt, a.pt.frame[sp ^ 1], sp, a.status);
}

static size_t dem_cluster_smem() { return (size_t)2 * kDemKmax * kDemThreads * 2 * sizeof(float4); }

// ---- fallback: cooperative grid with a bounded software barrier ------------

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }

// Returns false (and sets the timeout status) if the other blocks did not
// arrive within ~2^22 polls, or if another block already gave up.
__device__ bool grid_barrier(unsigned *bar, unsigned target, int *status) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        int good = 1;
        long long it = 0;
        while (ld_acquire(bar) < target) {
            if (++it > (1ll << 22) || (ld_volatile(status) & ST_TIMEOUT)) {
                atomicOr(status, ST_TIMEOUT);
                good = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// FP64 velocity Verlet with centres and half-step velocities exchanged
// through global memory (any number of spheres).  pt.V holds the full-step
// velocity between sub-steps; pt.X stays the start-of-step centre until the
// commit.
__global__ void __launch_bounds__(128) k_dem(const Lat L, const Parts pt, SFrame *fnext, const int sp,
                                             unsigned *bar, int *status) {
    const int G = gridDim.x * blockDim.x;
    const int g0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (g0 == 0) pt.rebuild[sp] = 0;
    const int ns = pt.substeps;
    const double h = 1.0 / ns;
    unsigned target = 0;
    for (int s = 0; s < ns; ++s) {
        const double *Xc = s == 0 ? pt.X : pt.Xb[s & 1];
        double *Xn = pt.Xb[(s + 1) & 1], *Vn = pt.Vh[(s + 1) & 1];
        for (int a = g0; a < pt.np; a += G) {
            const double k = pt.fixed[a] ? 0.0 : h / (2.0 * sphere_mass(pt, a));
            double x[3];
            for (int c = 0; c < 3; ++c) {
                const double vh = pt.V[3 * a + c] + (pt.Fh[3 * a + c] + pt.Fx[3 * a + c] + pt.Fc[3 * a + c]) * k;
                Vn[3 * a + c] = vh;
                x[c] = Xc[3 * a + c] + vh * h;
            }
            wrap_pos(L, x);
            for (int c = 0; c < 3; ++c) Xn[3 * a + c] = x[c];
        }
        target += gridDim.x;
        if (!grid_barrier(bar, target, status)) return;
        for (int a = g0; a < pt.np; a += G) {
            if (pt.fixed[a]) continue;
            double F[3];
            contact_force(L, pt, a, Xn + 3 * a, Vn + 3 * a, Xn, Vn, F);
            const double k = h / (2.0 * sphere_mass(pt, a));
            for (int c = 0; c < 3; ++c) {
                pt.Fc[3 * a + c] = F[c];
                pt.V[3 * a + c] = Vn[3 * a + c] + (pt.Fh[3 * a + c] + pt.Fx[3 * a + c] + F[c]) * k;
            }
        }
    }
    const double *Xe = pt.Xb[ns & 1];
    for (int a = g0; a < pt.np; a += G) {
        double x[3], v[3], w[3], f3[3], moved2 = 0.0;
        const double iI = pt.fixed[a] ? 0.0 : 1.0 / (0.4 * sphere_mass(pt, a) * pt.R[a] * pt.R[a]);
        for (int c = 0; c < 3; ++c) {
            x[c] = Xe[3 * a + c];
            v[c] = pt.V[3 * a + c];
            w[c] = pt.W[3 * a + c] + (pt.Th[3 * a + c] + pt.Tx[3 * a + c]) * iI;
            f3[c] = pt.Fc[3 * a + c];
            double dd = x[c] - pt.X[3 * a + c];
            if (c == 0 && dd > 0.5 * L.nx) dd -= L.nx;
            if (c == 0 && dd < -0.5 * L.nx) dd += L.nx;
            if (c == 1 && dd > 0.5 * L.ny) dd -= L.ny;
            if (c == 1 && dd < -0.5 * L.ny) dd += L.ny;
            moved2 += dd * dd;
        }
        commit(L, pt, fnext, a, x, v, w, f3, moved2, sp, status);
    }
}

int launch_neighbours(lbm_s *h, int force, cudaStream_t stream) {
    const int blocks = (h->pt.np * 32 + 255) / 256;
    k_neighbours<<<blocks, 256, 0, stream ? stream : h->stream>>>(h->L, h->pt, (int)(h->steps & 1), force,
                                                                 h->status);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int launch_contact(lbm_s *h) {
    k_contact<<<(h->pt.np + 127) / 128, 128, 0, h->stream>>>(h->L, h->pt);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int dem_max_blocks(int threads, int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_dem, threads, 0) == cudaSuccess ? LBM_OK
                                                                                                         : LBM_ERR_CUDA;
}

// Largest cluster (16, else 8) that can run k_dem_cluster; 0 if none, or if
// max_particles does not fit its registers.
int dem_cluster_setup(int max_particles, bool small) {
    if (cudaFuncSetAttribute(k_dem_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dem_cluster_smem()) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    // one simulation: the widest cluster (16 or 8 CTAs: measured equal at
    // 2000 spheres, narrower ones slower); a batch: the narrowest cluster
    // that gives every sphere its own thread, so that the members' clusters
    // run side by side
    const std::vector<int> sizes = small ? std::vector<int>{1, 2, 4, 8, 16} : std::vector<int>{16, 8};
    for (int cl : sizes) {
        if ((long long)cl * kDemThreads * kDemKmax < max_particles) continue;
        if (small && (long long)cl * kDemThreads < max_particles && cl < 16) continue;
        if (cl > 8 && cudaFuncSetAttribute(k_dem_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                          cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(cl);
        cfg.blockDim = dim3(kDemThreads);
        cfg.dynamicSmemBytes = dem_cluster_smem();
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_dem_cluster, &cfg) == cudaSuccess && n >= 1) return cl;
        cudaGetLastError();
    }
    return 0;
}

int dem_cluster_setup_batch(int cl) {
    if (cudaFuncSetAttribute(k_dem_cluster_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dem_cluster_smem()) !=
            cudaSuccess ||
        (cl > 8 && cudaFuncSetAttribute(k_dem_cluster_b, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                       cudaSuccess)) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

int launch_neighbours_batch(const lbm_batch_s *b, int sp) {
    if (b->max_np == 0) return LBM_OK;
    const int blocks = (b->max_np * 32 + 255) / 256;
    k_neighbours_b<<<dim3(blocks, b->n), 256, 0, b->stream>>>(b->dinst, sp);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

// One cluster of b->dem_cluster CTAs per instance.
int launch_dem_batch(const lbm_batch_s *b, int sp) {
    if (b->max_np == 0) return LBM_OK;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = b->dem_cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(b->dem_cluster, b->n);
    cfg.blockDim = dim3(kDemThreads);
    cfg.dynamicSmemBytes = dem_cluster_smem();
    cfg.stream = b->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const Inst *I = b->dinst;
    return cudaLaunchKernelEx(&cfg, k_dem_cluster_b, I, sp) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int launch_dem(lbm_s *h) {
    Lat L = h->L;
    Parts pt = h->pt;
    int *status = h->status;
    SFrame *fnext = h->pt.frame[(h->steps + 1) & 1];
    const int sp = (int)(h->steps & 1);
    if (h->dem_cluster > 0) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = h->dem_cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(h->dem_cluster);
        cfg.blockDim = dim3(kDemThreads);
        cfg.dynamicSmemBytes = dem_cluster_smem();
        cfg.stream = h->stream;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_dem_cluster, L, pt, fnext, sp, status) == cudaSuccess ? LBM_OK
                                                                                                 : LBM_ERR_CUDA;
    }
    if (cudaMemsetAsync(h->bar, 0, sizeof(unsigned), h->stream) != cudaSuccess) return LBM_ERR_CUDA;
    int blocks = (h->pt.np + h->dem_threads - 1) / h->dem_threads;
    if (blocks > h->dem_blocks) blocks = h->dem_blocks;
    if (blocks < 1) blocks = 1;
    unsigned *bar = h->bar;
    void *args[] = {&L, &pt, &fnext, (void *)&sp, &bar, &status};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_dem, dim3(blocks), dim3(h->dem_threads), args, 0,
                                                h->stream);
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

}  // namespace lbm
