// Sphere DEM (Sect. 2.1): linear spring-dashpot normal contact (Eq. 1) between
// spheres and with the z walls, velocity Verlet in dem_substeps sub-steps per
// lattice step with the hydrodynamic (and external) load held constant.
//
// Reading of Eq. (1): f^n = k_n delta - gamma_n v_n for an overlap delta > 0
// (unclipped), gamma_n = -2 ln(e) sqrt(m_eff k_n) / sqrt(pi^2 + ln(e)^2), which
// gives a normal restitution of exactly e.  A fixed sphere moves with its
// prescribed velocity and acts with infinite mass.
//
// Precision: centres, velocities and spins are integrated in FP64 (their
// drift needs it); the contact decision and the overlap delta are FP64 (delta
// is a small difference of O(R) numbers), the force law is FP32 and the
// per-sphere sums FP64.  FP64 throughput is low on this GPU, so the O(P^2)
// neighbour search runs in FP32 on a float copy of the centres with a skin of
// one lattice unit; a sphere that moves half a skin in one step raises the
// geometry error.
//
// Sub-steps need all centres of the previous sub-step.  One thread-block
// cluster runs all of them: each thread keeps its spheres in registers, the
// new centres and half-step velocities go through distributed shared memory,
// and a hardware cluster barrier (release / acquire) separates drift and
// force.
// Too many spheres for one cluster fall back to a cooperative launch with a
// bounded software grid barrier.
#include <cooperative_groups.h>

#include "lbm_internal.cuh"

namespace lbm {

constexpr double kPi = 3.14159265358979323846;
constexpr int kDemKmax = 4;       // spheres per thread held in registers
constexpr int kDemThreads = 256;  // threads per CTA of the cluster kernel

__device__ __forceinline__ double sphere_mass(const Parts &pt, int a) {
    const double r = pt.R[a];
    return pt.rho_s * (4.0 / 3.0) * kPi * r * r * r;
}

// Neighbour list of sphere a: every b != a with |X_a - X_b| < R_a + R_b + skin
// (minimum image in x, y), in increasing b.  One warp per sphere; centres are
// staged through shared memory in tiles.
constexpr int kNbrTile = 1024;

__global__ void __launch_bounds__(256) k_neighbours(const Lat L, const Parts pt, int *__restrict__ status) {
    __shared__ float4 tile[kNbrTile];
    const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const bool live = a < pt.np;
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
}

// Contact force on sphere a at centre xa, velocity va, given the centres Xs
// and velocities Vs of all spheres (FP64 arrays).
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
        if (d[0] > 0.5 * L.nx) d[0] -= L.nx;
        if (d[0] < -0.5 * L.nx) d[0] += L.nx;
        if (d[1] > 0.5 * L.ny) d[1] -= L.ny;
        if (d[1] < -0.5 * L.ny) d[1] += L.ny;
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

// After the last sub-step: commit the centres (and their FP32 copy) and flag
// a sphere that moved half a skin in the step or left the box.
__device__ __forceinline__ void commit(const Lat &L, const Parts &pt, int a, const double x[3], int *status) {
    double m2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        double dd = x[c] - pt.Xgeo[3 * a + c];
        const double n = c == 0 ? L.nx : (c == 1 ? L.ny : 1e300);
        if (dd > 0.5 * n) dd -= n;
        if (dd < -0.5 * n) dd += n;
        m2 += dd * dd;
        pt.X[3 * a + c] = x[c];
    }
    pt.Xf[a] = make_float4((float)x[0], (float)x[1], (float)x[2], (float)pt.R[a]);
    if (!(m2 < 0.25 * pt.skin * pt.skin) || !(x[2] > -0.5 && x[2] < L.nz - 0.5)) atomicOr(status, ST_FAST);
}

__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// All sub-steps of one lattice step in one cluster (gridDim.x CTAs).  Thread
// t of CTA c owns spheres a = c T + t + q G (q < kDemKmax, G = cluster
// threads) and keeps their state in registers; after each drift it publishes
// centre and half-step velocity in its CTA's shared memory (double-buffered
// by sub-step parity), where the force phase of every CTA reads them through
// distributed shared memory.
__global__ void __launch_bounds__(kDemThreads, 1) k_dem_cluster(const Lat L, const Parts pt, int *status) {
    extern __shared__ double dsm[];  // [2][kDemKmax * T][6]: x, y, z, vx, vy, vz
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int T = blockDim.x, G = gridDim.x * T, cap = kDemKmax * T;
    const int g0 = blockIdx.x * T + threadIdx.x;
    const int ns = pt.substeps;
    const double h = 1.0 / ns;
    const float kn = (float)pt.kn, ce = (float)pt.ce;
    double x[kDemKmax][3], v[kDemKmax][3], w[kDemKmax][3], F0[kDemKmax][3], T0[kDemKmax][3], fc[kDemKmax][3];
    double km[kDemKmax], kI[kDemKmax], Ra[kDemKmax], ma[kDemKmax];
    int nc[kDemKmax];
    bool fx[kDemKmax];
#pragma unroll
    for (int q = 0; q < kDemKmax; ++q) {
        const int a = g0 + q * G;
        if (a >= pt.np) break;
        Ra[q] = pt.R[a];
        ma[q] = sphere_mass(pt, a);
        fx[q] = pt.fixed[a] != 0;
        km[q] = fx[q] ? 0.0 : h / (2.0 * ma[q]);
        kI[q] = fx[q] ? 0.0 : h / (0.4 * ma[q] * Ra[q] * Ra[q]);
        nc[q] = pt.nbr_cnt[a];
        for (int c = 0; c < 3; ++c) {
            x[q][c] = pt.X[3 * a + c];
            v[q][c] = pt.V[3 * a + c];
            w[q][c] = pt.W[3 * a + c];
            F0[q][c] = pt.Fh[3 * a + c] + pt.Fx[3 * a + c];
            T0[q][c] = pt.Th[3 * a + c] + pt.Tx[3 * a + c];
            fc[q][c] = pt.Fc[3 * a + c];
        }
    }
    cluster_barrier();  // every CTA of the cluster is running before shared memory is shared
    for (int s = 0; s < ns; ++s) {
        double *buf = dsm + (size_t)((s + 1) & 1) * cap * 6;
#pragma unroll
        for (int q = 0; q < kDemKmax; ++q) {
            const int a = g0 + q * G;
            if (a >= pt.np) break;
            for (int c = 0; c < 3; ++c) {
                v[q][c] += (F0[q][c] + fc[q][c]) * km[q];  // half kick (fixed: km = 0)
                x[q][c] += v[q][c] * h;
            }
            wrap_pos(L, x[q]);
            double *me = buf + (size_t)(q * T + threadIdx.x) * 6;
            for (int c = 0; c < 3; ++c) {
                me[c] = x[q][c];
                me[3 + c] = v[q][c];
            }
        }
        cluster_barrier();
#pragma unroll
        for (int q = 0; q < kDemKmax; ++q) {
            const int a = g0 + q * G;
            if (a >= pt.np) break;
            if (fx[q]) continue;
            double F[3] = {0.0, 0.0, 0.0};
            for (int m = 0; m < nc[q]; ++m) {
                const int b = __ldg(pt.nbr + (long long)a * pt.max_nbr + m);
                const int qb = b / G, rb = b - qb * G, cb = rb / T, tb = rb - cb * T;
                const double *o = cluster.map_shared_rank(buf + (size_t)(qb * T + tb) * 6, cb);
                double d[3] = {x[q][0] - o[0], x[q][1] - o[1], x[q][2] - o[2]};
                if (d[0] > 0.5 * L.nx) d[0] -= L.nx;
                if (d[0] < -0.5 * L.nx) d[0] += L.nx;
                if (d[1] > 0.5 * L.ny) d[1] -= L.ny;
                if (d[1] < -0.5 * L.ny) d[1] += L.ny;
                const double Rb = __ldg(pt.R + b);
                const double Rs = Ra[q] + Rb;
                const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (!(d2 < Rs * Rs)) continue;
                const double dist = sqrt(d2);
                const double delta = Rs - dist;
                if (!(delta > 0.0) || dist == 0.0) continue;
                const float id = (float)(1.0 / dist);
                const float nx = (float)d[0] * id, ny = (float)d[1] * id, nz = (float)d[2] * id;
                const float vn = (float)(v[q][0] - o[3]) * nx + (float)(v[q][1] - o[4]) * ny +
                                 (float)(v[q][2] - o[5]) * nz;
                const double mb = pt.rho_s * (4.0 / 3.0) * kPi * Rb * Rb * Rb;
                const double meff = __ldg(pt.fixed + b) ? ma[q] : ma[q] * mb / (ma[q] + mb);
                const float fn = kn * (float)delta - ce * sqrtf((float)meff * kn) * vn;
                F[0] += (double)(fn * nx);
                F[1] += (double)(fn * ny);
                F[2] += (double)(fn * nz);
            }
            const float gw = ce * sqrtf((float)ma[q] * kn);
            const float vz = (float)v[q][2];
            const double lo = Ra[q] - (x[q][2] + 0.5);
            if (lo > 0.0) F[2] += (double)(kn * (float)lo - gw * vz);
            const double hi = Ra[q] - ((L.nz - 0.5) - x[q][2]);
            if (hi > 0.0) F[2] -= (double)(kn * (float)hi + gw * vz);
            for (int c = 0; c < 3; ++c) {
                fc[q][c] = F[c];
                v[q][c] += (F0[q][c] + F[c]) * km[q];
                w[q][c] += T0[q][c] * kI[q];
            }
        }
    }
    cluster_barrier();  // no CTA leaves while another may still read its shared memory
#pragma unroll
    for (int q = 0; q < kDemKmax; ++q) {
        const int a = g0 + q * G;
        if (a >= pt.np) break;
        for (int c = 0; c < 3; ++c) {
            pt.V[3 * a + c] = v[q][c];
            pt.W[3 * a + c] = w[q][c];
            pt.Fc[3 * a + c] = fc[q][c];
        }
        commit(L, pt, a, x[q], status);
    }
}

static size_t dem_cluster_smem() { return (size_t)2 * kDemKmax * kDemThreads * 6 * sizeof(double); }

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

__global__ void __launch_bounds__(128) k_dem(const Lat L, const Parts pt, unsigned *bar, int *status) {
    const int G = gridDim.x * blockDim.x;
    const int g0 = blockIdx.x * blockDim.x + threadIdx.x;
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
            const double m = sphere_mass(pt, a);
            const double k = h / (2.0 * m), kI = h / (0.4 * m * pt.R[a] * pt.R[a]);
            for (int c = 0; c < 3; ++c) {
                pt.V[3 * a + c] = Vn[3 * a + c] + (pt.Fh[3 * a + c] + pt.Fx[3 * a + c] + F[c]) * k;
                pt.W[3 * a + c] += (pt.Th[3 * a + c] + pt.Tx[3 * a + c]) * kI;
                pt.Fc[3 * a + c] = F[c];
            }
        }
    }
    const double *Xe = pt.Xb[ns & 1];
    for (int a = g0; a < pt.np; a += G) {
        double x[3] = {Xe[3 * a], Xe[3 * a + 1], Xe[3 * a + 2]};
        commit(L, pt, a, x, status);
    }
}

int launch_neighbours(lbm_s *h) {
    const int blocks = (h->pt.np * 32 + 255) / 256;
    k_neighbours<<<blocks, 256, 0, h->stream>>>(h->L, h->pt, h->status);
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
int dem_cluster_setup(int max_particles) {
    for (int cl : {16, 8}) {
        if ((long long)cl * kDemThreads * kDemKmax < max_particles) continue;
        if (cudaFuncSetAttribute(k_dem_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)dem_cluster_smem()) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
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

int launch_dem(lbm_s *h) {
    Lat L = h->L;
    Parts pt = h->pt;
    int *status = h->status;
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
        return cudaLaunchKernelEx(&cfg, k_dem_cluster, L, pt, status) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
    }
    if (cudaMemsetAsync(h->bar, 0, sizeof(unsigned), h->stream) != cudaSuccess) return LBM_ERR_CUDA;
    int blocks = (h->pt.np + h->dem_threads - 1) / h->dem_threads;
    if (blocks > h->dem_blocks) blocks = h->dem_blocks;
    if (blocks < 1) blocks = 1;
    unsigned *bar = h->bar;
    void *args[] = {&L, &pt, &bar, &status};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_dem, dim3(blocks), dim3(h->dem_threads), args, 0,
                                                h->stream);
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

}  // namespace lbm
