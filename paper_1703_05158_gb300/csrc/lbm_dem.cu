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
// Tangential contact law (Eqs. 2, 3; on when k_t > 0 and mu > 0, the
// template argument FRIC of the cluster kernel): the readings of the oracle
// (contact point at the middle of the overlap, v^r = v_a - v_b - ((R_a -
// delta/2) Om_a + (R_b - delta/2) Om_b) x n, f_t = -k_t delta_t - gamma_t v_t
// capped at mu max(f^n, 0) along -v_t with delta_t reset to -f_t / k_t,
// delta_t turned into the tangent plane and advanced by v_t h every
// sub-step, reset when the contact opens; walls move with their lattice
// velocity).  Each list entry keeps its delta_t (FP32) in tdisp, valid when
// its bit of the sphere's tmask is set; a list rebuild carries the state of
// the pairs that stay listed.  The spin then takes half kicks with the
// contact torque like the velocity (dOm in FP32 per sub-step, published with
// dx and dv).
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
// with friction each sphere holds more state: fewer spheres per thread
__host__ __device__ constexpr int dem_kmax(bool fric) { return fric ? 2 : kDemKmax; }
// Threads per CTA of the cluster kernel.  128 (a 16-CTA cluster holds
// 2048 spheres at one per thread, 4096 with friction at two) rather than
// 256: the DEM phase of 2000 spheres 0.053 -> 0.048 ms, with friction
// 0.062 -> 0.054 ms, the batched sweep unchanged.
#ifndef LBM_DEM_THREADS
#define LBM_DEM_THREADS 128
#endif
constexpr int kDemThreads = LBM_DEM_THREADS;

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
// shared memory); then compute, for the entries that can touch within the
// step (compacted in list order), the pair constants for the current
// centres and velocities:
//   pairA = (d0, c0),  d0 = X_a - X_b (minimum image), c0 = (R_a+R_b)^2 - |d0|^2
//   pairB = (V_a - V_b, gamma_n),  pairBM = (b, list position)
constexpr int kNbrTile = 1024;

constexpr int kMaxNbrFric = 64;  // list length the 64-bit contact mask covers

__device__ __forceinline__ void neighbours_body(const Lat &L, const Parts &pt, const int sp, const int force,
                                                int *__restrict__ status) {
    __shared__ float4 tile[kNbrTile];
    __shared__ int oid[8][kMaxNbrFric];     // with friction: the old list of each warp's sphere
    __shared__ float4 odisp[8][kMaxNbrFric];  // and the tangential displacement of its open contacts
    const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, wid = (threadIdx.x >> 5) & 7;
    const bool live = a < pt.np;
    const bool rebuild = force || *(volatile int *)(pt.rebuild + sp) != 0;
    if (rebuild) {
        int ocnt = 0;
        unsigned long long omask = 0ull;
        if (pt.fric && !force && live) {  // a forced rebuild starts every contact afresh
            ocnt = min(pt.nbr_cnt[a], min(pt.max_nbr, kMaxNbrFric));
            omask = pt.tmask[a];
            for (int m = lane; m < ocnt; m += 32) {
                const long long e = (long long)a * pt.max_nbr + m;
                oid[wid][m] = pt.nbr[e];
                odisp[wid][m] = (omask >> m) & 1ull ? pt.tdisp[e] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncwarp();
        }
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
        if (pt.fric && live) {  // the open contacts of pairs still listed keep their state
            const int ncnt = min(cnt, min(pt.max_nbr, kMaxNbrFric));
            unsigned long long nmask = 0ull;
            for (int r = 0; r * 32 < ncnt; ++r) {
                const int pos = r * 32 + lane;
                bool hit = false;
                if (pos < ncnt) {
                    const long long e = (long long)a * pt.max_nbr + pos;
                    const int b = pt.nbr[e];
                    for (int m = 0; m < ocnt; ++m)
                        if (oid[wid][m] == b) {
                            hit = (omask >> m) & 1ull;
                            if (hit) pt.tdisp[e] = odisp[wid][m];
                            break;
                        }
                }
                nmask |= (unsigned long long)__ballot_sync(0xffffffffu, hit) << (32 * r);
            }
            if (lane == 0) pt.tmask[a] = nmask;
            __syncwarp();
        }
    }
    if (!live) return;
    // the step's contact candidates: listed pairs whose gap can close within
    // the step (each sphere moves less than max_step, so pairs further apart
    // than R_a + R_b + 2 max_step cannot touch, nor did they touch at the end
    // of the last step), compacted in list order with their list position
    const int cnt = pt.nbr_cnt[a];
    const double reach = 2.0 * pt.max_step + 1e-3;
    int nact = 0;
    for (int m0 = 0; m0 < cnt; m0 += 32) {
        const int m = m0 + lane;
        bool act = false;
        int b = 0;
        double d[3] = {0.0, 0.0, 0.0}, Rs = 0.0, d2 = 0.0;
        if (m < cnt) {
            b = pt.nbr[(long long)a * pt.max_nbr + m];
            d[0] = pt.X[3 * a] - pt.X[3 * b];
            d[1] = pt.X[3 * a + 1] - pt.X[3 * b + 1];
            d[2] = pt.X[3 * a + 2] - pt.X[3 * b + 2];
            min_image(L, d);
            Rs = pt.R[a] + pt.R[b];
            d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            act = d2 < (Rs + reach) * (Rs + reach);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, act);
        if (act) {
            const double c0 = Rs * Rs - d2;
            const double ma = sphere_mass(pt, a), mb = sphere_mass(pt, b);
            const double meff = pt.fixed[b] ? ma : (pt.fixed[a] ? mb : ma * mb / (ma + mb));
            const float gam = (float)pt.ce * sqrtf((float)(meff * pt.kn));
            const long long e = (long long)a * pt.max_nbr + nact + __popc(bal & ((1u << lane) - 1u));
            pt.pairA[e] = make_float4((float)d[0], (float)d[1], (float)d[2], (float)c0);
            pt.pairB[e] = make_float4((float)(pt.V[3 * a] - pt.V[3 * b]), (float)(pt.V[3 * a + 1] - pt.V[3 * b + 1]),
                                      (float)(pt.V[3 * a + 2] - pt.V[3 * b + 2]), gam);
            pt.pairBM[e] = make_int2(b, m);
            if (pt.fric)
                pt.pairC[e] = make_float4((float)pt.W[3 * b], (float)pt.W[3 * b + 1], (float)pt.W[3 * b + 2],
                                          (float)pt.ct * sqrtf((float)(meff * pt.kt)));
        }
        nact += __popc(bal);
    }
    if (lane == 0) pt.nact[a] = nact;
}

// Tangential force of one contact (Eqs. 2, 3), FP64, delta_t = 0 (a contact
// as it opens): the trial force -gamma_t v_t, capped at mu max(f^n, 0) along
// -v_t.  Adds it to F and its moment (-l n) x f_t to T.
__device__ void open_contact_friction(const Parts &pt, const double n[3], const double vr[3], double fn, double gt,
                                      double l, double F[3], double T[3]) {
    const double vrn = vr[0] * n[0] + vr[1] * n[1] + vr[2] * n[2];
    double vt[3], ft[3], t2 = 0.0, v2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        vt[c] = vr[c] - vrn * n[c];
        ft[c] = -gt * vt[c];
        t2 += ft[c] * ft[c];
        v2 += vt[c] * vt[c];
    }
    const double cap = pt.mu * (fn > 0.0 ? fn : 0.0);
    if (t2 > cap * cap)  // t2 > 0 implies v_t != 0
        for (int c = 0; c < 3; ++c) ft[c] = -cap * vt[c] / sqrt(v2);
    for (int c = 0; c < 3; ++c) F[c] += ft[c];
    T[0] += -l * (n[1] * ft[2] - n[2] * ft[1]);
    T[1] += -l * (n[2] * ft[0] - n[0] * ft[2]);
    T[2] += -l * (n[0] * ft[1] - n[1] * ft[0]);
}

// Contact force (and, with friction, torque) on sphere a at centre xa,
// velocity va, spin wa, given the centres Xs, velocities Vs and spins Ws of
// all spheres (FP64 throughout; used for the initial contact force, where
// every contact is new, and by the cooperative fallback, which runs without
// friction).
__device__ void contact_force(const Lat &L, const Parts &pt, int a, const double xa[3], const double va[3],
                              const double *Xs, const double *Vs, double F[3], const double *wa = nullptr,
                              const double *Ws = nullptr, double *T = nullptr) {
    F[0] = F[1] = F[2] = 0.0;
    const bool fric = pt.fric && T;
    if (fric) T[0] = T[1] = T[2] = 0.0;
    const double ma = sphere_mass(pt, a);
    const double Ra = pt.R[a];
    const float kn = (float)pt.kn, ce = (float)pt.ce;
    const int cnt = pt.nbr_cnt[a];
    for (int m = 0; m < cnt; ++m) {
        const int b = pt.nbr[(long long)a * pt.max_nbr + m];
        // other blocks of the cooperative fallback write Xs / Vs within the
        // kernel: read them through L2 (__ldcg), never from a stale L1 line
        const double xb[3] = {__ldcg(Xs + 3 * b), __ldcg(Xs + 3 * b + 1), __ldcg(Xs + 3 * b + 2)};
        const double vb[3] = {__ldcg(Vs + 3 * b), __ldcg(Vs + 3 * b + 1), __ldcg(Vs + 3 * b + 2)};
        double d[3] = {xa[0] - xb[0], xa[1] - xb[1], xa[2] - xb[2]};
        min_image(L, d);
        const double Rs = Ra + pt.R[b];
        const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (!(d2 < Rs * Rs)) continue;
        const double dist = sqrt(d2);
        const double delta = Rs - dist;
        if (!(delta > 0.0) || dist == 0.0) continue;
        const float id = (float)(1.0 / dist);
        const float nx = (float)d[0] * id, ny = (float)d[1] * id, nz = (float)d[2] * id;
        const float vn = (float)(va[0] - vb[0]) * nx + (float)(va[1] - vb[1]) * ny + (float)(va[2] - vb[2]) * nz;
        const double mb = sphere_mass(pt, b);
        const double meff = pt.fixed[b] ? ma : (pt.fixed[a] ? mb : ma * mb / (ma + mb));
        const float fn = kn * (float)delta - ce * sqrtf((float)meff * kn) * vn;
        F[0] += (double)(fn * nx);
        F[1] += (double)(fn * ny);
        F[2] += (double)(fn * nz);
        if (fric) {
            const double n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
            const double la = Ra - 0.5 * delta, lb = pt.R[b] - 0.5 * delta;
            double S[3], vr[3];
            for (int c = 0; c < 3; ++c) S[c] = la * wa[c] + lb * Ws[3 * b + c];
            vr[0] = va[0] - vb[0] - (S[1] * n[2] - S[2] * n[1]);
            vr[1] = va[1] - vb[1] - (S[2] * n[0] - S[0] * n[2]);
            vr[2] = va[2] - vb[2] - (S[0] * n[1] - S[1] * n[0]);
            open_contact_friction(pt, n, vr, (double)fn, pt.ct * sqrt(meff * pt.kt), la, F, T);
        }
    }
    const float gw = ce * sqrtf((float)ma * kn);
    const float vz = (float)va[2];
    const double lo = Ra - (xa[2] + 0.5);
    if (lo > 0.0) F[2] += (double)(kn * (float)lo - gw * vz);
    const double hi = Ra - ((L.nz - 0.5) - xa[2]);
    if (hi > 0.0) F[2] -= (double)(kn * (float)hi + gw * vz);
    for (int side = 0; side < 2 && fric; ++side) {
        const double pen = side == 0 ? lo : hi;
        if (!(pen > 0.0)) continue;
        const double n[3] = {0.0, 0.0, side == 0 ? 1.0 : -1.0};
        const float *uw = side == 0 ? pt.ulo : pt.uhi;
        const double l = Ra - 0.5 * pen;
        const double fn = side == 0 ? (double)(kn * (float)lo - gw * vz) : (double)(kn * (float)hi + gw * vz);
        double vr[3];
        vr[0] = va[0] - uw[0] - (l * wa[1] * n[2] - l * wa[2] * n[1]);
        vr[1] = va[1] - uw[1] - (l * wa[2] * n[0] - l * wa[0] * n[2]);
        vr[2] = va[2] - uw[2] - (l * wa[0] * n[1] - l * wa[1] * n[0]);
        open_contact_friction(pt, n, vr, fn, pt.ct * sqrt(ma * pt.kt), l, F, T);
    }
}

__global__ void k_contact(const Lat L, const Parts pt) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= pt.np) return;
    double F[3], T[3] = {0.0, 0.0, 0.0};
    contact_force(L, pt, a, pt.X + 3 * a, pt.V + 3 * a, pt.X, pt.V, F, pt.W + 3 * a, pt.W, T);
    for (int c = 0; c < 3; ++c) {
        pt.Fc[3 * a + c] = F[c];
        pt.Tc[3 * a + c] = T[c];
    }
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

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }

// Returns false (and sets the timeout status) if the other blocks did not
// arrive within ~2^22 polls, or if another block already gave up.
#ifndef LBM_BAR_SLEEP_NS
#define LBM_BAR_SLEEP_NS 32  // pause between polls
#endif
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
#if LBM_BAR_SLEEP_NS > 0
            __nanosleep(LBM_BAR_SLEEP_NS);
#endif
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// FP32 tangential force of a contact (Eqs. 2, 3) with displacement d (in /
// out): d turned into the plane normal to n and advanced by v_t h; the trial
// force -k_t d - gamma_t v_t, capped at mu max(f^n, 0) along -v_t (along the
// trial force if v_t = 0) with d reset to -f_t / k_t.
__device__ __forceinline__ float3 tangential_force(float3 &d, const float3 n, const float3 vt, const float fn,
                                                   const float gt, const float kt, const float mu, const float h) {
    const float dn = d.x * n.x + d.y * n.y + d.z * n.z;
    d.x += vt.x * h - dn * n.x;
    d.y += vt.y * h - dn * n.y;
    d.z += vt.z * h - dn * n.z;
    float3 f = make_float3(-kt * d.x - gt * vt.x, -kt * d.y - gt * vt.y, -kt * d.z - gt * vt.z);
    const float t2 = f.x * f.x + f.y * f.y + f.z * f.z;
    const float cap = mu * fmaxf(fn, 0.f);
    if (t2 > cap * cap) {
        const float v2 = vt.x * vt.x + vt.y * vt.y + vt.z * vt.z;
        const float s = v2 > 0.f ? -cap * rsqrtf(v2) : cap * rsqrtf(t2);
        const float3 u = v2 > 0.f ? vt : f;
        f = make_float3(s * u.x, s * u.y, s * u.z);
        const float ik = -1.f / kt;
        d = make_float3(f.x * ik, f.y * ik, f.z * ik);
    }
    return f;
}

// Tangential force and its moment on a sphere at contact normal n (pointing
// into the sphere), lever l, relative velocity vr of the contact point.
__device__ __forceinline__ void friction_add(float3 &F, float3 &T, float3 &d, const float3 n, const float3 vr,
                                             const float l, const float fn, const float gt, const float kt,
                                             const float mu, const float h) {
    const float vrn = vr.x * n.x + vr.y * n.y + vr.z * n.z;
    const float3 vt = make_float3(vr.x - vrn * n.x, vr.y - vrn * n.y, vr.z - vrn * n.z);
    const float3 f = tangential_force(d, n, vt, fn, gt, kt, mu, h);
    F.x += f.x;
    F.y += f.y;
    F.z += f.z;
    T.x -= l * (n.y * f.z - n.z * f.y);
    T.y -= l * (n.z * f.x - n.x * f.z);
    T.z -= l * (n.x * f.y - n.y * f.x);
}

__device__ __forceinline__ float3 cross3(const float3 a, const float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// All sub-steps of the lattice step of parity sp in one cluster (gridDim.x
// CTAs).  Thread t of CTA c owns spheres a = c T + t + q G (q < K,
// G = cluster threads).  The step's neighbour pass has read rebuild[sp], so
// it is cleared here; the commits may set rebuild[sp ^ 1].  FRIC: with the
// tangential contact law (each sphere also publishes its spin change).
// GRID: the same sub-steps on a cooperative grid of any size: the spheres
// publish (dx, dv, dOm) in a global buffer xbuf [2][np][S] (read through L2)
// and a bounded grid barrier replaces the cluster barrier; used for sphere
// counts one cluster holds poorly.  Returns early (the step is then void and
// the timeout status set) if a barrier gives up.
template <bool FRIC, bool GRID>
__device__ __forceinline__ void dem_cluster_body(const Lat &L, const Parts &pt, SFrame *fnext, const int sp,
                                                 int *status, float4 *xbuf = nullptr, unsigned *bar = nullptr) {
    constexpr int S = FRIC ? 3 : 2;  // float4 per sphere in the exchange buffer: dx, dv (, dOm)
    constexpr int K = dem_kmax(FRIC);
    extern __shared__ float4 dsm[];  // [2][K * T][S]
    namespace cg = cooperative_groups;
    const int T = blockDim.x, G = gridDim.x * T, cap = K * T;
    unsigned target = 0;
    const int g0 = blockIdx.x * T + threadIdx.x;
    if (g0 == 0) pt.rebuild[sp] = 0;
    const int ns = pt.substeps;
    const float h = 1.f / ns, h2 = 0.5f * h;
    const float kn = (float)pt.kn, ce = (float)pt.ce;
    const float kt = (float)pt.kt, mu = (float)pt.mu;
    float3 dx[K], dv[K], v0[K], fa[K], fc[K];
    float im[K], Rf[K], Llo[K], Lhi[K], gw[K];
    int nc[K];
    bool fx[K];
    // with friction: spin change, start spin, torque / I, contact torque, 1 / I,
    // open-contact mask, wall displacements (w = 1: in contact), wall gamma_t
    float3 dw[FRIC ? K : 1], w0[FRIC ? K : 1], ta[FRIC ? K : 1], tc[FRIC ? K : 1];
    float iI[FRIC ? K : 1], gwt[FRIC ? K : 1];
    unsigned long long msk[FRIC ? K : 1];
    float4 wl[FRIC ? K : 1][2];
#pragma unroll
    for (int q = 0; q < K; ++q) {
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
        nc[q] = pt.nact[a];
        dx[q] = make_float3(0.f, 0.f, 0.f);
        dv[q] = make_float3(0.f, 0.f, 0.f);
        if constexpr (FRIC) {
            const double ii = 1.0 / (0.4 * m * R * R);
            iI[q] = (float)ii;
            w0[q] = make_float3((float)pt.W[3 * a], (float)pt.W[3 * a + 1], (float)pt.W[3 * a + 2]);
            ta[q] = make_float3((float)((pt.Th[3 * a] + pt.Tx[3 * a]) * ii),
                                (float)((pt.Th[3 * a + 1] + pt.Tx[3 * a + 1]) * ii),
                                (float)((pt.Th[3 * a + 2] + pt.Tx[3 * a + 2]) * ii));
            tc[q] = make_float3((float)pt.Tc[3 * a], (float)pt.Tc[3 * a + 1], (float)pt.Tc[3 * a + 2]);
            dw[q] = make_float3(0.f, 0.f, 0.f);
            msk[q] = pt.tmask[a];
            wl[q][0] = pt.twall[2 * a];
            wl[q][1] = pt.twall[2 * a + 1];
            gwt[q] = (float)pt.ct * sqrtf((float)m * kt);
        }
    }
    if constexpr (!GRID) cluster_barrier();  // every CTA of the cluster is running before shared memory is shared
    for (int s = 0; s < ns; ++s) {
        float4 *buf = GRID ? xbuf + (size_t)((s + 1) & 1) * pt.np * S : dsm + (size_t)((s + 1) & 1) * cap * S;
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const int a = g0 + q * G;
            if (a >= pt.np) break;
            if (!fx[q]) {  // half kick
                dv[q].x += (fa[q].x + fc[q].x * im[q]) * h2;
                dv[q].y += (fa[q].y + fc[q].y * im[q]) * h2;
                dv[q].z += (fa[q].z + fc[q].z * im[q]) * h2;
                if constexpr (FRIC) {
                    dw[q].x += (ta[q].x + tc[q].x * iI[q]) * h2;
                    dw[q].y += (ta[q].y + tc[q].y * iI[q]) * h2;
                    dw[q].z += (ta[q].z + tc[q].z * iI[q]) * h2;
                }
            }
            dx[q].x += (v0[q].x + dv[q].x) * h;
            dx[q].y += (v0[q].y + dv[q].y) * h;
            dx[q].z += (v0[q].z + dv[q].z) * h;
            float4 *me = buf + (GRID ? (size_t)a * S : (size_t)(q * T + threadIdx.x) * S);
            me[0] = make_float4(dx[q].x, dx[q].y, dx[q].z, 0.f);
            me[1] = make_float4(dv[q].x, dv[q].y, dv[q].z, 0.f);
            if constexpr (FRIC) me[2] = make_float4(dw[q].x, dw[q].y, dw[q].z, 0.f);
        }
        if constexpr (GRID) {
            target += gridDim.x;
            if (!grid_barrier(bar, target, status)) return;
        } else {
            cluster_barrier();
        }
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const int a = g0 + q * G;
            if (a >= pt.np) break;
            if (fx[q]) continue;
            float3 F = make_float3(0.f, 0.f, 0.f);
            float3 Tq = make_float3(0.f, 0.f, 0.f);
            // neighbours in groups of kNbrGroup: every load of a group is
            // issued before any of its arithmetic; the sum keeps list order
            constexpr int kNbrGroup = 4;
            for (int m0 = 0; m0 < nc[q]; m0 += kNbrGroup) {
                float4 A[kNbrGroup], Bv[kNbrGroup], ox[kNbrGroup], ov[kNbrGroup];
                float4 C[FRIC ? kNbrGroup : 1], ow[FRIC ? kNbrGroup : 1], td[FRIC ? kNbrGroup : 1];
                float Rb[kNbrGroup];
                int lm[kNbrGroup];  // list position of the candidate (its contact state)
#pragma unroll
                for (int u = 0; u < kNbrGroup; ++u) {
                    if (m0 + u >= nc[q]) break;
                    const long long e = (long long)a * pt.max_nbr + m0 + u;
                    const int2 bm = __ldg(pt.pairBM + e);
                    const int b = bm.x;
                    lm[u] = bm.y;
                    A[u] = __ldg(pt.pairA + e);
                    Bv[u] = __ldg(pt.pairB + e);
                    Rb[u] = __ldg(&pt.Xf[b].w);
                    if constexpr (FRIC)  // the open contact's displacement, loaded with the group
                        td[u] = (msk[q] >> lm[u]) & 1ull ? pt.tdisp[(long long)a * pt.max_nbr + lm[u]]
                                                         : make_float4(0.f, 0.f, 0.f, 0.f);
                    if constexpr (GRID) {
                        const float4 *o = buf + (size_t)b * S;
                        ox[u] = __ldcg(o);
                        ov[u] = __ldcg(o + 1);
                        if constexpr (FRIC) {
                            C[u] = __ldg(pt.pairC + e);
                            ow[u] = __ldcg(o + 2);
                        }
                    } else {
                        const int qb = b / G, rb = b - qb * G, cb = rb / T, tb = rb - cb * T;
                        const float4 *o = cg::this_cluster().map_shared_rank(buf + (size_t)(qb * T + tb) * S, cb);
                        ox[u] = o[0];
                        ov[u] = o[1];
                        if constexpr (FRIC) {
                            C[u] = __ldg(pt.pairC + e);
                            ow[u] = o[2];
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < kNbrGroup; ++u) {
                    if (m0 + u >= nc[q]) break;
                    const float Dx = dx[q].x - ox[u].x, Dy = dx[q].y - ox[u].y, Dz = dx[q].z - ox[u].z;
                    const float c =
                        A[u].w - 2.f * (A[u].x * Dx + A[u].y * Dy + A[u].z * Dz) - (Dx * Dx + Dy * Dy + Dz * Dz);
                    if (!(c > 0.f)) {
                        if constexpr (FRIC) msk[q] &= ~(1ull << lm[u]);  // the contact opened
                        continue;
                    }
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
                    if constexpr (FRIC) {
                        const int m = lm[u];
                        const long long e = (long long)a * pt.max_nbr + m;
                        const float la = Rf[q] - 0.5f * delta, lb = Rb[u] - 0.5f * delta;
                        const float3 n = make_float3(nx, ny, nz);
                        const float3 Sw = make_float3(la * (w0[q].x + dw[q].x) + lb * (C[u].x + ow[u].x),
                                                      la * (w0[q].y + dw[q].y) + lb * (C[u].y + ow[u].y),
                                                      la * (w0[q].z + dw[q].z) + lb * (C[u].z + ow[u].z));
                        const float3 Sn = cross3(Sw, n);
                        const float3 vr = make_float3(Bv[u].x + dv[q].x - ov[u].x - Sn.x,
                                                      Bv[u].y + dv[q].y - ov[u].y - Sn.y,
                                                      Bv[u].z + dv[q].z - ov[u].z - Sn.z);
                        float3 d = make_float3(td[u].x, td[u].y, td[u].z);
                        friction_add(F, Tq, d, n, vr, la, fn, C[u].w, kt, mu, h);
                        pt.tdisp[e] = make_float4(d.x, d.y, d.z, 0.f);
                        msk[q] |= 1ull << m;
                    }
                }
            }
            const float vz = v0[q].z + dv[q].z;
            const float lo = Llo[q] - dx[q].z;
            if (lo > 0.f) F.z += kn * lo - gw[q] * vz;
            const float hi = Lhi[q] + dx[q].z;
            if (hi > 0.f) F.z -= kn * hi + gw[q] * vz;
            if constexpr (FRIC) {
                const float3 w = make_float3(w0[q].x + dw[q].x, w0[q].y + dw[q].y, w0[q].z + dw[q].z);
                const float3 v = make_float3(v0[q].x + dv[q].x, v0[q].y + dv[q].y, vz);
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    const float pen = side == 0 ? lo : hi;
                    if (!(pen > 0.f)) {
                        wl[q][side] = make_float4(0.f, 0.f, 0.f, 0.f);  // the contact opened
                        continue;
                    }
                    const float sg = side == 0 ? 1.f : -1.f;
                    const float3 n = make_float3(0.f, 0.f, sg);
                    const float *uw = side == 0 ? pt.ulo : pt.uhi;
                    const float l = Rf[q] - 0.5f * pen;
                    const float3 Sn = cross3(make_float3(l * w.x, l * w.y, l * w.z), n);
                    const float3 vr = make_float3(v.x - uw[0] - Sn.x, v.y - uw[1] - Sn.y, v.z - uw[2] - Sn.z);
                    const float fn = side == 0 ? kn * lo - gw[q] * vz : kn * hi + gw[q] * vz;
                    float3 d = wl[q][side].w != 0.f ? make_float3(wl[q][side].x, wl[q][side].y, wl[q][side].z)
                                                    : make_float3(0.f, 0.f, 0.f);
                    friction_add(F, Tq, d, n, vr, l, fn, gwt[q], kt, mu, h);
                    wl[q][side] = make_float4(d.x, d.y, d.z, 1.f);
                }
                tc[q] = Tq;
                dw[q].x += (ta[q].x + Tq.x * iI[q]) * h2;
                dw[q].y += (ta[q].y + Tq.y * iI[q]) * h2;
                dw[q].z += (ta[q].z + Tq.z * iI[q]) * h2;
            }
            fc[q] = F;
            dv[q].x += (fa[q].x + F.x * im[q]) * h2;
            dv[q].y += (fa[q].y + F.y * im[q]) * h2;
            dv[q].z += (fa[q].z + F.z * im[q]) * h2;
        }
    }
    if constexpr (!GRID) cluster_barrier();  // no CTA leaves while another may still read its shared memory
#pragma unroll
    for (int q = 0; q < K; ++q) {
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
            if constexpr (FRIC) {
                w[0] += (double)dw[q].x;
                w[1] += (double)dw[q].y;
                w[2] += (double)dw[q].z;
            } else {
                for (int c = 0; c < 3; ++c) w[c] += (pt.Th[3 * a + c] + pt.Tx[3 * a + c]) * iI;
            }
        }
        if constexpr (FRIC) {
            pt.Tc[3 * a] = (double)tc[q].x;
            pt.Tc[3 * a + 1] = (double)tc[q].y;
            pt.Tc[3 * a + 2] = (double)tc[q].z;
            pt.tmask[a] = msk[q];
            pt.twall[2 * a] = wl[q][0];
            pt.twall[2 * a + 1] = wl[q][1];
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

template <bool FRIC>
__global__ void __launch_bounds__(kDemThreads, 1) k_dem_cluster(const Lat L, const Parts pt, SFrame *fnext,
                                                                const int sp, int *status) {
    dem_cluster_body<FRIC, false>(L, pt, fnext, sp, status);
}

#ifndef LBM_DEM_GRID_THREADS
#define LBM_DEM_GRID_THREADS 64
#endif
constexpr int kDemGridThreads = LBM_DEM_GRID_THREADS;  // threads per CTA of the grid form
// sphere count from which the automatic choice takes the grid form: one
// cluster then holds two or more spheres per thread (measured: 8136 spheres
// with friction, DEM 0.31 ms per step in the cluster, 0.14 ms in the grid)
constexpr int kDemGridFrom = 4096;

template <bool FRIC>
__global__ void __launch_bounds__(kDemGridThreads) k_dem_grid(const Lat L, const Parts pt, SFrame *fnext,
                                                              const int sp, int *status, float4 *xbuf,
                                                              unsigned *bar) {
    dem_cluster_body<FRIC, true>(L, pt, fnext, sp, status, xbuf, bar);
}

// Batched forms: instance blockIdx.y.
__global__ void __launch_bounds__(256) k_neighbours_b(const Inst *__restrict__ I, const int sp) {
    const Inst &a = I[blockIdx.y];
    if ((int)(blockIdx.x * (blockDim.x >> 5)) >= a.pt.np) return;
    neighbours_body(a.L, a.pt, sp, 0, a.status);
}

// FRIC = true when a member has friction; the clusters of members without
// it run the frictionless body.
template <bool FRIC>
__global__ void __launch_bounds__(kDemThreads, 1) k_dem_cluster_b(const Inst *__restrict__ I, const int sp) {
    const Inst &a = I[blockIdx.y];
    if (a.pt.np == 0) return;  // the whole cluster (one instance) leaves together
    if (FRIC && !a.pt.fric) dem_cluster_body<false, false>(a.L, a.pt, a.pt.frame[sp ^ 1], sp, a.status);
    else dem_cluster_body<FRIC, false>(a.L, a.pt, a.pt.frame[sp ^ 1], sp, a.status);
}

static size_t dem_cluster_smem(bool fric) {
    return (size_t)2 * dem_kmax(fric) * kDemThreads * (fric ? 3 : 2) * sizeof(float4);
}

// ---- fallback: cooperative grid with a bounded software barrier ------------

// Self-test of the bounded wait: one block waits at the grid barrier for a
// second block that does not exist, so the wait runs out of polls, sets the
// timeout status and returns.
__global__ void k_wait_probe(unsigned *bar, int *status) { grid_barrier(bar, 2u, status); }

int launch_wait_probe(lbm_s *h) {
    if (cudaMemsetAsync(h->bar, 0, sizeof(unsigned), h->stream) != cudaSuccess) return LBM_ERR_CUDA;
    k_wait_probe<<<1, 32, 0, h->stream>>>(h->bar, h->status);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
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

template <typename K>
static bool cluster_attrs(K kernel, bool fric, int cl) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dem_cluster_smem(fric)) !=
            cudaSuccess ||
        (cl > 8 && cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// Largest cluster (16, else 8) that can run k_dem_cluster; 0 if none, or if
// max_particles does not fit its registers.
int dem_cluster_setup(int max_particles, bool small, bool fric) {
    // one simulation: the widest cluster (16 or 8 CTAs: measured equal at
    // 2000 spheres, narrower ones slower); a batch: the narrowest cluster
    // that gives every sphere its own thread, so that the members' clusters
    // run side by side
    const std::vector<int> sizes = small ? std::vector<int>{1, 2, 4, 8, 16} : std::vector<int>{16, 8};
    for (int cl : sizes) {
        if ((long long)cl * kDemThreads * dem_kmax(fric) < max_particles) continue;
        if (small && (long long)cl * kDemThreads < max_particles && cl < 16) continue;
        if (!(fric ? cluster_attrs(k_dem_cluster<true>, true, cl) : cluster_attrs(k_dem_cluster<false>, false, cl)))
            continue;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(cl);
        cfg.blockDim = dim3(kDemThreads);
        cfg.dynamicSmemBytes = dem_cluster_smem(fric);
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        const cudaError_t e = fric ? cudaOccupancyMaxActiveClusters(&n, k_dem_cluster<true>, &cfg)
                                   : cudaOccupancyMaxActiveClusters(&n, k_dem_cluster<false>, &cfg);
        if (e == cudaSuccess && n >= 1) return cl;
        cudaGetLastError();
    }
    return 0;
}

int dem_cluster_setup_batch(int cl, bool fric) {
    const bool ok = fric ? cluster_attrs(k_dem_cluster_b<true>, true, cl) : cluster_attrs(k_dem_cluster_b<false>, false, cl);
    return ok ? LBM_OK : LBM_ERR_CUDA;
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
    cfg.dynamicSmemBytes = dem_cluster_smem(b->fric);
    cfg.stream = b->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const Inst *I = b->dinst;
    const cudaError_t e = b->fric ? cudaLaunchKernelEx(&cfg, k_dem_cluster_b<true>, I, sp)
                                  : cudaLaunchKernelEx(&cfg, k_dem_cluster_b<false>, I, sp);
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

// Largest co-resident grid of the grid form (blocks), 0 on failure.
int dem_grid_setup(bool fric, int sms) {
    int per_sm = 0;
    const cudaError_t e =
        fric ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dem_grid<true>, kDemGridThreads, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dem_grid<false>, kDemGridThreads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * sms;
}

// Spheres the grid form holds with `blocks` co-resident blocks.
long long dem_grid_capacity(bool fric, int blocks) { return (long long)blocks * kDemGridThreads * dem_kmax(fric); }

// Grid form: one sphere per thread while the co-resident grid allows, a
// cooperative launch (so every block is resident for the grid barriers).
static int launch_dem_grid(lbm_s *h, SFrame *fnext, int sp) {
    const bool fric = h->pt.fric != 0;
    const int np = h->pt.np;
    int blocks = (np + kDemGridThreads - 1) / kDemGridThreads;
    if (blocks > h->dem_grid_blocks) blocks = h->dem_grid_blocks;
    if (blocks < 1 || dem_grid_capacity(fric, blocks) < np) return LBM_ERR_UNSUPPORTED;
    if (cudaMemsetAsync(h->bar, 0, sizeof(unsigned), h->stream) != cudaSuccess) return LBM_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kDemGridThreads);
    cfg.stream = h->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const Lat L = h->L;
    const Parts pt = h->pt;
    const cudaError_t e =
        fric ? cudaLaunchKernelEx(&cfg, k_dem_grid<true>, L, pt, fnext, sp, h->status, h->xbuf, h->bar)
             : cudaLaunchKernelEx(&cfg, k_dem_grid<false>, L, pt, fnext, sp, h->status, h->xbuf, h->bar);
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int launch_dem(lbm_s *h) {
    Lat L = h->L;
    Parts pt = h->pt;
    int *status = h->status;
    SFrame *fnext = h->pt.frame[(h->steps + 1) & 1];
    const int sp = (int)(h->steps & 1);
    const bool grid = h->dem_grid_blocks > 0 &&
                      (h->dem_mode == LBM_DEM_GRID ||
                       (h->dem_mode == LBM_DEM_AUTO && (h->dem_cluster == 0 || pt.np > kDemGridFrom)));
    if (grid) return launch_dem_grid(h, fnext, sp);
    if (h->dem_cluster > 0) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = h->dem_cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(h->dem_cluster);
        cfg.blockDim = dim3(kDemThreads);
        const bool fric = pt.fric != 0;
        cfg.dynamicSmemBytes = dem_cluster_smem(fric);
        cfg.stream = h->stream;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const cudaError_t e = fric ? cudaLaunchKernelEx(&cfg, k_dem_cluster<true>, L, pt, fnext, sp, status)
                                   : cudaLaunchKernelEx(&cfg, k_dem_cluster<false>, L, pt, fnext, sp, status);
        return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
    }
    if (pt.fric) return LBM_ERR_UNSUPPORTED;  // the FP64 fallback keeps no tangential contact state
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
