// C ABI (include/lbm.h): validation, device allocation, launch order of one
// step, and copies in and out.  No arithmetic of the method lives here.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include <algorithm>
#include <vector>

#include "lbm_internal.cuh"

using namespace lbm;

namespace {

constexpr int kMaxNbr = 48;  // at most 64: the DEM keeps one contact bit per list entry
static_assert(kMaxNbr <= 64, "contact mask");
constexpr int kDemThreads = 128;   // fallback cooperative DEM
constexpr double kSkin = 1.5;      // neighbour-list skin (lattice units)
constexpr double kMaxStep = 0.25;  // largest displacement of a sphere in one step

// Profiler events of one step: on the main stream E0 before the geometry,
// E1 after it, E2 after the (near) collide, E3 after waiting for the far
// collide, E4 after the links, E5 after the DEM; on the second stream
// E6 / E7 around the far collide.  Phase k is the time between two of them.
enum { E0, E1, E2, E3, E4, E5, E6, E7, kProfEv };
constexpr int kPhaseFrom[LBM_PHASES] = {E0, E1, E3, E4, E6, E2};
constexpr int kPhaseTo[LBM_PHASES] = {E1, E2, E4, E5, E7, E3};

int status_to_code(int st) {
    if (st & ST_TIMEOUT) return LBM_ERR_TIMEOUT;
    if (st & ST_DIVERGED) return LBM_ERR_DIVERGED;
    if (st & (ST_NBR_OVERFLOW | ST_TILE)) return LBM_ERR_CAPACITY;
    if (st & ST_FAST) return LBM_ERR_GEOMETRY;
    return LBM_OK;
}



template <class T>
int dalloc(lbm_s *h, T **p, size_t n) {
    *p = nullptr;
    if (n == 0) return LBM_OK;
    if (cudaMalloc((void **)p, n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return LBM_ERR_NOMEM;
    }
    h->bytes += n * sizeof(T);
    return LBM_OK;
}

void release(lbm_s *h) {
    void *ptrs[] = {h->f, h->flag, h->owner, h->status, h->bar, h->ctr, h->pt.X, h->pt.V, h->pt.W, h->pt.R,
                    (void *)h->pt.fixed, h->pt.Fh, h->pt.Th, h->pt.Fc, h->pt.Fx, h->pt.Tx, h->pt.Xf,
                    h->pt.Xb[0], h->pt.Xb[1], h->pt.Vh[0], h->pt.Vh[1], h->pt.nbr, h->pt.nbr_cnt, h->pt.pairA,
                    h->pt.pairB, h->pt.Xbuild, h->pt.rebuild, h->pt.frame[0], h->pt.frame[1], h->pt.Fcorr,
                    h->pt.Tcorr, h->pt.Tc, h->pt.pairC, h->pt.tdisp, h->pt.tmask, h->pt.twall, h->zs, h->pt.pairBM, h->pt.nact,
                    h->xbuf,
                    h->zpart, h->zcnt};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->status_host) cudaFreeHost(h->status_host);
    for (int k = 0; k < 2; ++k) {
        if (h->load_stage[k]) cudaFreeHost(h->load_stage[k]);
        if (h->load_ev[k]) cudaEventDestroy(h->load_ev[k]);
    }
    if (h->ev) {
        for (int i = 0; i < kProfEv * h->ev_cap; ++i) cudaEventDestroy(h->ev[i]);
        std::free(h->ev);
        h->ev = nullptr;
    }
    void *ovl[] = {h->near[0], h->near[1], h->near_list[0], h->near_list[1], h->near_cnt,
                   h->far_list[0], h->far_list[1], h->far_cnt};
    for (void *p : ovl)
        if (p) cudaFree(p);
    cudaEvent_t evs[] = {h->ev_cf, h->ev_nm[0], h->ev_nm[1], h->ev_join};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    for (cudaGraphExec_t &g : h->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    if (h->stream2) cudaStreamDestroy(h->stream2);
    if (h->chain) cudaStreamDestroy(h->chain);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_nbr) cudaEventDestroy(h->ev_nbr);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

constexpr int kProfSteps = 2048;

// Fold the recorded events into the phase totals (synchronises).
int prof_flush(lbm_s *h) {
    if (!h->ev || h->ev_used == 0) return LBM_OK;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ERR_CUDA;
    if (h->stream2 && cudaStreamSynchronize(h->stream2) != cudaSuccess) return LBM_ERR_CUDA;
    if (h->chain && cudaStreamSynchronize(h->chain) != cudaSuccess) return LBM_ERR_CUDA;
    for (int s = 0; s < h->ev_used; ++s)
        for (int ph = 0; ph < LBM_PHASES; ++ph) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, h->ev[kProfEv * s + kPhaseFrom[ph]], h->ev[kProfEv * s + kPhaseTo[ph]]) !=
                cudaSuccess)
                return LBM_ERR_CUDA;
            h->prof_ms[ph] += ms;
        }
    h->prof_steps += h->ev_used;
    h->ev_used = 0;
    return LBM_OK;
}

inline int prof_mark(lbm_s *h, int k, cudaStream_t st) {
    if (!h->prof) return LBM_OK;
    return cudaEventRecord(h->ev[kProfEv * h->ev_used + k], st) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

// Sync the stream and fold the device status into the sticky error (the
// status word comes back to pinned host memory on the same stream, so one
// synchronisation covers both).
int settle(lbm_s *h) {
    if (cudaMemcpyAsync(h->status_host, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        if (!h->sticky) h->sticky = LBM_ERR_CUDA;
        return h->sticky;
    }
    const int c = status_to_code(*h->status_host);
    if (c && !h->sticky) h->sticky = c;
    return h->sticky;
}

bool finite3(const double *v, int n) {
    for (int i = 0; i < 3 * n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// Copy n bytes from a caller buffer (host or device) into device memory.
int copy_in(lbm_s *h, void *dst, const void *src, size_t n, int where) {
    if (n == 0) return LBM_OK;
    const cudaMemcpyKind k = where == LBM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    return cudaMemcpyAsync(dst, src, n, k, h->stream) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int copy_out(lbm_s *h, void *dst, const void *src, size_t n, int where) {
    if (n == 0 || !dst) return LBM_OK;
    const cudaMemcpyKind k = where == LBM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    return cudaMemcpyAsync(dst, src, n, k, h->stream) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

// ZIEB cylinder at rest: rho = 1 and H_p = 0 in both parity slots, piston
// velocity vp, inflow sums 0 (synchronous).
int zieb_reset(lbm_s *h, double vp) {
    const double z[5] = {1.0, 1.0, 0.0, 0.0, vp};
    if (cudaStreamSynchronize(h->stream) != cudaSuccess ||
        cudaMemcpy(h->zs, z, sizeof(z), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(h->zpart, 0, sizeof(double) * 2 * (size_t)h->zblocks) != cudaSuccess ||
        cudaMemset(h->zcnt, 0, sizeof(int) * 2 * (size_t)h->zblocks) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

// Run fn(device pointer) on a device buffer of n bytes: the caller's own if
// where == LBM_DEVICE, else a stream-ordered temporary copied to the host.
template <class Fn>
int with_out_buffer(lbm_s *h, void *user, size_t n, int where, Fn fn) {
    if (where == LBM_DEVICE) return fn(user);
    void *tmp = nullptr;
    if (cudaMallocAsync(&tmp, n, h->stream) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_NOMEM;
    }
    int rc = fn(tmp);
    if (rc == LBM_OK) rc = copy_out(h, user, tmp, n, LBM_HOST);
    cudaFreeAsync(tmp, h->stream);
    return rc;
}

}  // namespace

namespace lbm {
int settle_handle(lbm_s *h) { return settle(h); }
}  // namespace lbm

extern "C" {

const char *lbm_error_string(int code) {
    switch (code) {
        case LBM_OK: return "success";
        case LBM_ERR_ARG: return "invalid argument";
        case LBM_ERR_CUDA: return "CUDA runtime error";
        case LBM_ERR_NOMEM: return "device allocation failed";
        case LBM_ERR_CAPACITY: return "capacity exceeded (spheres, neighbours or link tile)";
        case LBM_ERR_DIVERGED: return "lattice diverged (non-positive or non-finite density)";
        case LBM_ERR_UNSUPPORTED: return "unsupported configuration";
        case LBM_ERR_TIMEOUT: return "device-side wait timed out";
        case LBM_ERR_GEOMETRY: return "a sphere moved a quarter of a lattice unit or more in one step, or left the box";
    }
    return "unknown error";
}

int lbm_create(const lbm_params *prm, lbm_handle *out) {
    if (!prm || !out) return LBM_ERR_ARG;
    *out = nullptr;
    const lbm_params &p = *prm;
    if (p.nx < 1 || p.ny < 1 || p.nz < 1) return LBM_ERR_ARG;
    if (p.periodic_z != 0) return LBM_ERR_UNSUPPORTED;
    if (!(p.tau0 > 0.5) || !std::isfinite(p.tau0)) return LBM_ERR_ARG;
    if (!(p.cs_smag >= 0.0) || !std::isfinite(p.cs_smag)) return LBM_ERR_ARG;
    if (!finite3(p.body_accel, 1) || !finite3(p.wall_vel_lo, 1) || !finite3(p.wall_vel_hi, 1)) return LBM_ERR_ARG;
    if (p.wall_vel_lo[2] != 0.0 || p.wall_vel_hi[2] != 0.0) return LBM_ERR_ARG;
    if (!(p.rho_particle > 0.0) || !(p.kn >= 0.0) || !(p.restitution > 0.0 && p.restitution <= 1.0) ||
        !std::isfinite(p.rho_particle) || !std::isfinite(p.kn))
        return LBM_ERR_ARG;
    if (p.dem_substeps < 1) return LBM_ERR_ARG;
    if (p.precision != LBM_FP32 && p.precision != LBM_BF16_DEV && p.precision != LBM_FP16_DEV) return LBM_ERR_ARG;
    if (p.max_particles < 0) return LBM_ERR_ARG;
    if (p.schedule != LBM_SCHEDULE_OVERLAP && p.schedule != LBM_SCHEDULE_SERIAL) return LBM_ERR_ARG;
    if (p.momentum_correction != 0 && p.momentum_correction != 1) return LBM_ERR_ARG;
    if (!(p.kt >= 0.0) || !(p.mu >= 0.0) || !(p.restitution_t > 0.0 && p.restitution_t <= 1.0) ||
        !std::isfinite(p.kt) || !std::isfinite(p.mu))
        return LBM_ERR_ARG;
    if (p.zieb != 0 && p.zieb != 1) return LBM_ERR_ARG;
    if (p.mea != LBM_MEA_PAPER && p.mea != LBM_MEA_GALILEAN) return LBM_ERR_ARG;
    if (p.dem_mode != LBM_DEM_AUTO && p.dem_mode != LBM_DEM_CLUSTER && p.dem_mode != LBM_DEM_GRID)
        return LBM_ERR_ARG;
    if (p.zieb && (!(p.zieb_area > 0.0) || !(p.zieb_volume > 0.0) || !std::isfinite(p.zieb_area) ||
                   !std::isfinite(p.zieb_volume) || !std::isfinite(p.zieb_piston_velocity)))
        return LBM_ERR_ARG;
    // the face update runs between steps; the overlapped schedule collides
    // far nodes (the face among them) of the next step meanwhile
    if (p.zieb && p.schedule != LBM_SCHEDULE_SERIAL) return LBM_ERR_UNSUPPORTED;
    if (p.max_particles > 0) {
        if (!(p.max_radius > 0.0 && p.max_radius <= 16.0)) return LBM_ERR_ARG;
        // a sphere's bounding box and link tile must not wrap onto itself
        const int span = 2 * ((int)std::ceil(p.max_radius) + 3) + 1;
        if (p.nx < span || p.ny < span) return LBM_ERR_ARG;
    }
    const long long plane = (long long)p.nx * p.ny;
    const long long N = plane * p.nz;
    // kernels index the population array with 32-bit element offsets
    if ((long long)Q * (plane * (p.nz + 2) + 64) >= (1ll << 31)) return LBM_ERR_UNSUPPORTED;

    lbm_s *h = new (std::nothrow) lbm_s();
    if (!h) return LBM_ERR_NOMEM;
    h->p = p;
    h->device = p.device;
    DeviceScope ds(p.device);
    if (cudaSetDevice(p.device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return LBM_ERR_CUDA;
    }
    int rc = LBM_OK;
    // the link / DEM / geometry chain outranks the far-node collisions of
    // the second stream when both have blocks waiting for an SM
    int prio_low = 0, prio_high = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) {
        cudaGetLastError();
        prio_low = prio_high = 0;
    }
    if (p.cuda_stream) {
        h->stream = (cudaStream_t)p.cuda_stream;
    } else {
        if (cudaStreamCreateWithPriority(&h->stream, cudaStreamNonBlocking, prio_high) != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return LBM_ERR_CUDA;
        }
        h->own_stream = true;
    }
    h->precision = p.precision;
    h->esize = p.precision == LBM_FP32 ? 4 : 2;
    h->L.nx = p.nx;
    h->L.ny = p.ny;
    h->L.nz = p.nz;
    h->L.plane = plane;
    h->L.N = N;
    h->L.S = ((plane * (p.nz + 2) + 63) / 64) * 64;
    h->ph.tau0 = (float)p.tau0;
    h->ph.smag = (float)(18.0 * std::sqrt(2.0) * p.cs_smag * p.cs_smag);
    for (int a = 0; a < 3; ++a) {
        h->ph.g[a] = (float)p.body_accel[a];
        h->ph.ulo[a] = (float)p.wall_vel_lo[a];
        h->ph.uhi[a] = (float)p.wall_vel_hi[a];
    }
    const int M = p.max_particles;
    Parts &pt = h->pt;
    pt.np = 0;
    pt.max_nbr = kMaxNbr;
    pt.kn = p.kn;
    const double le = std::log(p.restitution);
    pt.ce = -2.0 * le / std::sqrt(M_PI * M_PI + le * le);
    pt.rho_s = p.rho_particle;
    pt.substeps = p.dem_substeps;
    pt.skin = kSkin;
    pt.max_step = kMaxStep;
    pt.fric = p.kt > 0.0 && p.mu > 0.0;
    pt.gimea = p.mea == LBM_MEA_GALILEAN;
    pt.kt = p.kt;
    pt.mu = p.mu;
    {
        const double lt = std::log(p.restitution_t);
        pt.ct = p.restitution_t < 1.0 ? -2.0 * lt / std::sqrt(M_PI * M_PI + lt * lt) : 0.0;
    }
    for (int a = 0; a < 3; ++a) {
        pt.ulo[a] = (float)p.wall_vel_lo[a];
        pt.uhi[a] = (float)p.wall_vel_hi[a];
    }
    // a solid node lies within [-ceil(R) + 1, ceil(R)] of floor(X) per axis; the
    // link tile also holds x = s - c_j and x - c_j, two more nodes out
    h->tile_ext = (int)std::ceil(M > 0 ? p.max_radius : 1.0) + 2;
    h->link_cap = link_capacity(M > 0 ? p.max_radius : 1.0);

    unsigned char *fixed = nullptr;
    if (!rc) rc = dalloc(h, (unsigned char **)&h->f, (size_t)Q * h->L.S * h->esize);
    if (!rc) rc = dalloc(h, &h->flag, (size_t)N);
    if (!rc) rc = dalloc(h, &h->owner, (size_t)N);
    if (!rc) rc = dalloc(h, &h->status, 1);
    if (!rc) rc = dalloc(h, &h->bar, 1);
    if (!rc) rc = dalloc(h, &h->ctr, 4);
    if (!rc) rc = dalloc(h, &pt.X, 3 * (size_t)M);
    if (!rc) rc = dalloc(h, &pt.V, 3 * (size_t)M);
    if (!rc) rc = dalloc(h, &pt.W, 3 * (size_t)M);
    if (!rc) rc = dalloc(h, &pt.R, (size_t)M);
    if (!rc) rc = dalloc(h, &fixed, (size_t)M);
    pt.fixed = fixed;
    if (!rc) rc = dalloc(h, &pt.Fh, 3 * (size_t)M);
    if (!rc) rc = dalloc(h, &pt.Th, 3 * (size_t)M);
    if (!rc) rc = dalloc(h, &pt.Fc, 3 * (size_t)M);
    if (!rc) rc = dalloc(h, &pt.Fx, 3 * (size_t)M);
    if (!rc) rc = dalloc(h, &pt.Tx, 3 * (size_t)M);
    if (!rc) rc = dalloc(h, &pt.Xbuild, 3 * (size_t)M);
    if (!rc) rc = dalloc(h, &pt.rebuild, 2);
    if (!rc) rc = dalloc(h, &pt.Fcorr, 3 * (size_t)M);
    if (!rc) rc = dalloc(h, &pt.Tcorr, 3 * (size_t)M);
    if (!rc) rc = dalloc(h, &pt.Tc, 3 * (size_t)M);
    if (!rc && p.zieb) {
        h->zieb = 1;
        h->zA = p.zieb_area;
        h->zV0 = p.zieb_volume;
        h->zblocks = (int)(((long long)p.nx * p.ny + 255) / 256);
        rc = dalloc(h, &h->zs, 5);
        if (!rc) rc = dalloc(h, &h->zpart, 2 * (size_t)h->zblocks);
        if (!rc) rc = dalloc(h, &h->zcnt, 2 * (size_t)h->zblocks);
        h->zvp = p.zieb_piston_velocity;
        if (!rc) rc = zieb_reset(h, h->zvp);
    }
    if (!rc && pt.fric) {
        rc = dalloc(h, &pt.pairC, (size_t)M * kMaxNbr);
        if (!rc) rc = dalloc(h, &pt.tdisp, (size_t)M * kMaxNbr);
        if (!rc) rc = dalloc(h, &pt.tmask, (size_t)M);
        if (!rc) rc = dalloc(h, &pt.twall, 2 * (size_t)M);
    }
    pt.corr = p.momentum_correction;
    if (!rc) rc = dalloc(h, &pt.frame[0], (size_t)M);
    if (!rc) rc = dalloc(h, &pt.frame[1], (size_t)M);
    if (!rc) rc = dalloc(h, &pt.pairA, (size_t)M * kMaxNbr);
    if (!rc) rc = dalloc(h, &pt.pairB, (size_t)M * kMaxNbr);
    if (!rc) rc = dalloc(h, &pt.pairBM, (size_t)M * kMaxNbr);
    if (!rc) rc = dalloc(h, &h->xbuf, 2 * 3 * (size_t)M);
    if (!rc) rc = dalloc(h, &pt.nact, (size_t)M);
    if (!rc) rc = dalloc(h, &pt.Xf, (size_t)M);
    for (int b = 0; b < 2 && !rc; ++b) {
        rc = dalloc(h, &pt.Xb[b], 3 * (size_t)M);
        if (!rc) rc = dalloc(h, &pt.Vh[b], 3 * (size_t)M);
    }
    if (!rc) rc = dalloc(h, &pt.nbr, (size_t)M * kMaxNbr);
    if (!rc) rc = dalloc(h, &pt.nbr_cnt, (size_t)M);
    if (!rc && cudaMallocHost((void **)&h->status_host, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        rc = LBM_ERR_NOMEM;
    }
    if (!rc && M > 0 && links_setup(h->tile_ext, h->link_cap) != LBM_OK) rc = LBM_ERR_CUDA;
    // overlapped schedule (spheres only): near tags, second stream, events
    h->overlap = M > 0 && p.schedule == LBM_SCHEDULE_OVERLAP;
    if (!rc && h->overlap) {
        // groups of 64 bytes of a slot row (the DRAM access granularity), so
        // the near and far collides never share one
        h->near_shift = h->esize == 4 ? 4 : 5;
        h->near_ngx = (p.nx + (1 << h->near_shift) - 1) >> h->near_shift;
        h->near_groups = (long long)h->near_ngx * p.ny * p.nz;
        const long long NG = h->near_groups;
        rc = dalloc(h, &h->near[0], (size_t)NG);
        if (!rc) rc = dalloc(h, &h->near[1], (size_t)NG);
        // a sphere tags at most (2 ceil(R + 0.05) + 7)^3 nodes, so as many groups
        const long long e = 2 * (long long)std::ceil(p.max_radius + 0.05) + 7;
        const long long cap = std::min(NG, (long long)M * e * e * e);
        if (!rc) rc = dalloc(h, &h->near_list[0], (size_t)cap);
        if (!rc) rc = dalloc(h, &h->near_list[1], (size_t)cap);
        if (!rc) rc = dalloc(h, &h->near_cnt, 2);
        if (!rc) rc = dalloc(h, &h->far_list[0], (size_t)NG);
        if (!rc) rc = dalloc(h, &h->far_list[1], (size_t)NG);
        if (!rc) rc = dalloc(h, &h->far_cnt, 2);
        bool ok = !rc && cudaStreamCreateWithPriority(&h->stream2, cudaStreamNonBlocking, prio_low) == cudaSuccess;
        cudaEvent_t *evs[] = {&h->ev_cf, &h->ev_nm[0], &h->ev_nm[1], &h->ev_join};
        for (cudaEvent_t *e : evs) ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
        int user_prio = prio_high;
        if (ok && !h->own_stream) ok = cudaStreamGetPriority(h->stream, &user_prio) == cudaSuccess;
        if (ok && user_prio != prio_high)
            ok = cudaStreamCreateWithPriority(&h->chain, cudaStreamNonBlocking, prio_high) == cudaSuccess;
        if (ok)
            ok = cudaMemsetAsync(h->near[0], 0, (size_t)NG, h->stream) == cudaSuccess &&
                 cudaMemsetAsync(h->near[1], 0, (size_t)NG, h->stream) == cudaSuccess;
        if (!ok && !rc) {
            cudaGetLastError();
            rc = LBM_ERR_CUDA;
        }
    }
    if (!rc) {
        int per_sm = 0, sms = 0;
        if (dem_max_blocks(kDemThreads, &per_sm) != LBM_OK ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device) != cudaSuccess)
            rc = LBM_ERR_CUDA;
        h->dem_threads = kDemThreads;
        h->dem_blocks = per_sm * sms;
        h->sms = sms;
        if (!rc && h->dem_blocks < 1) rc = LBM_ERR_CUDA;
        h->dem_cluster = M > 0 ? dem_cluster_setup(M, false, h->pt.fric != 0) : 0;
        h->dem_mode = p.dem_mode;
        h->dem_grid_blocks = M > 0 ? dem_grid_setup(h->pt.fric != 0, sms) : 0;
        const bool grid_fits = h->dem_grid_blocks > 0 && dem_grid_capacity(h->pt.fric != 0, h->dem_grid_blocks) >= M;
        if (!grid_fits) h->dem_grid_blocks = 0;
        // the tangential contact state lives in the cluster and grid forms only
        if (!rc && M > 0 && h->pt.fric && h->dem_cluster == 0 && !grid_fits) rc = LBM_ERR_UNSUPPORTED;
        if (!rc && M > 0 && p.dem_mode == LBM_DEM_CLUSTER && h->dem_cluster == 0) rc = LBM_ERR_UNSUPPORTED;
        if (!rc && M > 0 && p.dem_mode == LBM_DEM_GRID && !grid_fits) rc = LBM_ERR_UNSUPPORTED;
    }
    if (!rc) {
        *h->status_host = 0;
        bool ok = cudaMemsetAsync(h->f, 0, (size_t)Q * h->L.S * h->esize, h->stream) == cudaSuccess &&
                  cudaMemsetAsync(h->flag, 0, (size_t)N, h->stream) == cudaSuccess &&
                  cudaMemsetAsync(h->owner, 0xff, (size_t)N * 4, h->stream) == cudaSuccess &&
                  cudaMemsetAsync(h->status, 0, sizeof(int), h->stream) == cudaSuccess &&
                  cudaMemsetAsync(h->ctr, 0, 4 * sizeof(unsigned long long), h->stream) == cudaSuccess &&
                  cudaStreamSynchronize(h->stream) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            rc = LBM_ERR_CUDA;
        }
    }
    if (rc) {
        release(h);
        delete h;
        return rc;
    }
    *out = h;
    return LBM_OK;
}

int lbm_destroy(lbm_handle h) {
    if (!h || h->batch) return LBM_ERR_ARG;  // batch members go with their batch
    DeviceScope ds(h->device);
    cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
    return LBM_OK;
}

int lbm_set_particles(lbm_handle h, int32_t n, const double *pos, const double *vel, const double *omega,
                      const double *radius, const uint8_t *fixed) {
    if (!h || n < 0) return LBM_ERR_ARG;
    if (n > h->p.max_particles) return LBM_ERR_CAPACITY;
    if (n > 0 && (!pos || !vel || !omega || !radius)) return LBM_ERR_ARG;
    if (n > 0 && (!finite3(pos, n) || !finite3(vel, n) || !finite3(omega, n))) return LBM_ERR_ARG;
    for (int a = 0; a < n; ++a) {
        if (!(radius[a] > 0.0 && radius[a] <= h->p.max_radius)) return LBM_ERR_ARG;
        const double x = pos[3 * a], y = pos[3 * a + 1], z = pos[3 * a + 2];
        if (!(x >= 0.0 && x < h->L.nx && y >= 0.0 && y < h->L.ny && z > -0.5 && z < h->L.nz - 0.5)) return LBM_ERR_ARG;
    }
    if (h->sticky) return h->sticky;
    DeviceScope ds(h->device);
    Parts &pt = h->pt;
    const size_t v3 = 3 * sizeof(double) * (size_t)n;
    int rc = LBM_OK;
    float4 *xf = n ? (float4 *)std::malloc(sizeof(float4) * (size_t)n) : nullptr;
    SFrame *fr = n ? (SFrame *)std::malloc(sizeof(SFrame) * (size_t)n) : nullptr;
    if (n && (!xf || !fr)) {
        std::free(xf);
        std::free(fr);
        return LBM_ERR_NOMEM;
    }
    for (int a = 0; a < n; ++a) {
        xf[a] = make_float4((float)pos[3 * a], (float)pos[3 * a + 1], (float)pos[3 * a + 2], (float)radius[a]);
        // the same operations as the device frame of the DEM commit
        SFrame &F = fr[a];
        for (int c = 0; c < 3; ++c) {
            const double b = std::floor(pos[3 * a + c]);
            F.b[c] = (int)b;
            F.fr[c] = (float)(pos[3 * a + c] - b);
            F.V[c] = (float)vel[3 * a + c];
            F.W[c] = (float)omega[3 * a + c];
        }
        F.R = (float)radius[a];
        F.R2 = F.R * F.R;
        F.pad[0] = F.pad[1] = 0.f;
    }
    if (!rc) rc = copy_in(h, pt.X, pos, v3, LBM_HOST);
    if (!rc) rc = copy_in(h, pt.Xbuild, pos, v3, LBM_HOST);
    if (!rc) rc = copy_in(h, pt.Xf, xf, sizeof(float4) * (size_t)n, LBM_HOST);
    if (!rc) rc = copy_in(h, pt.frame[0], fr, sizeof(SFrame) * (size_t)n, LBM_HOST);
    if (!rc) rc = copy_in(h, pt.frame[1], fr, sizeof(SFrame) * (size_t)n, LBM_HOST);
    if (!rc && n && cudaMemsetAsync(pt.rebuild, 0, 2 * sizeof(int), h->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    if (!rc) rc = copy_in(h, pt.V, vel, v3, LBM_HOST);
    if (!rc) rc = copy_in(h, pt.W, omega, v3, LBM_HOST);
    if (!rc) rc = copy_in(h, pt.R, radius, sizeof(double) * (size_t)n, LBM_HOST);
    if (!rc && n) {
        if (fixed)
            rc = copy_in(h, (void *)pt.fixed, fixed, (size_t)n, LBM_HOST);
        else if (cudaMemsetAsync((void *)pt.fixed, 0, (size_t)n, h->stream) != cudaSuccess)
            rc = LBM_ERR_CUDA;
    }
    double *zero[] = {pt.Fh, pt.Th, pt.Fc, pt.Fx, pt.Tx, pt.Fcorr, pt.Tcorr, pt.Tc};
    for (double *z : zero)
        if (!rc && n && cudaMemsetAsync(z, 0, v3, h->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    if (!rc && n && pt.fric &&
        (cudaMemsetAsync(pt.tmask, 0, sizeof(unsigned long long) * (size_t)n, h->stream) != cudaSuccess ||
         cudaMemsetAsync(pt.tdisp, 0, sizeof(float4) * (size_t)n * kMaxNbr, h->stream) != cudaSuccess ||
         cudaMemsetAsync(pt.twall, 0, sizeof(float4) * 2 * (size_t)n, h->stream) != cudaSuccess))
        rc = LBM_ERR_CUDA;
    if (!rc && cudaMemsetAsync(h->f, 0, (size_t)Q * h->L.S * h->esize, h->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    if (!rc && cudaMemsetAsync(h->flag, 0, (size_t)h->L.N, h->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    if (!rc && cudaMemsetAsync(h->owner, 0xff, (size_t)h->L.N * 4, h->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    if (!rc && cudaMemsetAsync(h->ctr, 0, 4 * sizeof(unsigned long long), h->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    pt.np = n;
    h->parity = 0;
    h->steps = 0;
    if (!rc && h->zieb) rc = zieb_reset(h, h->zvp);  // the cylinder starts at rest with the fluid
    if (!rc && n) rc = launch_neighbours(h, 1);
    if (!rc && n) rc = launch_mark(h, h->parity, 0);
    if (!rc && n) rc = launch_contact(h);
    if (!rc && n && h->overlap) {
        // near set of step 0 from the initial centres; events in a recorded state
        if (cudaMemsetAsync(h->near[0], 0, (size_t)h->near_groups, h->stream) != cudaSuccess ||
            cudaMemsetAsync(h->near[1], 0, (size_t)h->near_groups, h->stream) != cudaSuccess)
            rc = LBM_ERR_CUDA;
        if (!rc)
            rc = launch_near_mark(h, h->near[0], near_tag(0), h->pt.frame[0], h->near_list[0], h->near_cnt,
                                  h->far_list[0], h->far_cnt, h->stream);
        cudaEvent_t evs[] = {h->ev_cf, h->ev_nm[0], h->ev_nm[1]};
        for (cudaEvent_t e : evs)
            if (!rc && cudaEventRecord(e, h->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    }
    if (!rc) rc = settle(h);
    if (h->batch) h->batch->dirty = true;  // sphere counts and grids change
    h->graph_stale = true;
    std::free(xf);
    std::free(fr);
    if (rc == LBM_ERR_CUDA && !h->sticky) h->sticky = rc;
    return rc;
}

int lbm_set_particle_load(lbm_handle h, const double *force, const double *torque, int32_t where) {
    if (!h || (where != LBM_HOST && where != LBM_DEVICE)) return LBM_ERR_ARG;
    if (where == LBM_HOST && h->pt.np > 0 &&
        ((force && !finite3(force, h->pt.np)) || (torque && !finite3(torque, h->pt.np))))
        return LBM_ERR_ARG;
    if (h->sticky) return h->sticky;
    DeviceScope ds(h->device);
    const size_t v3 = 3 * sizeof(double) * (size_t)h->pt.np;
    int rc = LBM_OK;
    // host values: staged in pinned memory first (the caller may reuse its
    // buffers as soon as we return), copied to the device in stream order
    double *stage = nullptr;
    if (where == LBM_HOST && v3 && (force || torque)) {
        const int k = h->load_slot;
        if (!h->load_stage[k]) {
            const size_t cap = 6 * sizeof(double) * (size_t)(h->p.max_particles > 0 ? h->p.max_particles : 1);
            if (cudaMallocHost((void **)&h->load_stage[k], cap) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->load_ev[k], cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                return LBM_ERR_NOMEM;
            }
        } else if (cudaEventSynchronize(h->load_ev[k]) != cudaSuccess) {  // its last copy is done
            return LBM_ERR_CUDA;
        }
        stage = h->load_stage[k];
        if (force) std::memcpy(stage, force, v3);
        if (torque) std::memcpy(stage + 3 * (size_t)h->pt.np, torque, v3);
    }
    if (force)
        rc = copy_in(h, h->pt.Fx, stage ? stage : force, v3, where);
    else if (v3 && cudaMemsetAsync(h->pt.Fx, 0, v3, h->stream) != cudaSuccess)
        rc = LBM_ERR_CUDA;
    if (!rc) {
        if (torque)
            rc = copy_in(h, h->pt.Tx, stage ? stage + 3 * (size_t)h->pt.np : torque, v3, where);
        else if (v3 && cudaMemsetAsync(h->pt.Tx, 0, v3, h->stream) != cudaSuccess)
            rc = LBM_ERR_CUDA;
    }
    if (!rc && stage) {
        if (cudaEventRecord(h->load_ev[h->load_slot], h->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
        h->load_slot ^= 1;
    }
    if (rc) cudaGetLastError();
    return rc;
}

int lbm_set_populations(lbm_handle h, const double *f, int32_t where) {
    if (!h || !f || (where != LBM_HOST && where != LBM_DEVICE)) return LBM_ERR_ARG;
    if (h->sticky) return h->sticky;
    DeviceScope ds(h->device);
    const size_t n = (size_t)Q * h->L.N * sizeof(double);
    int rc = LBM_OK;
    if (where == LBM_DEVICE) {
        rc = launch_set_populations(h, f, h->parity);
    } else {
        void *tmp = nullptr;
        if (cudaMallocAsync(&tmp, n, h->stream) != cudaSuccess) {
            cudaGetLastError();
            return LBM_ERR_NOMEM;
        }
        rc = copy_in(h, tmp, f, n, LBM_HOST);
        if (!rc) rc = launch_set_populations(h, (const double *)tmp, h->parity);
        cudaFreeAsync(tmp, h->stream);
    }
    const int s = settle(h);
    return rc ? rc : s;
}

namespace {

// One serial step with spheres at the handle's current parity (no profiler
// marks), as captured into a step graph: after the marks (which read the
// neighbour lists) the lists are rebuilt on a side branch, concurrently with
// refill, collide and links (which do not read them); the DEM waits for both.
int serial_step_launches(lbm_s *h) {
    const int P = h->parity;
    auto ok = [](cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA; };
    int rc = launch_mark(h, P, h->pt.corr);
    if (!rc) rc = ok(cudaEventRecord(h->ev_fork, h->stream));
    if (!rc) rc = ok(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    if (!rc) rc = launch_neighbours(h, 0, h->side);
    if (!rc) rc = ok(cudaEventRecord(h->ev_nbr, h->side));
    if (!rc) rc = launch_refill(h, P);
    if (!rc) rc = launch_stream_collide(h, P);
    if (!rc) rc = launch_links(h, P, true);
    if (!rc && h->zieb) rc = launch_zieb(h, P);
    if (!rc) rc = ok(cudaStreamWaitEvent(h->stream, h->ev_nbr, 0));
    if (!rc) rc = launch_dem(h);
    return rc;
}

// Capture the serial step of each parity into a graph (the launchers read
// the parity and the step parity from the handle, so both are set for the
// capture and restored).
int capture_step_graphs(lbm_s *h) {
    if (!h->side) {
        if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_nbr, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return LBM_ERR_CUDA;
        }
    }
    for (cudaGraphExec_t &g : h->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    const int P0 = h->parity;
    const long long s0 = h->steps;
    int rc = LBM_OK;
    for (int k = 0; k < 2 && !rc; ++k) {
        const int P = P0 ^ k;
        h->parity = P;
        h->steps = s0 + k;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            rc = LBM_ERR_CUDA;
            break;
        }
        const int r = serial_step_launches(h);
        const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
        if (r || e != cudaSuccess) rc = r ? r : LBM_ERR_CUDA;
        if (!rc && cudaGraphInstantiate(&h->graph[P], g, 0) != cudaSuccess) rc = LBM_ERR_CUDA;
        if (g) cudaGraphDestroy(g);
    }
    h->parity = P0;
    h->steps = s0;
    if (rc) {
        cudaGetLastError();
        for (cudaGraphExec_t &g : h->graph)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
        return rc;
    }
    h->graph_stale = false;
    return LBM_OK;
}

}  // namespace

int lbm_step(lbm_handle h, int32_t nsteps) {
    if (!h || nsteps < 0 || h->batch) return LBM_ERR_ARG;  // batch members step through lbm_batch_step
    if (h->sticky) return h->sticky;
    const int polled = status_to_code(*h->status_host);  // mirror of an earlier call
    if (polled) {
        h->sticky = polled;
        return polled;
    }
    DeviceScope ds(h->device);
    int rc = LBM_OK;
    const bool parts = h->pt.np > 0;
    const bool ovl = parts && h->overlap;
    auto ok = [](cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA; };
    // the main-stream work runs on the high-priority `chain` stream, after
    // and before the caller's stream
    cudaStream_t user = h->stream;
    const bool handover = ovl && h->chain;
    if (handover) {
        rc = ok(cudaEventRecord(h->ev_join, user));
        if (!rc) rc = ok(cudaStreamWaitEvent(h->chain, h->ev_join, 0));
        if (!rc) h->stream = h->chain;
    }
    cudaStream_t A = h->stream, Bs = h->stream2;
    // Serial steps with spheres, unprofiled: replay the captured step graphs
    // (the captures need a stream other than the legacy default stream; they
    // are kept until the spheres are set again, so single steps replay them
    // too).
    if (!rc && parts && !ovl && !h->prof && nsteps >= 1 && h->stream) {
        if (h->graph_stale || !h->graph[0] || !h->graph[1]) rc = capture_step_graphs(h);
        for (int it = 0; it < nsteps && !rc; ++it) {
            // the link / refill counters report the last step of the call
            if (it == nsteps - 1) rc = ok(cudaMemsetAsync(h->ctr, 0, 2 * sizeof(unsigned long long), A));
            if (!rc) rc = ok(cudaGraphLaunch(h->graph[h->parity], A));
            if (!rc) {
                h->parity ^= 1;
                ++h->steps;
            }
        }
        nsteps = 0;  // done
    }
    // everything the caller enqueued since the last step (populations set,
    // loads, ...) precedes this call's far collisions
    if (ovl && !rc) rc = ok(cudaEventRecord(h->ev_nm[h->steps & 1], A));
    for (int it = 0; it < nsteps && !rc; ++it) {
        const int P = h->parity;
        const long long s = h->steps;
        const int cur = (int)(s & 1), nxt = (int)((s + 1) & 1);
        if (h->prof && h->ev_used == h->ev_cap) rc = prof_flush(h);
        if (!rc && it == nsteps - 1) rc = ok(cudaMemsetAsync(h->ctr, 0, 2 * sizeof(unsigned long long), A));
        if (ovl) {
            // second stream: the far-node collisions of step s, once the
            // near tags of step s exist (recorded after step s-1's near
            // collisions); far nodes touch nothing the link / DEM / geometry
            // work of steps s-1, s and the near collisions of step s touch
            if (!rc) rc = ok(cudaStreamWaitEvent(Bs, h->ev_nm[cur], 0));
            if (!rc) rc = prof_mark(h, E6, Bs);
            if (!rc) rc = launch_collide_list(h, P, h->far_list[cur], h->far_cnt + cur, Bs);
            if (!rc) rc = prof_mark(h, E7, Bs);
            if (!rc) rc = ok(cudaEventRecord(h->ev_cf, Bs));
        }
        if (!rc) rc = prof_mark(h, E0, A);
        if (!rc && parts) rc = launch_mark(h, P, h->pt.corr);
        if (!rc && parts) rc = launch_refill(h, P);
        if (!rc) rc = prof_mark(h, E1, A);
        if (ovl) {
            if (!rc) rc = launch_collide_list(h, P, h->near_list[cur], h->near_cnt + cur, A);
            if (!rc) rc = prof_mark(h, E2, A);
            // near tags and list of step s+1 from the centres step s uses,
            // while the far collisions of step s run
            if (!rc && near_tag(s + 1) == 1) rc = ok(cudaMemsetAsync(h->near[nxt], 0, (size_t)h->near_groups, A));
            if (!rc)
                rc = launch_near_mark(h, h->near[nxt], near_tag(s + 1), h->pt.frame[cur], h->near_list[nxt],
                                      h->near_cnt + nxt, h->far_list[nxt], h->far_cnt + nxt, A);
            if (!rc) rc = ok(cudaEventRecord(h->ev_nm[nxt], A));
            if (!rc) rc = ok(cudaStreamWaitEvent(A, h->ev_cf, 0));
        } else {
            if (!rc) rc = launch_stream_collide(h, P);
            if (!rc) rc = prof_mark(h, E2, A);
            if (!rc && h->prof) rc = prof_mark(h, E6, A);
            if (!rc && h->prof) rc = prof_mark(h, E7, A);
        }
        if (!rc) rc = prof_mark(h, E3, A);
        if (!rc && parts) rc = launch_links(h, P);
        if (!rc && h->zieb) rc = launch_zieb(h, P);
        if (!rc) rc = prof_mark(h, E4, A);
        if (!rc && parts) rc = launch_neighbours(h, 0);
        if (!rc && parts) rc = launch_dem(h);
        if (!rc) rc = prof_mark(h, E5, A);
        if (!rc) {
            if (h->prof) ++h->ev_used;
            h->parity ^= 1;
            ++h->steps;
        }
    }
    if (handover && h->stream == h->chain) {
        h->stream = user;
        const int r2 = ok(cudaEventRecord(h->ev_join, h->chain));
        const int r3 = r2 ? r2 : ok(cudaStreamWaitEvent(user, h->ev_join, 0));
        if (!rc) rc = r3;
    }
    if (!rc && cudaMemcpyAsync(h->status_host, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        rc = LBM_ERR_CUDA;
    if (rc) {
        cudaGetLastError();
        if (!h->sticky) h->sticky = rc;
    }
    return rc;
}

int lbm_forces(lbm_handle h, double *F, double *T, int32_t where) {
    if (!h || (where != LBM_HOST && where != LBM_DEVICE)) return LBM_ERR_ARG;
    DeviceScope ds(h->device);
    const size_t v3 = 3 * sizeof(double) * (size_t)h->pt.np;
    int rc = copy_out(h, F, h->pt.Fh, v3, where);
    if (!rc) rc = copy_out(h, T, h->pt.Th, v3, where);
    const int s = settle(h);
    return rc ? rc : s;
}

int lbm_particles(lbm_handle h, double *pos, double *vel, double *omega, int32_t where) {
    if (!h || (where != LBM_HOST && where != LBM_DEVICE)) return LBM_ERR_ARG;
    DeviceScope ds(h->device);
    const size_t v3 = 3 * sizeof(double) * (size_t)h->pt.np;
    int rc = copy_out(h, pos, h->pt.X, v3, where);
    if (!rc) rc = copy_out(h, vel, h->pt.V, v3, where);
    if (!rc) rc = copy_out(h, omega, h->pt.W, v3, where);
    const int s = settle(h);
    return rc ? rc : s;
}

int lbm_particle_state(lbm_handle h, double *F, double *T, double *pos, double *vel, double *omega,
                       int32_t where) {
    if (!h || (where != LBM_HOST && where != LBM_DEVICE)) return LBM_ERR_ARG;
    DeviceScope ds(h->device);
    const size_t v3 = 3 * sizeof(double) * (size_t)h->pt.np;
    int rc = copy_out(h, F, h->pt.Fh, v3, where);
    if (!rc) rc = copy_out(h, T, h->pt.Th, v3, where);
    if (!rc) rc = copy_out(h, pos, h->pt.X, v3, where);
    if (!rc) rc = copy_out(h, vel, h->pt.V, v3, where);
    if (!rc) rc = copy_out(h, omega, h->pt.W, v3, where);
    const int s = settle(h);
    return rc ? rc : s;
}

int lbm_fields(lbm_handle h, float *rho, float *u, int32_t where) {
    if (!h || (where != LBM_HOST && where != LBM_DEVICE)) return LBM_ERR_ARG;
    DeviceScope ds(h->device);
    const long long N = h->L.N;
    int rc = LBM_OK;
    if (where == LBM_DEVICE) {
        rc = launch_fields(h, rho, u, h->parity);
    } else {
        float *tmp = nullptr;
        if (cudaMallocAsync((void **)&tmp, 4 * sizeof(float) * (size_t)N, h->stream) != cudaSuccess) {
            cudaGetLastError();
            return LBM_ERR_NOMEM;
        }
        rc = launch_fields(h, tmp, tmp + N, h->parity);
        if (!rc && rho) rc = copy_out(h, rho, tmp, sizeof(float) * (size_t)N, LBM_HOST);
        if (!rc && u) rc = copy_out(h, u, tmp + N, 3 * sizeof(float) * (size_t)N, LBM_HOST);
        cudaFreeAsync(tmp, h->stream);
    }
    const int s = settle(h);
    return rc ? rc : s;
}

int lbm_populations(lbm_handle h, double *f, int32_t where) {
    if (!h || !f || (where != LBM_HOST && where != LBM_DEVICE)) return LBM_ERR_ARG;
    DeviceScope ds(h->device);
    const size_t n = (size_t)Q * h->L.N * sizeof(double);
    int rc = with_out_buffer(h, f, n, where, [&](void *d) { return launch_get_populations(h, (double *)d, h->parity); });
    const int s = settle(h);
    return rc ? rc : s;
}

int lbm_geometry(lbm_handle h, int32_t *owner, int32_t where) {
    if (!h || !owner || (where != LBM_HOST && where != LBM_DEVICE)) return LBM_ERR_ARG;
    DeviceScope ds(h->device);
    const size_t n = (size_t)h->L.N * sizeof(int32_t);
    int rc = with_out_buffer(h, owner, n, where, [&](void *d) { return launch_owner(h, (int32_t *)d); });
    const int s = settle(h);
    return rc ? rc : s;
}

int lbm_info(lbm_handle h, lbm_info_t *info) {
    if (!h || !info) return LBM_ERR_ARG;
    DeviceScope ds(h->device);
    unsigned long long c[4] = {0, 0, 0, 0};
    int rc = cudaMemsetAsync(h->ctr + 2, 0, sizeof(unsigned long long), h->stream) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
    if (!rc) rc = launch_count_fluid(h);
    if (!rc) rc = copy_out(h, c, h->ctr, sizeof(c), LBM_HOST);
    const int s = settle(h);
    std::memset(info, 0, sizeof(*info));
    info->nodes = h->L.N;
    info->fluid_nodes = (int64_t)c[2];
    info->links = (int64_t)c[0];
    info->refilled = (int64_t)c[1];
    info->steps = h->steps;
    info->particles = h->pt.np;
    info->precision = h->precision;
    info->device_bytes = (int64_t)h->bytes;
    return rc ? rc : s;
}

int lbm_zieb_state(lbm_handle h, double *out) {
    if (!h || !out || !h->zieb) return LBM_ERR_ARG;
    DeviceScope ds(h->device);
    const int P = h->parity;  // the slot the last step wrote
    double z[5];
    std::vector<double> part(h->zblocks);
    std::vector<int> cnt(h->zblocks);
    int rc = copy_out(h, z, h->zs, sizeof(z), LBM_HOST);
    if (!rc) rc = copy_out(h, part.data(), h->zpart + (size_t)P * h->zblocks, sizeof(double) * h->zblocks, LBM_HOST);
    if (!rc) rc = copy_out(h, cnt.data(), h->zcnt + (size_t)P * h->zblocks, sizeof(int) * h->zblocks, LBM_HOST);
    const int s = settle(h);
    if (rc || s) return rc ? rc : s;
    double su = 0.0;
    long long sc = 0;
    for (int b = 0; b < h->zblocks; ++b) {
        su += part[b];
        sc += cnt[b];
    }
    out[0] = z[P];
    out[1] = z[2 + P];
    out[2] = sc ? su / (double)sc : 0.0;
    return LBM_OK;
}

int lbm_zieb_set_piston(lbm_handle h, double vp) {
    if (!h || !h->zieb || !std::isfinite(vp)) return LBM_ERR_ARG;
    DeviceScope ds(h->device);
    int rc = copy_in(h, h->zs + 4, &vp, sizeof(double), LBM_HOST);
    const int s = settle(h);  // vp lives on this stack frame until the copy is done
    if (!rc && !s) h->zvp = vp;
    return rc ? rc : s;
}

int lbm_profile(lbm_handle h, int32_t enable) {
    if (!h) return LBM_ERR_ARG;
    DeviceScope ds(h->device);
    if (enable && !h->ev) {
        h->ev = (cudaEvent_t *)std::calloc(kProfEv * (size_t)kProfSteps, sizeof(cudaEvent_t));
        if (!h->ev) return LBM_ERR_NOMEM;
        for (int i = 0; i < kProfEv * kProfSteps; ++i)
            if (cudaEventCreate(&h->ev[i]) != cudaSuccess) {
                cudaGetLastError();
                for (int j = 0; j < i; ++j) cudaEventDestroy(h->ev[j]);
                std::free(h->ev);
                h->ev = nullptr;
                return LBM_ERR_CUDA;
            }
        h->ev_cap = kProfSteps;
    }
    int rc = LBM_OK;
    if (h->prof && !enable) rc = prof_flush(h);
    if (enable) {
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
        h->ev_used = 0;
        h->prof_steps = 0;
        for (double &m : h->prof_ms) m = 0.0;
    }
    h->prof = enable != 0;
    return rc;
}

int lbm_profile_read(lbm_handle h, double *ms, int64_t *steps) {
    if (!h) return LBM_ERR_ARG;
    DeviceScope ds(h->device);
    const int rc = prof_flush(h);
    if (ms)
        for (int i = 0; i < LBM_PHASES; ++i) ms[i] = h->prof_ms[i];
    if (steps) *steps = h->prof_steps;
    return rc;
}

int lbm_sync(lbm_handle h) {
    if (!h) return LBM_ERR_ARG;
    DeviceScope ds(h->device);
    return settle(h);
}

int lbm_selftest_wait(lbm_handle h) {
    if (!h) return LBM_ERR_ARG;
    DeviceScope ds(h->device);
    const int rc = launch_wait_probe(h);
    const int s = settle(h);
    return rc ? rc : s;
}

}  // extern "C"

// ---- batched form -----------------------------------------------------------

namespace {

void batch_release(lbm_batch_s *b) {
    for (cudaGraphExec_t &g : b->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    if (b->dinst) cudaFree(b->dinst);
    if (b->chunks) cudaFree(b->chunks);
    delete b->ctab;
    b->ctab = nullptr;
    b->dinst = nullptr;
    b->chunks = nullptr;
    if (b->m) {
        for (int i = 0; i < b->n; ++i)
            if (b->m[i]) {
                b->m[i]->batch = nullptr;
                lbm_destroy(b->m[i]);
            }
        delete[] b->m;
        b->m = nullptr;
    }
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    b->stream = nullptr;
}

// Chunk table: TPB consecutive nodes of one instance per entry.
int batch_chunks(const lbm_batch_s *b, int tpb, int2 **out, int *count) {
    std::vector<int2> c;
    for (int i = 0; i < b->n; ++i)
        for (long long n0 = 0; n0 < b->m[i]->L.N; n0 += tpb) c.push_back(make_int2(i, (int)n0));
    *out = nullptr;
    *count = (int)c.size();
    if (c.empty()) return LBM_OK;
    if (cudaMalloc((void **)out, c.size() * sizeof(int2)) != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return LBM_ERR_NOMEM;
    }
    if (cudaMemcpy(*out, c.data(), c.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(*out);
        *out = nullptr;
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

// Descriptors of the members' current state (sphere counts, pointers).
int batch_descriptors(lbm_batch_s *b) {
    std::vector<Inst> I((size_t)b->n);
    b->max_np = 0;
    for (int i = 0; i < b->n; ++i) {
        const lbm_s *h = b->m[i];
        Inst &a = I[i];
        a.L = h->L;
        a.ph = h->ph;
        a.pt = h->pt;
        a.f = h->f;
        a.flag = h->flag;
        a.owner = h->owner;
        a.status = h->status;
        a.ctr = h->ctr;
        a.dnx = FastDiv((unsigned)h->L.nx);
        a.dny = FastDiv((unsigned)h->L.ny);
        b->max_np = std::max(b->max_np, h->pt.np);
    }
    if (cudaMemcpy(b->dinst, I.data(), I.size() * sizeof(Inst), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    if (b->n <= kCollideTable) {
        if (!b->ctab) b->ctab = new (std::nothrow) CollideTable();
        if (!b->ctab) return LBM_ERR_NOMEM;
        for (int i = 0; i < b->n; ++i) {
            CInst &c = b->ctab->c[i];
            c.L = I[i].L;
            c.ph = I[i].ph;
            c.f = I[i].f;
            c.flag = I[i].flag;
            c.status = I[i].status;
            c.dnx = I[i].dnx;
            c.dny = I[i].dny;
        }
    }
    return LBM_OK;
}

// One lattice step of every member, parity P (= step parity).
int batch_enqueue(const lbm_batch_s *b, int P) {
    int rc = launch_mark_batch(b, P);
    if (!rc) rc = launch_refill_batch(b, P);
    if (!rc) rc = launch_collide_batch(b, P, b->tpb, b->minb, b->grid, b->chunks, b->nchunks);
    if (!rc) rc = launch_links_batch(b, P);
    if (!rc) rc = launch_neighbours_batch(b, P);
    if (!rc) rc = launch_dem_batch(b, P);
    return rc;
}

int batch_capture(lbm_batch_s *b, int P, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    const int rc = batch_enqueue(b, P);
    const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc ? rc : LBM_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

// Descriptors, chunk table of the tuned block size, and the two step graphs.
int batch_prepare(lbm_batch_s *b) {
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    for (cudaGraphExec_t &g : b->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    int rc = batch_descriptors(b);
    if (!rc && b->chunk_tpb != b->tpb) {
        if (b->chunks) cudaFree(b->chunks);
        b->chunks = nullptr;
        rc = batch_chunks(b, b->tpb, &b->chunks, &b->nchunks);
        b->chunk_tpb = rc ? 0 : b->tpb;
    }
    for (int P = 0; P < 2 && !rc; ++P) rc = batch_capture(b, P, &b->graph[P]);
    if (!rc) b->dirty = false;
    return rc;
}

// Members' common step parity, or -1 if they differ (or a member failed).
int batch_parity(const lbm_batch_s *b, int *err) {
    int P = -1;
    *err = LBM_OK;
    for (int i = 0; i < b->n; ++i) {
        lbm_s *h = b->m[i];
        if (h->sticky) {
            *err = h->sticky;
            return -1;
        }
        const int polled = status_to_code(*h->status_host);
        if (polled) {
            h->sticky = polled;
            *err = polled;
            return -1;
        }
        if (P < 0) P = h->parity;
        if (h->parity != P) {
            *err = LBM_ERR_ARG;
            return -1;
        }
    }
    return P;
}

}  // namespace

extern "C" {

int lbm_batch_create(const lbm_params *params, int32_t count, lbm_batch *out) {
    if (!params || !out || count < 1) return LBM_ERR_ARG;
    *out = nullptr;
    for (int i = 1; i < count; ++i)
        if (params[i].device != params[0].device || params[i].precision != params[0].precision ||
            params[i].cuda_stream != params[0].cuda_stream)
            return LBM_ERR_ARG;
    // Each link CTA scans its own sphere's tile (extent ceil(R) + 2, within
    // that of its member's max_radius), which the member's own box rule in
    // lbm_create keeps from wrapping onto itself; only the link kernel's
    // shared memory is sized for the batch's largest tile.
    lbm_batch_s *b = new (std::nothrow) lbm_batch_s();
    if (!b) return LBM_ERR_NOMEM;
    b->device = params[0].device;
    b->precision = params[0].precision;
    DeviceScope ds(b->device);
    if (cudaSetDevice(b->device) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return LBM_ERR_CUDA;
    }
    int rc = LBM_OK;
    if (params[0].cuda_stream) {
        b->stream = (cudaStream_t)params[0].cuda_stream;
    } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess) {
        b->own_stream = true;
    } else {
        cudaGetLastError();
        rc = LBM_ERR_CUDA;
    }
    b->m = rc ? nullptr : new (std::nothrow) lbm_s *[count]();
    if (!rc && !b->m) rc = LBM_ERR_NOMEM;
    if (!rc) b->n = count;
    int max_m = 0;
    for (int i = 0; i < count && !rc; ++i) {
        lbm_params p = params[i];
        p.cuda_stream = b->stream;
        p.schedule = LBM_SCHEDULE_SERIAL;
        rc = lbm_create(&p, &b->m[i]);
        if (rc) {
            b->m[i] = nullptr;
            break;
        }
        b->m[i]->batch = b;
        if (b->m[i]->zieb) {  // the face update is not part of the batched step
            rc = LBM_ERR_UNSUPPORTED;
            break;
        }
        if (p.max_particles > 0) {
            b->ext = std::max(b->ext, b->m[i]->tile_ext);
            b->cap = std::max(b->cap, b->m[i]->link_cap);
            max_m = std::max(max_m, p.max_particles);
        }
    }
    if (!rc && max_m > 0) {
        for (int i = 0; i < count; ++i) b->fric = b->fric || b->m[i]->pt.fric != 0;
        b->dem_cluster = dem_cluster_setup(max_m, true, b->fric);
        if (b->dem_cluster == 0) rc = LBM_ERR_UNSUPPORTED;  // the batched DEM needs one cluster per instance
        if (!rc) rc = dem_cluster_setup_batch(b->dem_cluster, b->fric);
        if (!rc) rc = links_setup_batch(b->ext, b->cap);
    }
    if (!rc && cudaMalloc((void **)&b->dinst, sizeof(Inst) * (size_t)count) != cudaSuccess) {
        cudaGetLastError();
        rc = LBM_ERR_NOMEM;
    }
    if (!rc && cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
        cudaGetLastError();
        rc = LBM_ERR_CUDA;
    }
    if (rc) {
        batch_release(b);
        delete b;
        return rc;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch b) {
    if (!b) return LBM_ERR_ARG;
    DeviceScope ds(b->device);
    cudaStreamSynchronize(b->stream);
    batch_release(b);
    delete b;
    return LBM_OK;
}

int lbm_batch_handle(lbm_batch b, int32_t i, lbm_handle *out) {
    if (!b || !out || i < 0 || i >= b->n) return LBM_ERR_ARG;
    *out = b->m[i];
    return LBM_OK;
}

int lbm_batch_tune(lbm_batch b, int32_t *threads, int32_t *blocks, float *ms) {
    if (!b) return LBM_ERR_ARG;
    DeviceScope ds(b->device);
    int err = LBM_OK;
    const int P = batch_parity(b, &err);
    if (P < 0) return err;
    // the trial launches collide the members' real state: keep a copy and put it back
    size_t total = 0;
    std::vector<size_t> off((size_t)b->n);
    for (int i = 0; i < b->n; ++i) {
        const lbm_s *h = b->m[i];
        off[i] = total;
        total += (size_t)Q * h->L.S * h->esize + (size_t)h->L.N + sizeof(int);
        total = (total + 255) & ~(size_t)255;
    }
    unsigned char *save = nullptr;
    if (cudaMalloc((void **)&save, total) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_NOMEM;
    }
    auto copy_state = [&](bool back) {
        for (int i = 0; i < b->n; ++i) {
            const lbm_s *h = b->m[i];
            const size_t fb = (size_t)Q * h->L.S * h->esize;
            unsigned char *s = save + off[i];
            void *dev[3] = {h->f, h->flag, h->status};
            const size_t sz[3] = {fb, (size_t)h->L.N, sizeof(int)};
            unsigned char *sv[3] = {s, s + fb, s + fb + h->L.N};
            for (int k = 0; k < 3; ++k) {
                const cudaError_t e = back ? cudaMemcpyAsync(dev[k], sv[k], sz[k], cudaMemcpyDeviceToDevice, b->stream)
                                           : cudaMemcpyAsync(sv[k], dev[k], sz[k], cudaMemcpyDeviceToDevice, b->stream);
                if (e != cudaSuccess) return LBM_ERR_CUDA;
            }
        }
        return LBM_OK;
    };
    int rc = batch_descriptors(b);
    if (!rc) rc = copy_state(false);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = LBM_ERR_CUDA;
    float best = 1e30f;
    int best_tpb = 0, best_minb = 0, best_grid = 0;
    const int shapes[6][2] = {{128, 8}, {128, 6}, {256, 4}, {256, 3}, {512, 2}, {512, 1}};
    for (const auto &sh : shapes) {
        if (rc) break;
        const int tpb = sh[0], minb = sh[1];
        int2 *ch = nullptr;
        int nch = 0, bps = 0;
        rc = batch_chunks(b, tpb, &ch, &nch);
        if (!rc) rc = collide_batch_occupancy(b->precision, P, tpb, minb, &bps, b->ctab != nullptr);
        if (!rc && nch > 0 && bps > 0) {
            // persistent grids of 1/2 and 1 times the resident blocks, and one block per chunk
            const int cands[3] = {std::max(1, b->sms * bps / 2), b->sms * bps, nch};
            for (int c = 0; c < 3 && !rc; ++c) {
                const int grid = std::min(cands[c], nch);
                rc = launch_collide_batch(b, P, tpb, minb, grid, ch, nch);  // warm-up
                if (!rc && cudaEventRecord(e0, b->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
                for (int r = 0; r < 3 && !rc; ++r) rc = launch_collide_batch(b, P, tpb, minb, grid, ch, nch);
                if (!rc && cudaEventRecord(e1, b->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
                float t = 0.f;
                if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
                    rc = LBM_ERR_CUDA;
                if (!rc && t / 3.f < best) {
                    best = t / 3.f;
                    best_tpb = tpb;
                    best_minb = minb;
                    best_grid = grid;
                }
            }
        }
        if (ch) cudaFree(ch);
    }
    const int rb = copy_state(true);
    if (!rc) rc = rb;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess && !rc) rc = LBM_ERR_CUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(save);
    if (rc) {
        cudaGetLastError();
        return rc;
    }
    if (best_tpb == 0) {  // nothing to collide: any launch shape does
        best_tpb = 256;
        best_minb = 4;
        best_grid = 1;
        best = 0.f;
    }
    b->tpb = best_tpb;
    b->minb = best_minb;
    b->grid = best_grid;
    b->dirty = true;
    if (threads) *threads = best_tpb;
    if (blocks) *blocks = best_grid;
    if (ms) *ms = best;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch b, int32_t nsteps) {
    if (!b || nsteps < 0) return LBM_ERR_ARG;
    DeviceScope ds(b->device);
    int err = LBM_OK;
    int P = batch_parity(b, &err);
    if (P < 0) return err;
    int rc = LBM_OK;
    if (!b->tpb) rc = lbm_batch_tune(b, nullptr, nullptr, nullptr);
    if (!rc && b->dirty) rc = batch_prepare(b);
    for (int it = 0; it < nsteps && !rc; ++it) {
        if (cudaGraphLaunch(b->graph[P], b->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
        if (!rc) {
            for (int i = 0; i < b->n; ++i) {
                b->m[i]->parity ^= 1;
                ++b->m[i]->steps;
            }
            P ^= 1;
        }
    }
    for (int i = 0; i < b->n && !rc; ++i) {
        lbm_s *h = b->m[i];
        if (cudaMemcpyAsync(h->status_host, h->status, sizeof(int), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
            rc = LBM_ERR_CUDA;
    }
    if (rc) {
        cudaGetLastError();
        for (int i = 0; i < b->n; ++i)
            if (!b->m[i]->sticky) b->m[i]->sticky = rc;
    }
    return rc;
}

int lbm_batch_sync(lbm_batch b) {
    if (!b) return LBM_ERR_ARG;
    DeviceScope ds(b->device);
    int rc = LBM_OK;
    for (int i = 0; i < b->n; ++i) {
        const int r = settle(b->m[i]);
        if (!rc) rc = r;
    }
    return rc;
}

}  // extern "C"
