// C ABI (include/lbm.h): validation, device allocation, launch order of one
// step, and copies in and out.  No arithmetic of the method lives here.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "lbm_internal.cuh"

using namespace lbm;

namespace {

constexpr int kMaxNbr = 48;
constexpr int kDemThreads = 128;   // fallback cooperative DEM
constexpr double kSkin = 1.5;      // neighbour-list skin (lattice units)
constexpr double kMaxStep = 0.25;  // largest displacement of a sphere in one step

int status_to_code(int st) {
    if (st & ST_TIMEOUT) return LBM_ERR_TIMEOUT;
    if (st & ST_DIVERGED) return LBM_ERR_DIVERGED;
    if (st & (ST_NBR_OVERFLOW | ST_TILE)) return LBM_ERR_CAPACITY;
    if (st & ST_FAST) return LBM_ERR_GEOMETRY;
    return LBM_OK;
}

struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int d) {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceScope() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

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
                    h->pt.pairB, h->pt.Xbuild, h->pt.rebuild, h->pt.frame[0], h->pt.frame[1]};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->status_host) cudaFreeHost(h->status_host);
    if (h->ev) {
        for (int i = 0; i < 5 * h->ev_cap; ++i) cudaEventDestroy(h->ev[i]);
        std::free(h->ev);
        h->ev = nullptr;
    }
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

constexpr int kProfSteps = 2048;

// Fold the recorded events into the phase totals (synchronises).
int prof_flush(lbm_s *h) {
    if (!h->ev || h->ev_used == 0) return LBM_OK;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ERR_CUDA;
    for (int s = 0; s < h->ev_used; ++s)
        for (int ph = 0; ph < 4; ++ph) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, h->ev[5 * s + ph], h->ev[5 * s + ph + 1]) != cudaSuccess) return LBM_ERR_CUDA;
            h->prof_ms[ph] += ms;
        }
    h->prof_steps += h->ev_used;
    h->ev_used = 0;
    return LBM_OK;
}

inline int prof_mark(lbm_s *h, int k) {
    if (!h->prof) return LBM_OK;
    return cudaEventRecord(h->ev[5 * h->ev_used + k], h->stream) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

// Sync the stream and fold the device status into the sticky error.
int settle(lbm_s *h) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        if (!h->sticky) h->sticky = LBM_ERR_CUDA;
        return h->sticky;
    }
    if (cudaMemcpy(h->status_host, h->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
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
        case LBM_ERR_GEOMETRY: return "a sphere moved half a lattice unit in one step or left the box";
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
    if (!(p.rho_particle > 0.0) || !(p.kn >= 0.0) || !(p.restitution > 0.0 && p.restitution <= 1.0)) return LBM_ERR_ARG;
    if (p.dem_substeps < 1) return LBM_ERR_ARG;
    if (p.precision != LBM_FP32 && p.precision != LBM_BF16_DEV && p.precision != LBM_FP16_DEV) return LBM_ERR_ARG;
    if (p.max_particles < 0) return LBM_ERR_ARG;
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
    if (p.cuda_stream) {
        h->stream = (cudaStream_t)p.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
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
    if (!rc) rc = dalloc(h, &pt.rebuild, 1);
    if (!rc) rc = dalloc(h, &pt.frame[0], (size_t)M);
    if (!rc) rc = dalloc(h, &pt.frame[1], (size_t)M);
    if (!rc) rc = dalloc(h, &pt.pairA, (size_t)M * kMaxNbr);
    if (!rc) rc = dalloc(h, &pt.pairB, (size_t)M * kMaxNbr);
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
    if (!rc) {
        int per_sm = 0, sms = 0;
        if (dem_max_blocks(kDemThreads, &per_sm) != LBM_OK ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device) != cudaSuccess)
            rc = LBM_ERR_CUDA;
        h->dem_threads = kDemThreads;
        h->dem_blocks = per_sm * sms;
        if (!rc && h->dem_blocks < 1) rc = LBM_ERR_CUDA;
        h->dem_cluster = M > 0 ? dem_cluster_setup(M) : 0;
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
    if (!h) return LBM_ERR_ARG;
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
    if (!rc && n && cudaMemsetAsync(pt.rebuild, 0, sizeof(int), h->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    if (!rc) rc = copy_in(h, pt.V, vel, v3, LBM_HOST);
    if (!rc) rc = copy_in(h, pt.W, omega, v3, LBM_HOST);
    if (!rc) rc = copy_in(h, pt.R, radius, sizeof(double) * (size_t)n, LBM_HOST);
    if (!rc && n) {
        if (fixed)
            rc = copy_in(h, (void *)pt.fixed, fixed, (size_t)n, LBM_HOST);
        else if (cudaMemsetAsync((void *)pt.fixed, 0, (size_t)n, h->stream) != cudaSuccess)
            rc = LBM_ERR_CUDA;
    }
    double *zero[] = {pt.Fh, pt.Th, pt.Fc, pt.Fx, pt.Tx};
    for (double *z : zero)
        if (!rc && n && cudaMemsetAsync(z, 0, v3, h->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    if (!rc && cudaMemsetAsync(h->f, 0, (size_t)Q * h->L.S * h->esize, h->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    if (!rc && cudaMemsetAsync(h->flag, 0, (size_t)h->L.N, h->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    if (!rc && cudaMemsetAsync(h->owner, 0xff, (size_t)h->L.N * 4, h->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    if (!rc && cudaMemsetAsync(h->ctr, 0, 4 * sizeof(unsigned long long), h->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    pt.np = n;
    h->parity = 0;
    h->steps = 0;
    if (!rc && n) rc = launch_neighbours(h, 1);
    if (!rc && n) rc = launch_mark(h);
    if (!rc && n) rc = launch_contact(h);
    if (!rc) rc = settle(h);
    std::free(xf);
    std::free(fr);
    if (rc == LBM_ERR_CUDA && !h->sticky) h->sticky = rc;
    return rc;
}

int lbm_set_particle_load(lbm_handle h, const double *force, const double *torque, int32_t where) {
    if (!h || (where != LBM_HOST && where != LBM_DEVICE)) return LBM_ERR_ARG;
    if (h->sticky) return h->sticky;
    DeviceScope ds(h->device);
    const size_t v3 = 3 * sizeof(double) * (size_t)h->pt.np;
    int rc = LBM_OK;
    if (force)
        rc = copy_in(h, h->pt.Fx, force, v3, where);
    else if (v3 && cudaMemsetAsync(h->pt.Fx, 0, v3, h->stream) != cudaSuccess)
        rc = LBM_ERR_CUDA;
    if (!rc) {
        if (torque)
            rc = copy_in(h, h->pt.Tx, torque, v3, where);
        else if (v3 && cudaMemsetAsync(h->pt.Tx, 0, v3, h->stream) != cudaSuccess)
            rc = LBM_ERR_CUDA;
    }
    // the caller may reuse its buffer as soon as we return
    if (!rc && where == LBM_HOST && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
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

int lbm_step(lbm_handle h, int32_t nsteps) {
    if (!h || nsteps < 0) return LBM_ERR_ARG;
    if (h->sticky) return h->sticky;
    const int polled = status_to_code(*h->status_host);  // mirror of an earlier call
    if (polled) {
        h->sticky = polled;
        return polled;
    }
    DeviceScope ds(h->device);
    int rc = LBM_OK;
    const bool parts = h->pt.np > 0;
    for (int it = 0; it < nsteps && !rc; ++it) {
        const int P = h->parity;
        if (h->prof && h->ev_used == h->ev_cap) rc = prof_flush(h);
        if (!rc && it == nsteps - 1 &&
            cudaMemsetAsync(h->ctr, 0, 2 * sizeof(unsigned long long), h->stream) != cudaSuccess)
            rc = LBM_ERR_CUDA;
        if (!rc) rc = prof_mark(h, 0);
        if (!rc && parts) rc = launch_mark(h);
        if (!rc && parts) rc = launch_refill(h, P);
        if (!rc) rc = prof_mark(h, 1);
        if (!rc) rc = launch_stream_collide(h, P);
        if (!rc) rc = prof_mark(h, 2);
        if (!rc && parts) rc = launch_links(h, P);
        if (!rc) rc = prof_mark(h, 3);
        if (!rc && parts) rc = launch_neighbours(h, 0);
        if (!rc && parts) rc = launch_dem(h);
        if (!rc) rc = prof_mark(h, 4);
        if (!rc) {
            if (h->prof) ++h->ev_used;
            h->parity ^= 1;
            ++h->steps;
        }
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

int lbm_profile(lbm_handle h, int32_t enable) {
    if (!h) return LBM_ERR_ARG;
    DeviceScope ds(h->device);
    if (enable && !h->ev) {
        h->ev = (cudaEvent_t *)std::calloc(5 * (size_t)kProfSteps, sizeof(cudaEvent_t));
        if (!h->ev) return LBM_ERR_NOMEM;
        for (int i = 0; i < 5 * kProfSteps; ++i)
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
        for (int i = 0; i < 4; ++i) ms[i] = h->prof_ms[i];
    if (steps) *steps = h->prof_steps;
    return rc;
}

int lbm_sync(lbm_handle h) {
    if (!h) return LBM_ERR_ARG;
    DeviceScope ds(h->device);
    return settle(h);
}

}  // extern "C"
