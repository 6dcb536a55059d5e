// lbm_fields_noalloc: the density / velocity read-out of lbm_fields to host
// memory, staged through a fixed device array instead of a temporary
// allocation, for callers that must not allocate device memory.
//
// The staging array below is part of the library image.  Its address is
// looked up once per device, with that device current, on the first call
// there; under lazy module loading that lookup is when the driver commits
// the array's 16 MiB on the device, which then holds it until the process
// exits (an allocation failure there is reported as LBM_ERR_NOMEM).  All calls on a device share the array and it keeps the last call's
// contents; the fields kernel writes every element it later copies, so
// nothing needs clearing.  Two calls whose work overlaps on the same GPU
// (handles on different streams) race on the array.
#include <mutex>

#include "lbm_internal.cuh"

namespace {

constexpr long long kNoallocMaxNodes = 1ll << 20;  // = LBM_NOALLOC_MAX_NODES
constexpr int kMaxDevices = 64;

// rho[N] then u[3][N] for the largest lattice this entry point accepts.
static __device__ __align__(256) float g_fields_staging[4 * kNoallocMaxNodes];

std::mutex g_mutex;
float *g_staging[kMaxDevices] = {};

// Device address of the staging array on `device` (which is current).
int staging_for(int device, float **out) {
    if (device < 0 || device >= kMaxDevices) return LBM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_staging[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_fields_staging);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? LBM_ERR_NOMEM : LBM_ERR_CUDA;
        }
        g_staging[device] = (float *)p;
    }
    *out = g_staging[device];
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_fields_noalloc(lbm_handle h, float *rho, float *u) {
    if (!h || (!rho && !u)) return LBM_ERR_ARG;
    const long long N = h->L.N;
    if (N > kNoallocMaxNodes) return LBM_ERR_CAPACITY;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != h->device && cudaSetDevice(h->device) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    float *stage = nullptr;
    int rc = staging_for(h->device, &stage);
    if (!rc) rc = lbm::launch_fields(h, stage, stage + N, h->parity);
    if (!rc && rho &&
        cudaMemcpyAsync(rho, stage, sizeof(float) * (size_t)N, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        rc = LBM_ERR_CUDA;
    if (!rc && u &&
        cudaMemcpyAsync(u, stage + N, 3 * sizeof(float) * (size_t)N, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        rc = LBM_ERR_CUDA;
    const int s = lbm::settle_handle(h);  // waits for the stream, folds in the device status
    if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
    return rc ? rc : s;
}
