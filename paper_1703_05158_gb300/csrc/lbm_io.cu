// Gather / scatter between the A-A storage and the natural layout of the ABI
// ([19][N] FP64 populations, FP32 density and velocity, owner ids).  The
// pre-collision population f_k(x) of the current time sits at
// in_slot(parity, k, x); values are w_k + stored deviation.
#include "lbm_internal.cuh"

namespace lbm {

template <typename T>
__global__ void k_get_populations(const Lat L, const T *__restrict__ f, const uint8_t *__restrict__ flag, int P,
                                  double *__restrict__ out) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= L.N) return;
    const int x = (int)(n % L.nx), y = (int)((n / L.nx) % L.ny);
    const bool solid = flag[n] & 1;
    const Nbr nb(L, x, y);
    for (int k = 0; k < Q; ++k)
        out[(long long)k * L.N + n] =
            solid ? 0.0 : (double)rw36(k) / 36.0 + (double)Store<T>::ld(f + in_slot(L, nb, P, k, n + L.plane));
}

template <typename T>
__global__ void k_set_populations(const Lat L, T *__restrict__ f, const uint8_t *__restrict__ flag, int P,
                                  const double *__restrict__ in) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= L.N) return;
    if (flag[n] & 1) return;
    const int x = (int)(n % L.nx), y = (int)((n / L.nx) % L.ny);
    const Nbr nb(L, x, y);
    for (int k = 0; k < Q; ++k)
        Store<T>::st(f + in_slot(L, nb, P, k, n + L.plane), (float)(in[(long long)k * L.N + n] - (double)rw36(k) / 36.0));
}

template <typename T>
__global__ void k_fields(const Lat L, const Phys ph, const T *__restrict__ f, const uint8_t *__restrict__ flag, int P,
                         float *__restrict__ rho, float *__restrict__ u) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= L.N) return;
    float r = 0.f, ux = 0.f, uy = 0.f, uz = 0.f;
    if (!(flag[n] & 1)) {
        const int x = (int)(n % L.nx), y = (int)((n / L.nx) % L.ny);
        const Nbr nb(L, x, y);
        float dr = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
        for (int k = 0; k < Q; ++k) {
            const float d = Store<T>::ld(f + in_slot(L, nb, P, k, n + L.plane));
            dr += d;
            jx += rcx(k) * d;
            jy += rcy(k) * d;
            jz += rcz(k) * d;
        }
        r = 1.f + dr;
        ux = jx / r + 0.5f * ph.g[0];
        uy = jy / r + 0.5f * ph.g[1];
        uz = jz / r + 0.5f * ph.g[2];
    }
    if (rho) rho[n] = r;
    if (u) {
        u[n] = ux;
        u[L.N + n] = uy;
        u[2 * L.N + n] = uz;
    }
}

__global__ void k_owner(const Lat L, const uint8_t *__restrict__ flag, const int32_t *__restrict__ owner,
                        int32_t *__restrict__ out) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= L.N) return;
    out[n] = (flag[n] & 1) ? owner[n] : -1;
}

__global__ void k_count_fluid(const Lat L, const uint8_t *__restrict__ flag, unsigned long long *__restrict__ ctr) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const unsigned fluid = (n < L.N && !(flag[n] & 1)) ? 1u : 0u;
    const unsigned c = __popc(__ballot_sync(0xffffffffu, fluid));
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(ctr + 2, (unsigned long long)c);
}

static inline unsigned blocks_of(long long N) { return (unsigned)((N + 255) / 256); }

int launch_get_populations(lbm_s *h, double *out, int P) {
    const unsigned g = blocks_of(h->L.N);
    switch (h->precision) {
        case LBM_FP32: k_get_populations<float><<<g, 256, 0, h->stream>>>(h->L, (const float *)h->f, h->flag, P, out); break;
        case LBM_BF16_DEV:
            k_get_populations<__nv_bfloat16><<<g, 256, 0, h->stream>>>(h->L, (const __nv_bfloat16 *)h->f, h->flag, P, out);
            break;
        case LBM_FP16_DEV: k_get_populations<__half><<<g, 256, 0, h->stream>>>(h->L, (const __half *)h->f, h->flag, P, out); break;
        default: return LBM_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int launch_set_populations(lbm_s *h, const double *in, int P) {
    const unsigned g = blocks_of(h->L.N);
    switch (h->precision) {
        case LBM_FP32: k_set_populations<float><<<g, 256, 0, h->stream>>>(h->L, (float *)h->f, h->flag, P, in); break;
        case LBM_BF16_DEV:
            k_set_populations<__nv_bfloat16><<<g, 256, 0, h->stream>>>(h->L, (__nv_bfloat16 *)h->f, h->flag, P, in);
            break;
        case LBM_FP16_DEV: k_set_populations<__half><<<g, 256, 0, h->stream>>>(h->L, (__half *)h->f, h->flag, P, in); break;
        default: return LBM_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int launch_fields(lbm_s *h, float *rho, float *u, int P) {
    const unsigned g = blocks_of(h->L.N);
    switch (h->precision) {
        case LBM_FP32: k_fields<float><<<g, 256, 0, h->stream>>>(h->L, h->ph, (const float *)h->f, h->flag, P, rho, u); break;
        case LBM_BF16_DEV:
            k_fields<__nv_bfloat16><<<g, 256, 0, h->stream>>>(h->L, h->ph, (const __nv_bfloat16 *)h->f, h->flag, P, rho, u);
            break;
        case LBM_FP16_DEV: k_fields<__half><<<g, 256, 0, h->stream>>>(h->L, h->ph, (const __half *)h->f, h->flag, P, rho, u); break;
        default: return LBM_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int launch_owner(lbm_s *h, int32_t *out) {
    k_owner<<<blocks_of(h->L.N), 256, 0, h->stream>>>(h->L, h->flag, h->owner, out);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int launch_count_fluid(lbm_s *h) {
    k_count_fluid<<<blocks_of(h->L.N), 256, 0, h->stream>>>(h->L, h->flag, h->ctr);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

}  // namespace lbm
