// Zoom-in with Effective Boundaries (Sect. 2.6): the plane z = 0 is the
// first simulated plane x_S next to a virtual piston cylinder (volume V_0,
// cross-section A_p, piston displacement H_p) that replaces the fluid below.
// Run after the link kernel of a step of parity P, on the populations the
// next step reads:
//   rho^{n+1} = rho^n exp[(v_p A_p - v_f^n A_p) / (V_0 - A_p H_p^n)]   (Eq. 8)
// with v_f^n the mean u_z over the face's fluid nodes left by the previous
// update (0 at the start); at each fluid node of the face, rho* sums the 14
// populations streamed in from the lattice and the five that would come from
// the cylinder (c_z = +1) at the values the node's own collision gave them
// (nothing streamed into them); the one normal to the face takes
// f_12 = rho^{n+1} - (rho* - f_12) (Eq. 9), u = sum f c / rho^{n+1}, and all
// 19 populations become f^eq(rho^{n+1}, u).  The halfway bounce-back the
// collide kernel pushed for the wall z = -1/2 is overwritten.
//
// A step at which V_0 - A_p H_p is no longer positive (the piston has
// swept the cylinder) or rho^{n+1} is not finite sets the sticky divergence
// status and keeps rho^n.
//
// One thread per face node.  Every block recomputes rho^{n+1} from the
// state of the previous update (the per-block sums of u_z, reduced in block
// order, so the result does not depend on timing); block 0 stores it.  The
// cylinder state and the sums are double-buffered by step parity.
#include "lbm_internal.cuh"

namespace lbm {

constexpr int kZiebThreads = 256;
static_assert(cx(12) == 0 && cy(12) == 0 && cz(12) == 1, "population 12 is the one normal to the face");

template <typename T>
__global__ void __launch_bounds__(kZiebThreads) k_zieb(const Lat L, T *__restrict__ f,
                                                      const uint8_t *__restrict__ flag, const int P,
                                                      double *__restrict__ zs, double *__restrict__ zpart,
                                                      int *__restrict__ zcnt, const int nblk, const double A,
                                                      const double V0, int *__restrict__ status) {
    __shared__ double s_rho1;
    __shared__ double red[kZiebThreads / 32];
    __shared__ int redc[kZiebThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const double *part = zpart + (size_t)P * nblk;
    const int *pc = zcnt + (size_t)P * nblk;
    if (wid == 0) {
        double su = 0.0;
        int sc = 0;
        for (int b = lane; b < nblk; b += 32) {
            su += part[b];
            sc += pc[b];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            su += __shfl_xor_sync(0xffffffffu, su, o);
            sc += __shfl_xor_sync(0xffffffffu, sc, o);
        }
        if (lane == 0) {
            const double vf = sc ? su / sc : 0.0;
            const double rho0 = zs[P], H = zs[2 + P], vp = zs[4];
            double rho1 = rho0 * exp((vp * A - vf * A) / (V0 - A * H));
            if (!(V0 - A * H > 0.0) || !isfinite(rho1)) {  // the piston has emptied the cylinder
                if (blockIdx.x == 0) atomicOr(status, ST_DIVERGED);
                rho1 = rho0;
            }
            s_rho1 = rho1;
            if (blockIdx.x == 0) {
                zs[P ^ 1] = rho1;
                zs[2 + (P ^ 1)] = H + vp;
            }
        }
    }
    __syncthreads();
    const double rho1d = s_rho1;
    const float rho1 = (float)rho1d, drho = (float)(rho1d - 1.0);
    const int i = blockIdx.x * kZiebThreads + threadIdx.x;
    float uz = 0.f;
    int cnt = 0;
    if (i < L.nx * L.ny && !(flag[i] & 1)) {
        const int x = i % L.nx, y = i / L.nx;
        const Nbr nb(L, x, y);
        const long long s = (long long)i + L.plane;
        float d[Q], sum = 0.f;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const long long a = rcz(k) == 1 ? post_slot(L, nb, P, k, s) : in_slot(L, nb, P ^ 1, k, s);
            d[k] = Store<T>::ld(f + a);
            sum += d[k];
        }
        // deviations: f_12 - w_12 = (rho^{n+1} - 1) - (sum d - d_12), as sum w = 1
        d[12] = drho - (sum - d[12]);
        float mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            mx += rcx(k) * d[k];
            my += rcy(k) * d[k];
            mz += rcz(k) * d[k];
        }
        const float ir = 1.f / rho1;
        const float ux = mx * ir, uy = my * ir;
        uz = mz * ir;
        const float uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const float cu = rcx(k) * ux + rcy(k) * uy + rcz(k) * uz;
            const float dq = (float)rw36(k) / 36.f * (drho + rho1 * (3.f * cu + 4.5f * cu * cu - 1.5f * uu));
            Store<T>::st(f + in_slot(L, nb, P ^ 1, k, s), dq);
        }
        cnt = 1;
    }
    // block sums of u_z and of the fluid face nodes, in a fixed order
    double su = (double)uz;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        su += __shfl_xor_sync(0xffffffffu, su, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) {
        red[wid] = su;
        redc[wid] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        int c = 0;
        for (int w = 0; w < kZiebThreads / 32; ++w) {
            t += red[w];
            c += redc[w];
        }
        zpart[(size_t)(P ^ 1) * nblk + blockIdx.x] = t;
        zcnt[(size_t)(P ^ 1) * nblk + blockIdx.x] = c;
    }
}

int launch_zieb(lbm_s *h, int P) {
    const dim3 g(h->zblocks);
    switch (h->precision) {
        case LBM_FP32:
            k_zieb<float><<<g, kZiebThreads, 0, h->stream>>>(h->L, (float *)h->f, h->flag, P, h->zs, h->zpart,
                                                             h->zcnt, h->zblocks, h->zA, h->zV0, h->status);
            break;
        case LBM_BF16_DEV:
            k_zieb<__nv_bfloat16><<<g, kZiebThreads, 0, h->stream>>>(h->L, (__nv_bfloat16 *)h->f, h->flag, P,
                                                                     h->zs, h->zpart, h->zcnt, h->zblocks, h->zA,
                                                                     h->zV0, h->status);
            break;
        case LBM_FP16_DEV:
            k_zieb<__half><<<g, kZiebThreads, 0, h->stream>>>(h->L, (__half *)h->f, h->flag, P, h->zs, h->zpart,
                                                              h->zcnt, h->zblocks, h->zA, h->zV0, h->status);
            break;
        default: return LBM_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

}  // namespace lbm
