// Fused collide-and-stream kernel (Sect. 2.2) on the one-array A-A layout.
//
// Per fluid node: read the 19 pre-collision deviations d_i = f_i - w_i, form
// rho (Eq. 5) and the force-shifted velocity (Eq. 6, u = sum f c / rho + g/2),
// the non-equilibrium momentum flux Pi_ab = sum c_a c_b (f - f^eq) against the
// equilibrium of Eq. (9), the Smagorinsky relaxation time of Eq. (18)
//   tau* = tau0 + 1/2 [sqrt(tau0^2 + 18 sqrt(2) C^2 Q / rho) - tau0],
//   Q = sqrt(Pi_ab Pi_ab),
// relax (Eq. 12) and add the body-force source of Guo, Zheng & Shi (2002),
//   (1 - 1/(2 tau*)) w_i [3 (c_i - u).F + 9 (c_i.u)(c_i.F)],  F = rho g,
// then write the 19 post-collision deviations in place (A-A, so streaming is
// implicit in the addressing of the next step).  Nodes next to the z walls
// also write the halfway bounce-back value of Eqs. (19, 21) with q = 1/2,
//   f_k(x, t+1) = f^c_opp(k)(x) + 6 w_k (c_k . u_wall),
// straight into the slot the next step reads for the population arriving
// from the wall, so no separate wall pass is needed.  Sphere links are
// completed afterwards by the link kernel.
//
// Roofline: HBM-bound.  Algorithmic traffic per fluid node and step is
// 19 loads + 19 stores of the stored type plus one flag byte.
#include "lbm_internal.cuh"

namespace lbm {

// Neighbour offsets in 32-bit element units (x, y periodic; z never wraps).
struct Off32 {
    int xm, xp, ym, yp, zp;
    __device__ __forceinline__ Off32(const Lat &L, int x, int y) {
        xm = x == 0 ? L.nx - 1 : -1;
        xp = x == L.nx - 1 ? 1 - L.nx : 1;
        ym = y == 0 ? L.nx * (L.ny - 1) : -L.nx;
        yp = y == L.ny - 1 ? -L.nx * (L.ny - 1) : L.nx;
        zp = (int)L.plane;
    }
    __device__ __forceinline__ int operator()(int ox, int oy, int oz) const {
        return (ox < 0 ? xm : (ox > 0 ? xp : 0)) + (oy < 0 ? ym : (oy > 0 ? yp : 0)) + oz * zp;
    }
};

template <int ODD, typename T>
__global__ void __launch_bounds__(256, 4) k_stream_collide(const Lat L, const Phys ph, T *__restrict__ f,
                                                        uint8_t *__restrict__ flag, int *__restrict__ status) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= L.nx) return;
    const int n = x + L.nx * (y + L.ny * z);
    const uint8_t fl = flag[n];
    if (fl & 1) return;      // solid: its slots are mailboxes of the link kernel
    if (fl) flag[n] = 0;     // refilled this step: plain fluid from now on
    const int s = n + (int)L.plane;
    const int S = (int)L.S;
    const Off32 nb(L, x, y);

    float d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int a = ODD ? opp(i) * S + s + nb(-cx(i), -cy(i), -cz(i)) : i * S + s;
        d[i] = Store<T>::ld(f + a);
    }

    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += d[i];
        if (cx(i)) jx += cx(i) > 0 ? d[i] : -d[i];
        if (cy(i)) jy += cy(i) > 0 ? d[i] : -d[i];
        if (cz(i)) jz += cz(i) > 0 ? d[i] : -d[i];
    }
    const float rho = 1.f + drho;
    if (!(rho > 0.f)) atomicOr(status, ST_DIVERGED);
    const float ir = 1.f / rho;
    const float ux = jx * ir + 0.5f * ph.g[0];
    const float uy = jy * ir + 0.5f * ph.g[1];
    const float uz = jz * ir + 0.5f * ph.g[2];
    const float uu = ux * ux + uy * uy + uz * uz;

    float tau = ph.tau0;
    if (ph.smag > 0.f) {
        // Pi^neq_ab = sum c_a c_b (f - f^eq) = m_ab - drho delta_ab / 3 - rho u_a u_b, with
        // m_ab = sum c_a c_b d_i and the D3Q19 identity sum c_a c_b f^eq = rho (delta_ab/3 + u_a u_b)
        float mxx = 0.f, myy = 0.f, mzz = 0.f, mxy = 0.f, mxz = 0.f, myz = 0.f;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if (cx(i)) mxx += d[i];
            if (cy(i)) myy += d[i];
            if (cz(i)) mzz += d[i];
            if (cx(i) * cy(i)) mxy += cx(i) * cy(i) > 0 ? d[i] : -d[i];
            if (cx(i) * cz(i)) mxz += cx(i) * cz(i) > 0 ? d[i] : -d[i];
            if (cy(i) * cz(i)) myz += cy(i) * cz(i) > 0 ? d[i] : -d[i];
        }
        const float t3 = drho * (1.f / 3.f);
        const float pxx = mxx - t3 - rho * ux * ux, pyy = myy - t3 - rho * uy * uy, pzz = mzz - t3 - rho * uz * uz;
        const float pxy = mxy - rho * ux * uy, pxz = mxz - rho * ux * uz, pyz = myz - rho * uy * uz;
        const float q2 = pxx * pxx + pyy * pyy + pzz * pzz + 2.f * (pxy * pxy + pxz * pxz + pyz * pyz);
        tau = ph.tau0 + 0.5f * (sqrtf(ph.tau0 * ph.tau0 + ph.smag * sqrtf(q2) * ir) - ph.tau0);
    }
    const float om = 1.f / tau;

    // Relaxation towards Eq. (9) (deviation form), by opposite pairs (i, i+9):
    // f^eq - w = w [drho + rho (4.5 (c.u)^2 - 1.5 u^2)]  +/-  3 w rho (c.u)
    const float base = drho - 1.5f * rho * uu;
    d[0] += om * (wf(0) * base - d[0]);
    const bool forced = ph.g[0] != 0.f || ph.g[1] != 0.f || ph.g[2] != 0.f;
    const float fx = rho * ph.g[0], fy = rho * ph.g[1], fz = rho * ph.g[2];
    const float uF = ux * fx + uy * fy + uz * fz;
    const float sk = 1.f - 0.5f * om;
    if (forced) d[0] += sk * wf(0) * (-3.f * uF);
#pragma unroll
    for (int i = 1; i <= 9; ++i) {
        const int k = i + 9;  // opp(i)
        const float cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
        const float sym = wf(i) * (base + 4.5f * rho * cu * cu);
        const float asym = 3.f * wf(i) * rho * cu;
        d[i] += om * (sym + asym - d[i]);
        d[k] += om * (sym - asym - d[k]);
        if (forced) {
            // Guo source: w [3 (c - u).F + 9 (c.u)(c.F)], even and odd parts
            const float cF = cx(i) * fx + cy(i) * fy + cz(i) * fz;
            const float se = sk * wf(i) * (9.f * cu * cF - 3.f * uF);
            const float so = sk * wf(i) * 3.f * cF;
            d[i] += se + so;
            d[k] += se - so;
        }
    }

#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int a = ODD ? i * S + s + nb(cx(i), cy(i), cz(i)) : opp(i) * S + s;
        Store<T>::st(f + a, d[i]);
    }

    // Walls: push the halfway bounce-back population into the slot the next
    // step (parity !ODD) reads for the direction coming from the wall.
    if (z == 0) {
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            if (cz(k) != 1) continue;
            const float v = d[opp(k)] + 6.f * wf(k) * (cx(k) * ph.ulo[0] + cy(k) * ph.ulo[1] + cz(k) * ph.ulo[2]);
            const int a = ODD ? k * S + s : opp(k) * S + s + nb(-cx(k), -cy(k), -cz(k));
            Store<T>::st(f + a, v);
        }
    }
    if (z == L.nz - 1) {
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            if (cz(k) != -1) continue;
            const float v = d[opp(k)] + 6.f * wf(k) * (cx(k) * ph.uhi[0] + cy(k) * ph.uhi[1] + cz(k) * ph.uhi[2]);
            const int a = ODD ? k * S + s : opp(k) * S + s + nb(-cx(k), -cy(k), -cz(k));
            Store<T>::st(f + a, v);
        }
    }
}

template <int ODD, typename T>
static int launch_sc(lbm_s *h) {
    const int bx = h->L.nx >= 256 ? 256 : ((h->L.nx + 31) / 32) * 32;
    dim3 grid((h->L.nx + bx - 1) / bx, h->L.ny, h->L.nz);
    k_stream_collide<ODD, T><<<grid, bx, 0, h->stream>>>(h->L, h->ph, (T *)h->f, h->flag, h->status);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int launch_stream_collide(lbm_s *h, int parity) {
    switch (h->precision) {
        case LBM_FP32: return parity ? launch_sc<1, float>(h) : launch_sc<0, float>(h);
        case LBM_BF16_DEV: return parity ? launch_sc<1, __nv_bfloat16>(h) : launch_sc<0, __nv_bfloat16>(h);
        case LBM_FP16_DEV: return parity ? launch_sc<1, __half>(h) : launch_sc<0, __half>(h);
    }
    return LBM_ERR_ARG;
}

}  // namespace lbm
