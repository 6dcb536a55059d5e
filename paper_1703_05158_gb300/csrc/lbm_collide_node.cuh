// The collision of one node (Sect. 2.2), shared by every kernel that
// collides: the fused stream-collide kernels of lbm_collide.cu and the
// channel kernels of the differentiation form (lbm_channel.cu).
#pragma once

#include "lbm_internal.cuh"

namespace lbm {

// Collision of one node (deviations in d, in place): rho (Eq. 5), the
// force-shifted velocity (Eq. 6), Pi^neq and the Smagorinsky relaxation
// time (Eq. 18), BGK relaxation towards Eq. (9) by opposite pairs, and the
// Guo source.  Every collide kernel calls this one function.  Each multiply
// and add is an explicit round-to-nearest intrinsic (fused where written
// __fmaf_rn), so the compiler cannot contract differently in different
// kernels and a node gets bitwise the same result from any of them; the
// products with lattice-vector components (0 or +-1) round the same either
// way and are left to the compiler.
__device__ __forceinline__ void collide_node(const Phys &ph, float (&d)[Q], int *status) {
    // moments from the sums and differences of opposite pairs (i, i + 9):
    // rho and the second moments take sp_i = d_i + d_i+9, the momentum
    // takes dm_i = d_i - d_i+9 (c_i+9 = -c_i)
    float sp[10], dm[10];
#pragma unroll
    for (int i = 1; i <= 9; ++i) {
        static_assert(opp(1) == 10 && opp(9) == 18, "opposite pairs are (i, i + 9)");
        sp[i] = __fadd_rn(d[i], d[i + 9]);
        dm[i] = __fsub_rn(d[i], d[i + 9]);
    }
    float drho = d[0], jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 1; i <= 9; ++i) {
        drho = __fadd_rn(drho, sp[i]);
        if (cx(i)) jx = cx(i) > 0 ? __fadd_rn(jx, dm[i]) : __fsub_rn(jx, dm[i]);
        if (cy(i)) jy = cy(i) > 0 ? __fadd_rn(jy, dm[i]) : __fsub_rn(jy, dm[i]);
        if (cz(i)) jz = cz(i) > 0 ? __fadd_rn(jz, dm[i]) : __fsub_rn(jz, dm[i]);
    }
    const float rho = __fadd_rn(1.f, drho);
    if (!(rho > 0.f)) atomicOr(status, ST_DIVERGED);
    const float ir = __fdiv_rn(1.f, rho);
    const float ux = __fmaf_rn(jx, ir, 0.5f * ph.g[0]);  // g/2 is exact
    const float uy = __fmaf_rn(jy, ir, 0.5f * ph.g[1]);
    const float uz = __fmaf_rn(jz, ir, 0.5f * ph.g[2]);
    const float uu = __fmaf_rn(uz, uz, __fmaf_rn(uy, uy, __fmul_rn(ux, ux)));
    float tau = ph.tau0;
    if (ph.smag > 0.f) {
        // Pi^neq_ab = sum c_a c_b (f - f^eq) = m_ab - drho delta_ab / 3 - rho u_a u_b, with
        // m_ab = sum c_a c_b d_i and the D3Q19 identity sum c_a c_b f^eq = rho (delta_ab/3 + u_a u_b)
        float mxx = 0.f, myy = 0.f, mzz = 0.f, mxy = 0.f, mxz = 0.f, myz = 0.f;
#pragma unroll
        for (int i = 1; i <= 9; ++i) {
            if (cx(i)) mxx = __fadd_rn(mxx, sp[i]);
            if (cy(i)) myy = __fadd_rn(myy, sp[i]);
            if (cz(i)) mzz = __fadd_rn(mzz, sp[i]);
            if (cx(i) * cy(i)) mxy = cx(i) * cy(i) > 0 ? __fadd_rn(mxy, sp[i]) : __fsub_rn(mxy, sp[i]);
            if (cx(i) * cz(i)) mxz = cx(i) * cz(i) > 0 ? __fadd_rn(mxz, sp[i]) : __fsub_rn(mxz, sp[i]);
            if (cy(i) * cz(i)) myz = cy(i) * cz(i) > 0 ? __fadd_rn(myz, sp[i]) : __fsub_rn(myz, sp[i]);
        }
        const float t3 = __fmul_rn(drho, 1.f / 3.f);
        const float rux = __fmul_rn(rho, ux), ruy = __fmul_rn(rho, uy), ruz = __fmul_rn(rho, uz);
        const float pxx = __fmaf_rn(-rux, ux, __fsub_rn(mxx, t3));
        const float pyy = __fmaf_rn(-ruy, uy, __fsub_rn(myy, t3));
        const float pzz = __fmaf_rn(-ruz, uz, __fsub_rn(mzz, t3));
        const float pxy = __fmaf_rn(-rux, uy, mxy), pxz = __fmaf_rn(-rux, uz, mxz), pyz = __fmaf_rn(-ruy, uz, myz);
        const float off = __fmaf_rn(pyz, pyz, __fmaf_rn(pxz, pxz, __fmul_rn(pxy, pxy)));
        const float q2 = __fmaf_rn(2.f, off, __fmaf_rn(pzz, pzz, __fmaf_rn(pyy, pyy, __fmul_rn(pxx, pxx))));
        const float inner = __fmaf_rn(__fmul_rn(ph.smag, __fsqrt_rn(q2)), ir, __fmul_rn(ph.tau0, ph.tau0));
        tau = __fmaf_rn(0.5f, __fsub_rn(__fsqrt_rn(inner), ph.tau0), ph.tau0);
    }
    const float om = __fdiv_rn(1.f, tau);

    // Relaxation towards Eq. (9) (deviation form), by opposite pairs (i, i+9):
    // f^eq - w = w [drho + rho (4.5 (c.u)^2 - 1.5 u^2)]  +/-  3 w rho (c.u),
    // written d' = (1 - om) d + om (f^eq - w) with om folded into the two
    // weight classes' factors (w = 1/18 for the axes, 1/36 for the diagonals)
    const float base = __fmaf_rn(-__fmul_rn(1.5f, rho), uu, drho);
    const float keep = __fsub_rn(1.f, om);
    d[0] = __fmaf_rn(keep, d[0], __fmul_rn(__fmul_rn(om, wf(0)), base));
    const bool forced = ph.g[0] != 0.f || ph.g[1] != 0.f || ph.g[2] != 0.f;
    const float fx = __fmul_rn(rho, ph.g[0]), fy = __fmul_rn(rho, ph.g[1]), fz = __fmul_rn(rho, ph.g[2]);
    const float uF = __fmaf_rn(uz, fz, __fmaf_rn(uy, fy, __fmul_rn(ux, fx)));
    const float sk = __fmaf_rn(-0.5f, om, 1.f);
    if (forced) d[0] = __fmaf_rn(__fmul_rn(sk, wf(0)), __fmul_rn(-3.f, uF), d[0]);
    // per weight class c (0: 1/18, 1: 1/36): om w, om w 4.5 rho, om w base, om 3 w rho
    float ow45[2], owb[2], ow3[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const float ow = __fmul_rn(om, c == 0 ? wf(1) : wf(4));
        ow45[c] = __fmul_rn(ow, __fmul_rn(4.5f, rho));
        owb[c] = __fmul_rn(ow, base);
        ow3[c] = __fmul_rn(__fmul_rn(3.f, ow), rho);
    }
#pragma unroll
    for (int i = 1; i <= 9; ++i) {
        const int k = i + 9;  // opp(i)
        const int c = w36(i) == 2 ? 0 : 1;
        const float cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
        const float sym = __fmaf_rn(__fmul_rn(ow45[c], cu), cu, owb[c]);  // om (f^eq - w), even part
        const float asym = __fmul_rn(ow3[c], cu);                           // odd part
        d[i] = __fmaf_rn(keep, d[i], __fadd_rn(sym, asym));
        d[k] = __fmaf_rn(keep, d[k], __fsub_rn(sym, asym));
        if (forced) {
            // Guo source: w [3 (c - u).F + 9 (c.u)(c.F)], even and odd parts
            const float cF = cx(i) * fx + cy(i) * fy + cz(i) * fz;
            const float skw = __fmul_rn(sk, wf(i));
            const float se = __fmul_rn(skw, __fmaf_rn(__fmul_rn(9.f, cu), cF, __fmul_rn(-3.f, uF)));
            const float so = __fmul_rn(__fmul_rn(3.f, skw), cF);
            d[i] = __fadd_rn(d[i], __fadd_rn(se, so));
            d[k] = __fadd_rn(d[k], __fsub_rn(se, so));
        }
    }
}

// Halfway bounce-back value of Eqs. (19, 21) with q = 1/2 for the
// population k arriving from a wall moving at u: d_stored + 6 w_k (c_k.u).
__device__ __forceinline__ float wall_push(int k, float dstored, const float *u) {
    return __fmaf_rn(6.f * wf(k), cx(k) * u[0] + cy(k) * u[1] + cz(k) * u[2], dstored);
}

}  // namespace lbm
