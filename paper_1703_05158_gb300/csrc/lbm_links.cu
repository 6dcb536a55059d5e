// Interpolated bounce-back on sphere links and momentum exchange (Sect. 2.3),
// one CTA per sphere, run after the collide kernel of a step.
//
// The CTA stages a code per node of a cube around the sphere in shared
// memory (0 fluid, 1 other solid or outside the box, 2 owned by this sphere).
// Every pair (solid node s owned by the sphere, direction j) with x = s - c_j
// fluid is a cut link.  Its fraction q is the smallest root of
// |x + t c_j - X| = R in FP32, written as c0 / (-b + sqrt(b^2 - a c0)) and
// evaluated with the same round-to-nearest operations as the oracle.  The
// population k = opp(j) that x receives from the solid side is (Eq. 19 with
// the moving-boundary term of Eq. 21, deviations from w throughout):
//   q <  1/2, x - c_j fluid: 2q d^c_j(x) + (1-2q) d^c_j(x - c_j) + 6 w_j (c_k.u_b)
//   q <  1/2, otherwise:     d^c_j(x) + 6 w_j (c_k.u_b)
//   q >= 1/2:                d^c_j(x)/(2q) + (2q-1)/(2q) d^c_k(x) + (3/q) w_j (c_k.u_b)
// with u_b = V + Om x (x + q c_j - X).  It is written where the next step
// reads f_k(x).  All inputs are post-collision values of the finished step
// and all outputs are slots no other link reads, so links are independent.
//
// Momentum exchange (Eqs. 25, 26): the sphere receives
//   dP = (f^c_j(x) + f_k(x, t+1)) c_j,   torque (x_b - X) x dP,
// and with the Galilean-invariant option (Wen, Zhang & Fang 2014; not in the
// paper) also -(f^c_j(x) - f_k(x, t+1)) u_b.
// With f = w + d this splits into the deviation part (d^c_j + d_k) c_j,
// summed in FP32 per thread and per warp (shuffles), and the rest part
// 2 w_j c_j = (36 w_j / 18) c_j, counted exactly in integers; (x_b - X) x c_j
// = (x - X) x c_j since c_j x c_j = 0.  The CTA combines the warp sums in
// FP64 in a fixed order, so the force is deterministic.
#include <cmath>

#include "lbm_internal.cuh"

namespace lbm {

// Wrap a coordinate that is at most one box length outside [0, n).
__device__ __forceinline__ int wrap1(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// Tile index t -> offsets (ox, oy, oz) in [-ext, ext]; the divisions by B and
// B^2 use multiply-high with m = floor((2^32 - 1) / d) + 1, exact for the
// tile sizes here (t < 2^17, d <= 2^12).
__device__ __forceinline__ void tile_xyz(int t, int B, int B2, unsigned mB, unsigned mB2, int ext, int &ox, int &oy,
                                         int &oz) {
    const int z = (int)__umulhi((unsigned)t, mB2);
    const int r = t - z * B2;
    const int y = (int)__umulhi((unsigned)r, mB);
    ox = r - y * B - ext;
    oy = y - ext;
    oz = z - ext;
}

template <typename T, bool GI>
__device__ __forceinline__ void links_body(const Lat &L, const Parts &pt, const SFrame *__restrict__ fcur,
                                           T *__restrict__ f, uint8_t *__restrict__ flag,
                                           const int32_t *__restrict__ owner, const int P, const int ext,
                                           const unsigned mB, const unsigned mB2, const int cap,
                                           int *__restrict__ status, unsigned long long *__restrict__ ctr) {
    extern __shared__ unsigned char smem[];
    const int B = 2 * ext + 1, B2 = B * B, B3 = B2 * B;
    uint32_t *list = (uint32_t *)smem;            // cap entries: tile index << 5 | direction
    uint8_t *code = smem + 4 * (size_t)cap;       // B3 node codes
    uint16_t *nodes = (uint16_t *)(code + ((B3 + 15) & ~15));  // the sphere's own nodes, tile order
    const int ncap = (B3 + 1) / 2;                // a ball fills at most 52% of its cube
    __shared__ float redf[8][6];
    __shared__ int redi[8][6];
    __shared__ double sh[12];
    __shared__ int wsum[8];
    const int p = blockIdx.x;
    const SFrame Fr = fcur[p];
    const int b[3] = {Fr.b[0], Fr.b[1], Fr.b[2]};
    const float fr[3] = {Fr.fr[0], Fr.fr[1], Fr.fr[2]};
    const float R2 = Fr.R2;
    double Xp[3] = {0.0, 0.0, 0.0};
    if (threadIdx.x == 0)
        for (int a = 0; a < 3; ++a) Xp[a] = pt.X[3 * p + a];  // used by the final sums

    // 1. node codes of the tile: 0 fluid, 1 other solid / outside, 2 this sphere
    //    (kTileBatch nodes per thread per round so that their loads overlap)
    constexpr int kTileBatch = 12;
    for (int t0 = threadIdx.x; t0 < B3; t0 += kTileBatch * blockDim.x) {
        int nn[kTileBatch];
        uint8_t fl[kTileBatch];
#pragma unroll
        for (int u = 0; u < kTileBatch; ++u) {
            const int t = t0 + u * blockDim.x;
            nn[u] = -1;
            if (t < B3) {
                int ox, oy, oz;
                tile_xyz(t, B, B2, mB, mB2, ext, ox, oy, oz);
                const int z = b[2] + oz;
                if (z >= 0 && z < L.nz) {
                    const int y = wrap1(b[1] + oy, L.ny), x = wrap1(b[0] + ox, L.nx);
                    nn[u] = x + L.nx * (y + L.ny * z);
                }
            }
            fl[u] = nn[u] >= 0 ? __ldcg(flag + nn[u]) : (uint8_t)1;
        }
        int ow[kTileBatch];
#pragma unroll
        for (int u = 0; u < kTileBatch; ++u) ow[u] = (nn[u] >= 0 && (fl[u] & 1)) ? __ldcg(owner + nn[u]) : -1;
#pragma unroll
        for (int u = 0; u < kTileBatch; ++u) {
            const int t = t0 + u * blockDim.x;
            if (t < B3) code[t] = (fl[u] & 1) ? (ow[u] == p ? 2 : 1) : 0;
        }
    }
    __syncthreads();

    // 2. cut links (s owned, x = s - c_j fluid) into a list in tile order,
    //    direction minor.  (a) the sphere's own nodes are compacted in tile
    //    order (threads own contiguous tile ranges, one block scan); (b) the
    //    flattened (node, direction) pairs are tested in rounds of one pair per
    //    thread and the links appended with warp ballots, so no warp walks
    //    directions for nodes that are not its own.
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int chunk = (B3 + blockDim.x - 1) / blockDim.x;
    const int t_lo = min(B3, (int)threadIdx.x * chunk), t_hi = min(B3, t_lo + chunk);
    int mine = 0;
    for (int t = t_lo; t < t_hi; ++t) mine += code[t] == 2;
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    int nbase = 0, nn = 0;
    for (int w = 0; w < nw; ++w) {
        if (w < wid) nbase += wsum[w];
        nn += wsum[w];
    }
    {
        int pos = nbase + incl - mine;
        for (int t = t_lo; t < t_hi; ++t)
            if (code[t] == 2) {
                if (pos < ncap) nodes[pos] = (uint16_t)t;
                ++pos;
            }
    }
    if (nn > ncap && threadIdx.x == 0) atomicOr(status, ST_TILE);
    nn = min(nn, ncap);
    __syncthreads();
    // (b) thread i takes the owned nodes i, i + T, ... (tile order is kept
    //     because node k's links precede node k+1's): an unrolled test of the
    //     18 directions gives a mask, one block scan of the counts places them
    int total = 0, pos0 = 0;
    for (int k0 = 0; k0 < nn; k0 += blockDim.x) {
        const int k = k0 + threadIdx.x;
        unsigned mask = 0u;
        int t = 0;
        if (k < nn) {
            t = nodes[k];
#pragma unroll
            for (int j = 1; j < Q; ++j)
                if (code[t - (cx(j) + B * (cy(j) + B * cz(j)))] == 0) mask |= 1u << j;
        }
        const int c = __popc(mask);
        int inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) wsum[wid] = inc;
        __syncthreads();
        int off = total, round = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < wid) off += wsum[w];
            round += wsum[w];
        }
        int pos = off + inc - c;
        while (mask) {
            const int j = __ffs(mask) - 1;
            mask &= mask - 1u;
            if (pos < cap) list[pos] = ((uint32_t)t << 5) | (uint32_t)j;
            ++pos;
        }
        total += round;
        __syncthreads();
    }
    (void)pos0;
    if (total > cap && threadIdx.x == 0) atomicOr(status, ST_TILE);
    total = min(total, cap);
    __syncthreads();

    // 3. bounce-back and momentum exchange, links spread over the threads
    const float *V = Fr.V, *W = Fr.W;
    float Fd[3] = {0.f, 0.f, 0.f}, Td[3] = {0.f, 0.f, 0.f};
    int I[3] = {0, 0, 0}, J[3] = {0, 0, 0};
    const int S = (int)L.S, plane = (int)L.plane;
    // kLinkBatch links per thread per round: the fractions q are computed
    // first, then the two populations each link needs are loaded together
    constexpr int kLinkBatch = 6;
    for (int l0 = threadIdx.x; l0 < total; l0 += kLinkBatch * blockDim.x) {
        float ld[kLinkBatch][2], lq[kLinkBatch], ldx[kLinkBatch][3];
        int lt[kLinkBatch], lj[kLinkBatch], dst[kLinkBatch], lbr[kLinkBatch];
#pragma unroll
        for (int u = 0; u < kLinkBatch; ++u) {
            const int l = l0 + u * blockDim.x;
            lt[u] = -1;
            if (l >= total) continue;
            const uint32_t e = list[l];
            const int t = (int)(e >> 5), j = (int)(e & 31u), k = ropp(j);
            const int cjx = rcx(j), cjy = rcy(j), cjz = rcz(j);
            const int off = cjx + B * (cjy + B * cjz);
            int ox, oy, oz;
            tile_xyz(t, B, B2, mB, mB2, ext, ox, oy, oz);
            ox -= cjx;
            oy -= cjy;
            oz -= cjz;
            // link fraction q of the fluid node x = s - c_j (FP32, the oracle's operations)
            const float dx = __fsub_rn((float)ox, fr[0]), dy = __fsub_rn((float)oy, fr[1]),
                        dz = __fsub_rn((float)oz, fr[2]);
            const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
            const float qa = (float)(cjx * cjx + cjy * cjy + cjz * cjz);
            const float qb = __fadd_rn(__fadd_rn(__fmul_rn((float)cjx, dx), __fmul_rn((float)cjy, dy)),
                                       __fmul_rn((float)cjz, dz));
            const float c0 = __fsub_rn(d2, R2);
            float disc = __fsub_rn(__fmul_rn(qb, qb), __fmul_rn(qa, c0));
            if (disc < 0.f) disc = 0.f;
            float q = __fdiv_rn(c0, __fadd_rn(-qb, __fsqrt_rn(disc)));
            q = fminf(fmaxf(q, 0.f), 1.f);
            // branch of Eq. (19): 0 interpolate with x - c_j, 1 halfway fallback, 2 q >= 1/2
            const int br = q < 0.5f ? (code[t - 2 * off] == 0 ? 0 : 1) : 2;
            // storage indices of x, of the solid node s = x + c_j and of x - c_j
            const int xx = wrap1(b[0] + ox, L.nx), xy = wrap1(b[1] + oy, L.ny), xz = b[2] + oz;
            const int sx = xx + L.nx * (xy + L.ny * xz) + plane;
            const int ss = wrap1(xx + cjx, L.nx) + L.nx * (wrap1(xy + cjy, L.ny) + L.ny * (xz + cjz)) + plane;
            const int sb = wrap1(xx - cjx, L.nx) + L.nx * (wrap1(xy - cjy, L.ny) + L.ny * (xz - cjz)) + plane;
            // post-collision d^c_j(x) and, by branch, d^c_j(x - c_j) or d^c_k(x)
            ld[u][0] = Store<T>::ld(f + (P == 0 ? k * S + sx : j * S + ss));
            ld[u][1] = br == 1 ? 0.f
                               : Store<T>::ld(f + (br == 0 ? (P == 0 ? k * S + sb : j * S + sx)
                                                           : (P == 0 ? j * S + sx : k * S + sb)));
            dst[u] = P == 0 ? j * S + ss : k * S + sx;  // where the next step reads f_k(x)
            lt[u] = t;
            lj[u] = j;
            lq[u] = q;
            lbr[u] = br;
            ldx[u][0] = dx;
            ldx[u][1] = dy;
            ldx[u][2] = dz;
        }
#pragma unroll
        for (int u = 0; u < kLinkBatch; ++u) {
            if (lt[u] < 0) continue;
            const int t = lt[u], j = lj[u];
            const int cjx = rcx(j), cjy = rcy(j), cjz = rcz(j);
            int ox, oy, oz;
            tile_xyz(t, B, B2, mB, mB2, ext, ox, oy, oz);
            ox -= cjx;
            oy -= cjy;
            oz -= cjz;
            const float dx = ldx[u][0], dy = ldx[u][1], dz = ldx[u][2], q = lq[u];
            const float dcj = ld[u][0];
            const float lx = dx + q * cjx, ly = dy + q * cjy, lz = dz + q * cjz;
            const float ubx = V[0] + (W[1] * lz - W[2] * ly);
            const float uby = V[1] + (W[2] * lx - W[0] * lz);
            const float ubz = V[2] + (W[0] * ly - W[1] * lx);
            const float cku = -(cjx * ubx + cjy * uby + cjz * ubz);
            const float wj = (float)rw36(j) * (1.f / 36.f);
            float dn;
            if (lbr[u] == 0) {
                dn = 2.f * q * dcj + (1.f - 2.f * q) * ld[u][1] + 6.f * wj * cku;
            } else if (lbr[u] == 1) {
                dn = dcj + 6.f * wj * cku;
            } else {
                const float i2q = 0.5f / q;
                dn = dcj * i2q + (2.f * q - 1.f) * i2q * ld[u][1] + 3.f / q * wj * cku;
            }
            Store<T>::st(f + dst[u], dn);

            const float m = dcj + dn;
            Fd[0] += m * cjx;
            Fd[1] += m * cjy;
            Fd[2] += m * cjz;
            Td[0] += m * (dy * cjz - dz * cjy);
            Td[1] += m * (dz * cjx - dx * cjz);
            Td[2] += m * (dx * cjy - dy * cjx);
            if (GI && pt.gimea) {  // Galilean-invariant form: - (f^c_j - f_k) u_b, the weights cancel
                const float e = dcj - dn;
                Fd[0] -= e * ubx;
                Fd[1] -= e * uby;
                Fd[2] -= e * ubz;
                Td[0] -= e * (ly * ubz - lz * uby);
                Td[1] -= e * (lz * ubx - lx * ubz);
                Td[2] -= e * (lx * uby - ly * ubx);
            }
            const int w = rw36(j);
            I[0] += w * cjx;
            I[1] += w * cjy;
            I[2] += w * cjz;
            J[0] += w * (oy * cjz - oz * cjy);
            J[1] += w * (oz * cjx - ox * cjz);
            J[2] += w * (ox * cjy - oy * cjx);
        }
    }

    // 4. the nodes of this sphere become "owned at the previous geometry"
    //    (3: still solid for every reader) for the next step's mark pass
    for (int i = threadIdx.x; i < nn; i += blockDim.x) {
        int ox, oy, oz;
        tile_xyz(nodes[i], B, B2, mB, mB2, ext, ox, oy, oz);
        const int z = b[2] + oz, y = wrap1(b[1] + oy, L.ny), x = wrap1(b[0] + ox, L.nx);
        flag[x + L.nx * (y + L.ny * z)] = 3;
    }

    // 5. warp sums in FP32, then FP64 across warps in a fixed order
    float v[6] = {Fd[0], Fd[1], Fd[2], Td[0], Td[1], Td[2]};
    int iv[6] = {I[0], I[1], I[2], J[0], J[1], J[2]};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            v[a] += __shfl_xor_sync(0xffffffffu, v[a], o);
            iv[a] += __shfl_xor_sync(0xffffffffu, iv[a], o);
        }
    }
    if (lane == 0) {
        for (int a = 0; a < 6; ++a) {
            redf[wid][a] = v[a];
            redi[wid][a] = iv[a];
        }
    }
    __syncthreads();
    // lanes 0..11 of warp 0 each sum one component over the warps in FP64
    if (threadIdx.x < 12) {
        const int a = threadIdx.x;
        double sum = 0.0;
        for (int w = 0; w < nw; ++w) sum += a < 6 ? (double)redf[w][a] : (double)redi[w][a - 6];
        sh[a] = sum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double frac[3];
        for (int a = 0; a < 3; ++a) frac[a] = Xp[a] - (double)b[a];  // exact: X - floor(X)
        // rest part 2 w_j c_j: F = I/18, T = (J - frac x I)/18
        const double Ix = sh[6], Iy = sh[7], Iz = sh[8];
        double *F = pt.Fh + 3 * p, *Tq = pt.Th + 3 * p;
        constexpr double i18 = 1.0 / 18.0;
        F[0] = sh[0] + Ix * i18;
        F[1] = sh[1] + Iy * i18;
        F[2] = sh[2] + Iz * i18;
        Tq[0] = sh[3] + (sh[9] - (frac[1] * Iz - frac[2] * Iy)) * i18;
        Tq[1] = sh[4] + (sh[10] - (frac[2] * Ix - frac[0] * Iz)) * i18;
        Tq[2] = sh[5] + (sh[11] - (frac[0] * Iy - frac[1] * Ix)) * i18;
        if (pt.corr)  // momentum of the nodes covered / uncovered this step
            for (int a = 0; a < 3; ++a) {
                F[a] += pt.Fcorr[3 * p + a];
                Tq[a] += pt.Tcorr[3 * p + a];
            }
        atomicAdd(ctr, (unsigned long long)total);
    }
}

// GI: compiled with the Galilean-invariant momentum exchange (taken where
// the handle asks for it).
template <typename T, bool GI>
__global__ void __launch_bounds__(256, 3) k_links(const Lat L, const Parts pt, const SFrame *__restrict__ fcur,
                                               T *__restrict__ f,
                                               uint8_t *__restrict__ flag, const int32_t *__restrict__ owner,
                                               const int P, const int ext, const unsigned mB, const unsigned mB2,
                                               const int cap, int *__restrict__ status,
                                               unsigned long long *__restrict__ ctr) {
    links_body<T, GI>(L, pt, fcur, f, flag, owner, P, ext, mB, mB2, cap, status, ctr);
}

// Batched: instance blockIdx.y; parity P is also the step parity.
template <typename T, bool GI>
__global__ void __launch_bounds__(256, 3) k_links_b(const Inst *__restrict__ I, const int P, const int ext,
                                                 const unsigned mB, const unsigned mB2, const int cap) {
    const Inst &a = I[blockIdx.y];
    if ((int)blockIdx.x >= a.pt.np) return;
    links_body<T, GI>(a.L, a.pt, a.pt.frame[P], (T *)a.f, a.flag, a.owner, P, ext, mB, mB2, cap, a.status, a.ctr);
}

int link_capacity(double max_radius) {
    const double r = max_radius < 1.0 ? 1.0 : max_radius;
    return (int)std::ceil(80.0 * r * r) + 64;
}

size_t link_smem(int ext, int cap) {
    const size_t B = 2 * (size_t)ext + 1, B3 = B * B * B;
    return 4 * (size_t)cap + ((B3 + 15) & ~(size_t)15) + 2 * ((B3 + 1) / 2);
}

// Raise (never lower: other handles may need more) a kernel's dynamic
// shared memory limit to smem bytes.
template <typename K>
static cudaError_t raise_smem(K kernel, size_t smem) {
    cudaFuncAttributes at;
    cudaError_t e = cudaFuncGetAttributes(&at, kernel);
    if (e == cudaSuccess && at.maxDynamicSharedSizeBytes < (int)smem)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

template <bool GI>
static cudaError_t raise_all(size_t smem) {
    cudaError_t e = raise_smem(k_links<float, GI>, smem);
    if (e == cudaSuccess) e = raise_smem(k_links<__nv_bfloat16, GI>, smem);
    if (e == cudaSuccess) e = raise_smem(k_links<__half, GI>, smem);
    if (e == cudaSuccess) e = raise_smem(k_links_b<float, GI>, smem);
    if (e == cudaSuccess) e = raise_smem(k_links_b<__nv_bfloat16, GI>, smem);
    if (e == cudaSuccess) e = raise_smem(k_links_b<__half, GI>, smem);
    return e;
}

int links_setup(int ext, int cap) {
    const size_t smem = link_smem(ext, cap);
    cudaError_t e = raise_all<false>(smem);
    if (e == cudaSuccess) e = raise_all<true>(smem);
    if (e != cudaSuccess) cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

template <typename T, bool GI>
static void links_launch(lbm_s *h, int parity, size_t smem, const SFrame *fcur, int ext, unsigned mB, unsigned mB2,
                         int cap) {
    k_links<T, GI><<<h->pt.np, 256, smem, h->stream>>>(h->L, h->pt, fcur, (T *)h->f, h->flag, h->owner, parity, ext,
                                                       mB, mB2, cap, h->status, h->ctr);
}

template <typename T>
static void links_launch_t(lbm_s *h, int parity, size_t smem, const SFrame *fcur, int ext, unsigned mB, unsigned mB2,
                           int cap) {
    if (h->pt.gimea) links_launch<T, true>(h, parity, smem, fcur, ext, mB, mB2, cap);
    else links_launch<T, false>(h, parity, smem, fcur, ext, mB, mB2, cap);
}

int launch_links(lbm_s *h, int parity) {
    const int ext = h->tile_ext, cap = h->link_cap;
    const size_t smem = link_smem(ext, cap);
    const SFrame *fcur = h->pt.frame[h->steps & 1];
    const unsigned B = 2u * ext + 1u, mB = 0xFFFFFFFFu / B + 1u, mB2 = 0xFFFFFFFFu / (B * B) + 1u;
    switch (h->precision) {
        case LBM_FP32: links_launch_t<float>(h, parity, smem, fcur, ext, mB, mB2, cap); break;
        case LBM_BF16_DEV: links_launch_t<__nv_bfloat16>(h, parity, smem, fcur, ext, mB, mB2, cap); break;
        case LBM_FP16_DEV: links_launch_t<__half>(h, parity, smem, fcur, ext, mB, mB2, cap); break;
        default: return LBM_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int links_setup_batch(int ext, int cap) { return links_setup(ext, cap); }

// A batch with any member on the Galilean-invariant exchange takes the GI
// kernels; each instance still follows its own setting.
template <typename T>
static void links_launch_batch(const lbm_batch_s *b, int P, size_t smem, int ext, unsigned mB, unsigned mB2, int cap) {
    bool gi = false;
    for (int i = 0; i < b->n; ++i) gi = gi || b->m[i]->pt.gimea != 0;
    const dim3 grid(b->max_np, b->n);
    if (gi) k_links_b<T, true><<<grid, 256, smem, b->stream>>>(b->dinst, P, ext, mB, mB2, cap);
    else k_links_b<T, false><<<grid, 256, smem, b->stream>>>(b->dinst, P, ext, mB, mB2, cap);
}

int launch_links_batch(const lbm_batch_s *b, int P) {
    if (b->max_np == 0) return LBM_OK;
    const int ext = b->ext, cap = b->cap;
    const size_t smem = link_smem(ext, cap);
    const unsigned B = 2u * ext + 1u, mB = 0xFFFFFFFFu / B + 1u, mB2 = 0xFFFFFFFFu / (B * B) + 1u;
    switch (b->precision) {
        case LBM_FP32: links_launch_batch<float>(b, P, smem, ext, mB, mB2, cap); break;
        case LBM_BF16_DEV: links_launch_batch<__nv_bfloat16>(b, P, smem, ext, mB, mB2, cap); break;
        case LBM_FP16_DEV: links_launch_batch<__half>(b, P, smem, ext, mB, mB2, cap); break;
        default: return LBM_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

}  // namespace lbm
