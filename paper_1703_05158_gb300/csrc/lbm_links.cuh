// Interpolated bounce-back on sphere links and momentum exchange (Sect. 2.3)
// for one sphere per CTA, after the collide of its neighbourhood: the phases
// of the link kernels (lbm_links.cu).
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
#pragma once

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


// Geometry of a link CTA's tile: B = 2 ext + 1 nodes per edge around floor(X).
struct Tile {
    int ext, B, B2, B3;
    unsigned mB, mB2;
    __device__ __forceinline__ Tile(int e, unsigned mb, unsigned mb2)
        : ext(e), B(2 * e + 1), B2((2 * e + 1) * (2 * e + 1)), B3((2 * e + 1) * (2 * e + 1) * (2 * e + 1)), mB(mb),
          mB2(mb2) {}
    __device__ __forceinline__ void xyz(int t, int &ox, int &oy, int &oz) const {
        tile_xyz(t, B, B2, mB, mB2, ext, ox, oy, oz);
    }
    __device__ __forceinline__ int ncap() const { return (B3 + 1) / 2; }  // a ball fills at most 52% of its cube
};

// Which flags a link tile reads as solid.  cur == 0: bit 0 (every reader
// after the step's refill); cur != 0: exactly the mark value of the current
// geometry (while the refill may still be turning nodes of the previous
// geometry, which carry the other mark value, into fluid).
struct SolidOf {
    uint8_t cur;
    __device__ __forceinline__ bool operator()(uint8_t fl) const { return cur ? fl == cur : (fl & 1) != 0; }
};

// Shared memory of a CTA that builds a link list: the list (cap entries,
// tile index << 5 | direction), the node codes of the tile, the sphere's own
// nodes in tile order.
struct LinkShared {
    uint32_t *list;
    uint8_t *code;
    uint16_t *nodes;
    __device__ __forceinline__ LinkShared(unsigned char *smem, int cap, int B3)
        : list((uint32_t *)smem), code(smem + 4 * (size_t)cap), nodes((uint16_t *)(code + ((B3 + 15) & ~15))) {}
};

// 1. Node codes of sphere p's tile: 0 fluid, 1 other solid / outside the box,
//    2 owned by p (kTileBatch nodes per thread per round so that their loads
//    overlap).  Flags and owners are read through L2.
__device__ __forceinline__ void link_codes(const Lat &L, const int b[3], const uint8_t *__restrict__ flag,
                                           const int32_t *__restrict__ owner, const int p, const Tile &tl,
                                           const SolidOf solid, uint8_t *__restrict__ code) {
    constexpr int kTileBatch = 12;
    for (int t0 = threadIdx.x; t0 < tl.B3; t0 += kTileBatch * blockDim.x) {
        int nn[kTileBatch];
        uint8_t fl[kTileBatch];
#pragma unroll
        for (int u = 0; u < kTileBatch; ++u) {
            const int t = t0 + u * blockDim.x;
            nn[u] = -1;
            if (t < tl.B3) {
                int ox, oy, oz;
                tl.xyz(t, ox, oy, oz);
                const int z = b[2] + oz;
                if (z >= 0 && z < L.nz) {
                    const int y = wrap1(b[1] + oy, L.ny), x = wrap1(b[0] + ox, L.nx);
                    nn[u] = x + L.nx * (y + L.ny * z);
                }
            }
            fl[u] = nn[u] >= 0 ? __ldcg(flag + nn[u]) : (uint8_t)1;
        }
        bool sd[kTileBatch];
        int ow[kTileBatch];
#pragma unroll
        for (int u = 0; u < kTileBatch; ++u) {
            sd[u] = nn[u] < 0 || solid(fl[u]);
            ow[u] = (nn[u] >= 0 && sd[u]) ? __ldcg(owner + nn[u]) : -1;
        }
#pragma unroll
        for (int u = 0; u < kTileBatch; ++u) {
            const int t = t0 + u * blockDim.x;
            if (t < tl.B3) code[t] = sd[u] ? (ow[u] == p ? 2 : 1) : 0;
        }
    }
}

// 2. Cut links (s owned, x = s - c_j fluid) into sh.list in tile order,
//    direction minor; returns their count (at most cap).  (a) the sphere's
//    own nodes are compacted in tile order (threads own contiguous tile
//    ranges, one block scan); (b) thread i takes the owned nodes i, i + T,
//    ... (tile order is kept because node k's links precede node k+1's): an
//    unrolled test of the 18 directions gives a mask, one block scan of the
//    counts places them.  Starts and ends with a block barrier.
__device__ __forceinline__ int link_enumerate(const LinkShared &sh, const Tile &tl, const int cap,
                                              int *__restrict__ status) {
    __shared__ int wsum[8];
    __syncthreads();  // the codes are complete
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ncap = tl.ncap();
    const int chunk = (tl.B3 + blockDim.x - 1) / blockDim.x;
    const int t_lo = min(tl.B3, (int)threadIdx.x * chunk), t_hi = min(tl.B3, t_lo + chunk);
    int mine = 0;
    for (int t = t_lo; t < t_hi; ++t) mine += sh.code[t] == 2;
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
            if (sh.code[t] == 2) {
                if (pos < ncap) sh.nodes[pos] = (uint16_t)t;
                ++pos;
            }
    }
    if (nn > ncap && threadIdx.x == 0) atomicOr(status, ST_TILE);
    nn = min(nn, ncap);
    __syncthreads();
    int total = 0;
    for (int k0 = 0; k0 < nn; k0 += blockDim.x) {
        const int k = k0 + threadIdx.x;
        unsigned mask = 0u;
        int t = 0;
        if (k < nn) {
            t = sh.nodes[k];
#pragma unroll
            for (int j = 1; j < Q; ++j)
                if (sh.code[t - (cx(j) + tl.B * (cy(j) + tl.B * cz(j)))] == 0) mask |= 1u << j;
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
            if (pos < cap) sh.list[pos] = ((uint32_t)t << 5) | (uint32_t)j;
            ++pos;
        }
        total += round;
        __syncthreads();
    }
    if (total > cap && threadIdx.x == 0) atomicOr(status, ST_TILE);
    return min(total, cap);
}

// Relative position (FP32) of the fluid node x = s - c_j of link (t, j) to
// the sphere centre, and its tile offsets.
__device__ __forceinline__ void link_rel(const Tile &tl, const float fr[3], int t, int j, int &ox, int &oy, int &oz,
                                         float &dx, float &dy, float &dz) {
    tl.xyz(t, ox, oy, oz);
    ox -= rcx(j);
    oy -= rcy(j);
    oz -= rcz(j);
    dx = __fsub_rn((float)ox, fr[0]);
    dy = __fsub_rn((float)oy, fr[1]);
    dz = __fsub_rn((float)oz, fr[2]);
}

// Fraction q of link (t, j) (FP32, the oracle's operations: the smallest
// root of |x + q c_j - X| = R as c0 / (-b + sqrt(b^2 - a c0))) and the
// branch of Eq. (19): 0 interpolate with x - c_j, 1 halfway fallback (x - c_j
// not fluid), 2 q >= 1/2.
__device__ __forceinline__ void link_fraction(const Tile &tl, const float fr[3], const float R2,
                                              const uint8_t *__restrict__ code, int t, int j, float &q, int &br) {
    int ox, oy, oz;
    float dx, dy, dz;
    link_rel(tl, fr, t, j, ox, oy, oz, dx, dy, dz);
    const int cjx = rcx(j), cjy = rcy(j), cjz = rcz(j);
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    const float qa = (float)(cjx * cjx + cjy * cjy + cjz * cjz);
    const float qb =
        __fadd_rn(__fadd_rn(__fmul_rn((float)cjx, dx), __fmul_rn((float)cjy, dy)), __fmul_rn((float)cjz, dz));
    const float c0 = __fsub_rn(d2, R2);
    float disc = __fsub_rn(__fmul_rn(qb, qb), __fmul_rn(qa, c0));
    if (disc < 0.f) disc = 0.f;
    q = __fdiv_rn(c0, __fadd_rn(-qb, __fsqrt_rn(disc)));
    q = fminf(fmaxf(q, 0.f), 1.f);
    const int off = cjx + tl.B * (cjy + tl.B * cjz);
    br = q < 0.5f ? (code[t - 2 * off] == 0 ? 0 : 1) : 2;
}

// Per-thread partial sums of a CTA's links: the deviation part in FP32, the
// rest part 2 w_j c_j in integers (36 w_j c_j summed, divided by 18 at the end).
struct LinkAcc {
    float Fd[3] = {0.f, 0.f, 0.f}, Td[3] = {0.f, 0.f, 0.f};
    int I[3] = {0, 0, 0}, J[3] = {0, 0, 0};
};

// 3. Bounce-back and momentum exchange of links l = threadIdx.x,
//    threadIdx.x + blockDim.x, ... < total of the sphere with frame Fr;
//    src(l, t, j, q, br) gives link l.  BATCH links per thread per round
//    have their populations in flight together; CG: populations read
//    through L2 only.  Every product and sum is an explicit round-to-nearest
//    operation, so each kernel that inlines this rounds alike.
template <typename T, bool GI, int BATCH, bool CG, typename Src>
__device__ __forceinline__ void link_apply(const Lat &L, const Parts &pt, const SFrame &Fr, T *__restrict__ f,
                                           const int P, const Tile &tl, const int total, Src src, LinkAcc &acc) {
    const int S = (int)L.S, plane = (int)L.plane;
    for (int l0 = threadIdx.x; l0 < total; l0 += BATCH * blockDim.x) {
        float ld[BATCH][2], lq[BATCH];
        int lt[BATCH], lj[BATCH], dst[BATCH], lbr[BATCH];
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            const int l = l0 + u * blockDim.x;
            lt[u] = -1;
            if (l >= total) continue;
            int t, j, br;
            float q;
            src(l, t, j, q, br);
            const int k = ropp(j), cjx = rcx(j), cjy = rcy(j), cjz = rcz(j);
            int ox, oy, oz;
            tl.xyz(t, ox, oy, oz);
            ox -= cjx;
            oy -= cjy;
            oz -= cjz;
            // storage indices of x, of the solid node s = x + c_j and of x - c_j
            const int xx = wrap1(Fr.b[0] + ox, L.nx), xy = wrap1(Fr.b[1] + oy, L.ny), xz = Fr.b[2] + oz;
            const int sx = xx + L.nx * (xy + L.ny * xz) + plane;
            const int ss = wrap1(xx + cjx, L.nx) + L.nx * (wrap1(xy + cjy, L.ny) + L.ny * (xz + cjz)) + plane;
            const int sb = wrap1(xx - cjx, L.nx) + L.nx * (wrap1(xy - cjy, L.ny) + L.ny * (xz - cjz)) + plane;
            // post-collision d^c_j(x) and, by branch, d^c_j(x - c_j) or d^c_k(x)
            const T *a0 = f + (P == 0 ? k * S + sx : j * S + ss);
            const T *a1 = f + (br == 0 ? (P == 0 ? k * S + sb : j * S + sx) : (P == 0 ? j * S + sx : k * S + sb));
            ld[u][0] = CG ? Store<T>::ldcg(a0) : Store<T>::ld(a0);
            ld[u][1] = br == 1 ? 0.f : (CG ? Store<T>::ldcg(a1) : Store<T>::ld(a1));
            dst[u] = P == 0 ? j * S + ss : k * S + sx;  // where the next step reads f_k(x)
            lt[u] = t;
            lj[u] = j;
            lq[u] = q;
            lbr[u] = br;
        }
        const float *V = Fr.V, *W = Fr.W;
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            if (lt[u] < 0) continue;
            const int t = lt[u], j = lj[u];
            const float fj[3] = {(float)rcx(j), (float)rcy(j), (float)rcz(j)};
            int ox, oy, oz;
            float dx, dy, dz;
            link_rel(tl, Fr.fr, t, j, ox, oy, oz, dx, dy, dz);
            const float q = lq[u], dcj = ld[u][0];
            // boundary point x_b = x + q c_j relative to X, and its velocity u_b = V + Om x (x_b - X)
            const float lx = __fadd_rn(dx, fj[0] * q), ly = __fadd_rn(dy, fj[1] * q), lz = __fadd_rn(dz, fj[2] * q);
            const float ubx = __fadd_rn(V[0], __fsub_rn(__fmul_rn(W[1], lz), __fmul_rn(W[2], ly)));
            const float uby = __fadd_rn(V[1], __fsub_rn(__fmul_rn(W[2], lx), __fmul_rn(W[0], lz)));
            const float ubz = __fadd_rn(V[2], __fsub_rn(__fmul_rn(W[0], ly), __fmul_rn(W[1], lx)));
            const float cku = -__fadd_rn(__fadd_rn(fj[0] * ubx, fj[1] * uby), fj[2] * ubz);  // c_k = -c_j
            const float wj = (float)rw36(j) * (1.f / 36.f);
            const float q2 = 2.f * q;  // exact
            float dn;
            if (lbr[u] == 0) {
                dn = __fadd_rn(__fadd_rn(__fmul_rn(q2, dcj), __fmul_rn(__fsub_rn(1.f, q2), ld[u][1])),
                               __fmul_rn(__fmul_rn(6.f, wj), cku));
            } else if (lbr[u] == 1) {
                dn = __fadd_rn(dcj, __fmul_rn(__fmul_rn(6.f, wj), cku));
            } else {
                const float i2q = __fdiv_rn(0.5f, q);
                dn = __fadd_rn(__fadd_rn(__fmul_rn(dcj, i2q), __fmul_rn(__fmul_rn(__fsub_rn(q2, 1.f), i2q), ld[u][1])),
                               __fmul_rn(__fmul_rn(__fdiv_rn(3.f, q), wj), cku));
            }
            Store<T>::st(f + dst[u], dn);

            const float m = __fadd_rn(dcj, dn);
            const float cxr[3] = {__fsub_rn(dy * fj[2], dz * fj[1]), __fsub_rn(dz * fj[0], dx * fj[2]),
                                  __fsub_rn(dx * fj[1], dy * fj[0])};  // (x - X) x c_j
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                acc.Fd[a] = __fadd_rn(acc.Fd[a], m * fj[a]);
                acc.Td[a] = __fmaf_rn(m, cxr[a], acc.Td[a]);
            }
            if (GI && pt.gimea) {  // Galilean-invariant form: - (f^c_j - f_k) u_b, the weights cancel
                const float e = __fsub_rn(dcj, dn);
                const float ub[3] = {ubx, uby, ubz};
                const float lxu[3] = {__fsub_rn(__fmul_rn(ly, ubz), __fmul_rn(lz, uby)),
                                      __fsub_rn(__fmul_rn(lz, ubx), __fmul_rn(lx, ubz)),
                                      __fsub_rn(__fmul_rn(lx, uby), __fmul_rn(ly, ubx))};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    acc.Fd[a] = __fmaf_rn(-e, ub[a], acc.Fd[a]);
                    acc.Td[a] = __fmaf_rn(-e, lxu[a], acc.Td[a]);
                }
            }
            const int w = rw36(j), cjx = rcx(j), cjy = rcy(j), cjz = rcz(j);
            acc.I[0] += w * cjx;
            acc.I[1] += w * cjy;
            acc.I[2] += w * cjz;
            acc.J[0] += w * (oy * cjz - oz * cjy);
            acc.J[1] += w * (oz * cjx - ox * cjz);
            acc.J[2] += w * (ox * cjy - oy * cjx);
        }
    }
}

// 4. Warp sums in FP32, then FP64 across warps in a fixed order; thread 0
//    writes sphere p's load (plus the covered / uncovered-node momentum of
//    the step with the correction) and counts its links.
__device__ __forceinline__ void link_reduce_store(const Parts &pt, const int p, const int b[3], const LinkAcc &acc,
                                                  const int total, unsigned long long *__restrict__ ctr) {
    __shared__ float redf[8][6];
    __shared__ int redi[8][6];
    __shared__ double sh[12];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float v[6] = {acc.Fd[0], acc.Fd[1], acc.Fd[2], acc.Td[0], acc.Td[1], acc.Td[2]};
    int iv[6] = {acc.I[0], acc.I[1], acc.I[2], acc.J[0], acc.J[1], acc.J[2]};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            v[a] = __fadd_rn(v[a], __shfl_xor_sync(0xffffffffu, v[a], o));
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
        for (int w = 0; w < nw; ++w) sum = __dadd_rn(sum, a < 6 ? (double)redf[w][a] : (double)redi[w][a - 6]);
        sh[a] = sum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double frac[3];
        for (int a = 0; a < 3; ++a) frac[a] = pt.X[3 * p + a] - (double)b[a];  // exact: X - floor(X)
        // rest part 2 w_j c_j: F = I/18, T = (J - frac x I)/18
        const double Ix = sh[6], Iy = sh[7], Iz = sh[8];
        double *F = pt.Fh + 3 * p, *Tq = pt.Th + 3 * p;
        constexpr double i18 = 1.0 / 18.0;
        const double Iv[3] = {Ix, Iy, Iz};
        const double fxI[3] = {__dsub_rn(__dmul_rn(frac[1], Iz), __dmul_rn(frac[2], Iy)),
                               __dsub_rn(__dmul_rn(frac[2], Ix), __dmul_rn(frac[0], Iz)),
                               __dsub_rn(__dmul_rn(frac[0], Iy), __dmul_rn(frac[1], Ix))};
        for (int a = 0; a < 3; ++a) {
            double Fa = __dadd_rn(sh[a], __dmul_rn(Iv[a], i18));
            double Ta = __dadd_rn(sh[3 + a], __dmul_rn(__dsub_rn(sh[9 + a], fxI[a]), i18));
            if (pt.corr) {  // momentum of the nodes covered / uncovered this step
                Fa = __dadd_rn(Fa, pt.Fcorr[3 * p + a]);
                Ta = __dadd_rn(Ta, pt.Tcorr[3 * p + a]);
            }
            F[a] = Fa;
            Tq[a] = Ta;
        }
        atomicAdd(ctr, (unsigned long long)total);
    }
}

// The links of sphere p in one pass (one CTA, at most 256 threads): node
// codes, link list, bounce-back and momentum exchange, per-sphere sums.  Run
// after the step's collide and refill.
template <typename T, bool GI, int BATCH = 6, bool CG = false>
__device__ __forceinline__ void links_body(const Lat &L, const Parts &pt, const SFrame *__restrict__ fcur,
                                           T *__restrict__ f, const uint8_t *__restrict__ flag,
                                           const int32_t *__restrict__ owner, const int P, const int ext,
                                           const int cap, int *__restrict__ status,
                                           unsigned long long *__restrict__ ctr, const int p) {
    extern __shared__ unsigned char smem[];
    const SFrame Fr = fcur[p];
    // The sphere's own tile: its solid nodes lie within ceil(R) of floor(X)
    // (the marks' box), their links' fluid nodes x = s - c_j and x - c_j
    // within two more.  ext (shared memory is sized for it) bounds it; a
    // small sphere among large ones scans only its own box.  Nodes are
    // listed in (z, y, x) order whatever the extent, so the link list, and
    // every sum over it, is the same for any extent that holds the sphere.
    const int e = min(ext, (int)ceilf(Fr.R) + 2);
    const unsigned B = 2u * (unsigned)e + 1u;
    const Tile tl(e, 0xFFFFFFFFu / B + 1u, 0xFFFFFFFFu / (B * B) + 1u);
    const LinkShared sh(smem, cap, tl.B3);
    link_codes(L, Fr.b, flag, owner, p, tl, SolidOf{0}, sh.code);
    const int total = link_enumerate(sh, tl, cap, status);
    // Launched as a programmatic dependent of the collide, the CTA may start
    // while the collide's last blocks run: the codes and the list read only
    // the marks (a refilled node's flag turns from 2 to 0 in the collide,
    // fluid either way), the populations only after the collide grid has
    // completed and its writes are visible.  In an ordinary launch this
    // wait returns at once.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    LinkAcc acc;
    link_apply<T, GI, BATCH, CG>(L, pt, Fr, f, P, tl, total,
                                 [&](int l, int &t, int &j, float &q, int &br) {
                                     const uint32_t e = sh.list[l];
                                     t = (int)(e >> 5);
                                     j = (int)(e & 31u);
                                     link_fraction(tl, Fr.fr, Fr.R2, sh.code, t, j, q, br);
                                 },
                                 acc);
    link_reduce_store(pt, p, Fr.b, acc, total, ctr);
}

}  // namespace lbm
