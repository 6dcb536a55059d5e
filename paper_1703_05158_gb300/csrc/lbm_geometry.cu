// Node geometry and refill (Sect. 2.3), one CTA per sphere over its bounding
// box.
//
// flag[n] (bit 0 = solid):
//   0       fluid
//   1 or 3  solid, owner[n] = its sphere: the marks of a step of even step
//           count write 1, those of an odd step 3 (the mark value `cur` of
//           the step), so a solid node of the previous geometry that the
//           current marks did not take keeps the other value
//   2       fluid now, solid at the previous step (the refill turns nodes of
//           the other mark value into 2; the collide kernel turns 2 into 0)
//
//   mark:   nodes inside sphere p at the current centre, unless a
//           neighbouring sphere that also contains the node has a smaller
//           |x - X| - R (ties to the smaller index) -> cur, owner p
//   refill: nodes of sphere p left at the previous step's mark value take
//           the equilibrium (Eq. 9) at the surface velocity of p and at the
//           mean density of the neighbours fluid before and after (flag 0),
//           then become 2.
// After the refill every solid node carries the current mark value, and
// bit 0 is the fluid / solid class for every reader.
//
// Inside tests and keys are FP32 on relative coordinates
// (float)(x - b) - (float)(X - b), b = floor(X) (the sphere frames written
// by the DEM, see SFrame), evaluated with
// round-to-nearest intrinsics so that no multiply-add is contracted: the
// same operations, in the same order, as the FP64 oracle uses for its
// geometric decisions, so both sides classify every node identically.
#include "lbm_internal.cuh"

namespace lbm {

__device__ __forceinline__ float rel(int o, float fr) { return __fsub_rn((float)o, fr); }

__device__ __forceinline__ float dist2(float dx, float dy, float dz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Wrap a coordinate that is at most one box length outside [0, n).
__device__ __forceinline__ int wrapi(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// Offset of periodic coordinate x from base b, folded into [-n/2, n/2).
// Every caller passes a node coordinate x in [0, n) and the floor b of a
// centre in [0, n] (positions are wrapped into the box after each move),
// so x - b lies in [-n, n) and one conditional add replaces the remainder.
__device__ __forceinline__ int fold(int x, int b, int n) {
    int d = x - b;
    if (d < 0) d += n;
    if (2 * d >= n) d -= n;
    return d;
}

// Offsets (ox, oy, oz) in [0, B)^3 of box index t = ox + B (oy + B oz),
// advanced by a fixed stride with carries (one division per thread at the
// start, none per step).
struct BoxWalk {
    int ox, oy, oz, sx, sy, sz, B;
    __device__ __forceinline__ BoxWalk(int t, int stride, int b) : B(b) {
        ox = t % B;
        oy = (t / B) % B;
        oz = t / (B * B);
        sx = stride % B;
        sy = (stride / B) % B;
        sz = stride / (B * B);
    }
    __device__ __forceinline__ void next() {
        ox += sx;
        int c = ox >= B;
        if (c) ox -= B;
        oy += sy + c;
        c = oy >= B;
        if (c) oy -= B;
        oz += sz + c;
    }
};

// Half width of the box (around floor(X)) holding every node inside a sphere
// of FP32 radius R: offsets lie in [-ceil(R) + 1, ceil(R)].
__device__ __forceinline__ int ext_of(float R) { return (int)ceilf(R); }

constexpr int MAX_NBR_SMEM = 64;

// Momentum m of a node and its moment l x m, accumulated into acc[0..5]
// (sign +1 or -1); round-to-nearest intrinsics keep the compiler from
// contracting the cross products, so every kernel that inlines this rounds
// alike.
__device__ __forceinline__ double cross_rn(double a, double b, double c, double d) {
    return __dsub_rn(__dmul_rn(a, b), __dmul_rn(c, d));
}
__device__ __forceinline__ void add_moment(double *acc, double sign, float lx, float ly, float lz, double mx,
                                           double my, double mz) {
    const double m[6] = {mx, my, mz, cross_rn(ly, mz, lz, my), cross_rn(lz, mx, lx, mz), cross_rn(lx, my, ly, mx)};
#pragma unroll
    for (int a = 0; a < 6; ++a) acc[a] = sign > 0.0 ? __dadd_rn(acc[a], m[a]) : __dsub_rn(acc[a], m[a]);
}

// Node at offset (ox, oy, oz) from floor(X_p) (each in [-e, e]) if sphere p
// wins it, else -1.
__device__ __forceinline__ int mark_node(const Lat &L, const SFrame &F, const SFrame *nf, const int *nid,
                                         const int cnt, const int p, const int ox, const int oy, const int oz) {
    const int z = F.b[2] + oz;
    if (z < 0 || z >= L.nz) return -1;
    const float d2 = dist2(rel(ox, F.fr[0]), rel(oy, F.fr[1]), rel(oz, F.fr[2]));
    if (!(d2 < F.R2)) return -1;
    const float key = __fsub_rn(__fsqrt_rn(d2), F.R);
    const int x = wrapi(F.b[0] + ox, L.nx), y = wrapi(F.b[1] + oy, L.ny);
    for (int m = 0; m < cnt; ++m) {
        const SFrame &G = nf[m];
        const float e2 = dist2(rel(fold(x, G.b[0], L.nx), G.fr[0]), rel(fold(y, G.b[1], L.ny), G.fr[1]),
                               rel(z - G.b[2], G.fr[2]));
        if (!(e2 < G.R2)) continue;
        const float k2 = __fsub_rn(__fsqrt_rn(e2), G.R);
        if (k2 < key || (k2 == key && nid[m] < p)) return -1;
    }
    return x + L.nx * (y + L.ny * z);
}

// The plain marks: flag cur and owner p on every node sphere p wins.
__device__ __forceinline__ void mark_body(const Lat &L, const Parts &pt, const SFrame *__restrict__ fcur,
                                          uint8_t *__restrict__ flag, int32_t *__restrict__ owner, const uint8_t cur) {
    const int p = blockIdx.x;
    __shared__ SFrame nf[MAX_NBR_SMEM];
    __shared__ int nid[MAX_NBR_SMEM];
    const int cnt = min(pt.nbr_cnt[p], MAX_NBR_SMEM);
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const int q = pt.nbr[(long long)p * pt.max_nbr + t];
        nid[t] = q;
        nf[t] = fcur[q];
    }
    const SFrame F = fcur[p];
    __syncthreads();
    const int e = ext_of(F.R), B = 2 * e + 1, B3 = B * B * B;
    BoxWalk w(threadIdx.x, blockDim.x, B);
    for (int t = threadIdx.x; t < B3; t += blockDim.x, w.next()) {
        const int n = mark_node(L, F, nf, nid, cnt, p, w.ox - e, w.oy - e, w.oz - e);
        if (n < 0) continue;
        flag[n] = cur;
        owner[n] = p;
    }
}

// Marks with the optional momentum correction (Aidun, Lu & Ding 1998; not
// part of the paper): a node that was fluid (flag 0) and is now won by
// sphere p hands its momentum sum_i c_i f_i (read from the pre-collision
// slots of parity P) and the moment about X_p to the sphere.  Per round of
// kCovRound box offsets: the previous flags of the round's nodes are
// fetched into shared memory first (only p writes a node p wins, so these
// are the values before this step's marks), the marks compact the covered
// nodes, which are then put in ascending node order and summed one warp per
// node (lane i loads f_i); the CTA writes the total to Fcorr / Tcorr (zero
// when it covers nothing).  blockDim.x = 256.
template <typename T>
__device__ __forceinline__ void mark_corr_body(const Lat &L, const Parts &pt, const SFrame *__restrict__ fcur,
                                               uint8_t *__restrict__ flag, int32_t *__restrict__ owner,
                                               const T *__restrict__ f, const int P, const uint8_t cur) {
    constexpr int kCovRound = 1024;
    const int p = blockIdx.x;
    __shared__ SFrame nf[MAX_NBR_SMEM];
    __shared__ int nid[MAX_NBR_SMEM];
    __shared__ uint8_t prev[kCovRound];
    __shared__ int clist[kCovRound];
    __shared__ int ccount;
    __shared__ double wacc[8][6];  // per warp: its nodes' momentum and moment, in node order
    const int cnt = min(pt.nbr_cnt[p], MAX_NBR_SMEM);
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const int q = pt.nbr[(long long)p * pt.max_nbr + t];
        nid[t] = q;
        nf[t] = fcur[q];
    }
    const SFrame F = fcur[p];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x < 8 * 6) wacc[threadIdx.x / 6][threadIdx.x % 6] = 0.0;
    if (threadIdx.x == 0) ccount = 0;
    const int e = ext_of(F.R), B = 2 * e + 1, B3 = B * B * B;
    for (int t0 = 0; t0 < B3; t0 += kCovRound) {
        const int t1 = min(B3, t0 + kCovRound);
        for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
            const int z = F.b[2] + t / (B * B) - e;
            const int y = wrapi(F.b[1] + (t / B) % B - e, L.ny), x = wrapi(F.b[0] + t % B - e, L.nx);
            prev[t - t0] = z >= 0 && z < L.nz ? flag[x + L.nx * (y + L.ny * z)] : 1;
        }
        __syncthreads();
        for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
            const int n = mark_node(L, F, nf, nid, cnt, p, t % B - e, (t / B) % B - e, t / (B * B) - e);
            if (n < 0) continue;
            if (prev[t - t0] == 0) clist[atomicAdd(&ccount, 1)] = n;
            flag[n] = cur;
            owner[n] = p;
        }
        __syncthreads();
        const int total = ccount;
        __syncthreads();  // every thread has read ccount (and prev) before they are rewritten
        if (threadIdx.x == 0) ccount = 0;
        if (total == 0) continue;
        // ascending node order (the entries are distinct): rank, then scatter
        int v[kCovRound / 256], r[kCovRound / 256];
#pragma unroll
        for (int j = 0; j < kCovRound / 256; ++j) {
            const int k = threadIdx.x + 256 * j;
            r[j] = -1;
            if (k < total) {
                v[j] = clist[k];
                int rank = 0;
                for (int i = 0; i < total; ++i) rank += clist[i] < v[j];
                r[j] = rank;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kCovRound / 256; ++j)
            if (r[j] >= 0) clist[r[j]] = v[j];
        __syncthreads();
        for (int k = wid; k < total; k += nw) {
            const int m = clist[k];
            const int x = m % L.nx, y = (m / L.nx) % L.ny, z = m / (L.nx * L.ny);
            float d = 0.f;
            if (lane >= 1 && lane < Q) {
                const Nbr nb(L, x, y);
                d = Store<T>::ld(f + in_slot(L, nb, P, lane, (long long)m + L.plane));
            }
            float mx = lane < Q ? rcx(lane) * d : 0.f, my = lane < Q ? rcy(lane) * d : 0.f,
                  mz = lane < Q ? rcz(lane) * d : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mx += __shfl_xor_sync(0xffffffffu, mx, o);
                my += __shfl_xor_sync(0xffffffffu, my, o);
                mz += __shfl_xor_sync(0xffffffffu, mz, o);
            }
            if (lane == 0)
                add_moment(wacc[wid], 1.0, rel(fold(x, F.b[0], L.nx), F.fr[0]), rel(fold(y, F.b[1], L.ny), F.fr[1]),
                           rel(z - F.b[2], F.fr[2]), mx, my, mz);
        }
        __syncthreads();  // clist is rewritten by the next round
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int a = threadIdx.x;
        double sum = 0.0;
        for (int w = 0; w < nw; ++w) sum = __dadd_rn(sum, wacc[w][a]);
        (a < 3 ? pt.Fcorr : pt.Tcorr)[3 * p + a % 3] = sum;
    }
}

// CORR = false: the plain marks (no population reads); true: with the
// momentum correction where the argument corr (per instance) asks for it.
// Threads of the plain marks and refill (the momentum-correction forms keep
// 256: their node sorts assume it).
#ifndef LBM_GEOM_THREADS
#define LBM_GEOM_THREADS 128
#endif
constexpr int kGeomThreads = LBM_GEOM_THREADS;

// The plain forms are bounded so that the CTAs of a few thousand spheres
// are resident at once (one wave): 32 registers for the marks, 40 for the
// refill.
template <typename T, bool CORR>
__global__ void __launch_bounds__(CORR ? 256 : kGeomThreads, CORR ? 4 : 2048 / kGeomThreads) k_mark(const Lat L, const Parts pt, const SFrame *__restrict__ fcur,
                                              uint8_t *__restrict__ flag, int32_t *__restrict__ owner,
                                              const T *__restrict__ f, const int P, const int corr,
                                              const uint8_t cur) {
    if (CORR && corr) mark_corr_body<T>(L, pt, fcur, flag, owner, f, P, cur);
    else mark_body(L, pt, fcur, flag, owner, cur);
}

// Batched: instance blockIdx.y at step parity sp (also the population
// parity); block (0, i) also clears the instance's link / refill counters.
template <typename T, bool CORR>
__global__ void __launch_bounds__(256, CORR ? 4 : 8) k_mark_b(const Inst *__restrict__ I, const int sp) {
    const Inst &a = I[blockIdx.y];
    if (blockIdx.x == 0 && threadIdx.x < 2) a.ctr[threadIdx.x] = 0ull;
    if ((int)blockIdx.x >= a.pt.np) return;
    const uint8_t cur = mark_value(sp);
    if (CORR && a.pt.corr) mark_corr_body<T>(a.L, a.pt, a.pt.frame[sp], a.flag, a.owner, (const T *)a.f, sp, cur);
    else mark_body(a.L, a.pt, a.pt.frame[sp], a.flag, a.owner, cur);
}

// One CTA per sphere: collect the uncovered nodes of its previous bounding
// box, then one warp per node: lane i (1..18) sums the 19 populations of
// neighbour x + c_i if it is fluid before and after, the warp reduces the
// mean, and lanes 0..18 write the 19 equilibrium populations.
constexpr int kRefillCap = 512;

template <typename T, bool CORR>
__device__ __forceinline__ void refill_body(const Lat &L, const SFrame *__restrict__ fcur,
                                            const SFrame *__restrict__ fprev, T *__restrict__ f,
                                            uint8_t *__restrict__ flag, const int32_t *__restrict__ owner,
                                            const int P, unsigned long long *__restrict__ ctr,
                                            int *__restrict__ status, const Parts &pt, const uint8_t cur) {
    __shared__ int list[kRefillCap];
    const uint8_t prev_mark = (uint8_t)(4 - cur);  // the other mark value: the previous step's geometry
    __shared__ int count;
    const int p = blockIdx.x;
    const SFrame Fp = fprev[p];  // the node geometry of the previous step was built from this centre
    const int e = ext_of(Fp.R), B = 2 * e + 1;
    const int bx = Fp.b[0], by = Fp.b[1], bz = Fp.b[2];
    if (threadIdx.x == 0) count = 0;
    __syncthreads();
    // the box is scanned kScanBatch offsets per thread at a time, their
    // flags and owners loaded together (one memory round trip per batch)
    constexpr int kScanBatch = 4;
    const int B3 = B * B * B;
    BoxWalk w(threadIdx.x, blockDim.x, B);
    for (int t0 = threadIdx.x; t0 < B3; t0 += kScanBatch * blockDim.x) {
        int n[kScanBatch];
#pragma unroll
        for (int j = 0; j < kScanBatch; ++j) {
            const int z = bz + w.oz - e;
            const bool in = t0 + j * (int)blockDim.x < B3 && z >= 0 && z < L.nz;
            n[j] = in ? wrapi(bx + w.ox - e, L.nx) + L.nx * (wrapi(by + w.oy - e, L.ny) + L.ny * z) : -1;
            w.next();
        }
        uint8_t fl[kScanBatch];
        int32_t ow[kScanBatch];
#pragma unroll
        for (int j = 0; j < kScanBatch; ++j) {
            fl[j] = n[j] >= 0 ? flag[n[j]] : 0;
            ow[j] = n[j] >= 0 ? owner[n[j]] : -1;
        }
#pragma unroll
        for (int j = 0; j < kScanBatch; ++j) {
            if (fl[j] != prev_mark || ow[j] != p) continue;  // prev_mark is 1 or 3, never the 0 of a skipped offset
            const int k = atomicAdd(&count, 1);
            if (k < kRefillCap) list[k] = n[j];
            else atomicOr(status, ST_TILE);
        }
    }
    __syncthreads();
    if constexpr (CORR) {
        // with the correction, ascending node order (the entries are
        // distinct), so that the per-sphere sums below do not depend on timing
        const int cnt = min(count, kRefillCap);
        int v[kRefillCap / 256], r[kRefillCap / 256];
#pragma unroll
        for (int j = 0; j < kRefillCap / 256; ++j) {
            const int k = threadIdx.x + 256 * j;
            r[j] = -1;
            if (k < cnt && threadIdx.x < 256) {
                v[j] = list[k];
                int rank = 0;
                for (int i = 0; i < cnt; ++i) rank += list[i] < v[j];
                r[j] = rank;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kRefillCap / 256; ++j)
            if (r[j] >= 0) list[r[j]] = v[j];
        __syncthreads();
    }
    const int total = min(count, kRefillCap);
    if (total == 0) return;
    const SFrame F = fcur[p];  // current centre, velocity and spin, for the surface velocity
    const float *V = F.V, *W = F.W;
    const int lane = threadIdx.x & 31;
    __shared__ double wacc[8][6];  // with CORR, per warp: the momentum its refilled nodes take, in node order
    if (CORR && threadIdx.x < 8 * 6) wacc[threadIdx.x / 6][threadIdx.x % 6] = 0.0;
    if (CORR) __syncthreads();
    for (int k = threadIdx.x >> 5; k < total; k += blockDim.x >> 5) {
        const int n = list[k];
        const int x = n % L.nx, y = (n / L.nx) % L.ny, z = n / (L.nx * L.ny);
        float dr = 0.f;
        int ok = 0;
        if (lane >= 1 && lane < Q) {
            const int zz = z + rcz(lane);
            if (zz >= 0 && zz < L.nz) {
                const int yy = wrapi(y + rcy(lane), L.ny), xx = wrapi(x + rcx(lane), L.nx);
                const int m = xx + L.nx * (yy + L.ny * zz);
                // the neighbour's populations are loaded with its flag (every
                // node has its 19 slots), and summed only if it is fluid
                const uint8_t fm = flag[m];
                const Nbr nb(L, xx, yy);
                const long long sm = m + L.plane;
                float v[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) v[i] = Store<T>::ld(f + in_slot(L, nb, P, i, sm));
                if (fm == 0) {
#pragma unroll
                    for (int i = 0; i < Q; ++i) dr += v[i];
                    ok = 1;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dr += __shfl_xor_sync(0xffffffffu, dr, o);
            ok += __shfl_xor_sync(0xffffffffu, ok, o);
        }
        const float drho = ok ? dr / (float)ok : 0.f;
        const float rho = 1.f + drho;
        // surface velocity of the sphere at this node (current centre)
        const float lx = rel(fold(x, F.b[0], L.nx), F.fr[0]);
        const float ly = rel(fold(y, F.b[1], L.ny), F.fr[1]);
        const float lz = rel(z - F.b[2], F.fr[2]);
        const float ux = V[0] + (W[1] * lz - W[2] * ly);
        const float uy = V[1] + (W[2] * lx - W[0] * lz);
        const float uz = V[2] + (W[0] * ly - W[1] * lx);
        const float uu = ux * ux + uy * uy + uz * uz;
        if (lane < Q) {
            const int i = lane;
            const float cu = rcx(i) * ux + rcy(i) * uy + rcz(i) * uz;
            const float dq = (float)rw36(i) / 36.f * (drho + rho * (3.f * cu + 4.5f * cu * cu - 1.5f * uu));
            const Nbr nb(L, x, y);
            Store<T>::st(f + in_slot(L, nb, P, i, (long long)n + L.plane), dq);
        }
        if (lane == 0) {
            flag[n] = 2;
            atomicAdd(ctr + 1, 1ull);
            // momentum correction: the sphere pays the momentum rho u_s of
            // the equilibrium it leaves behind
            if (CORR && pt.corr)
                add_moment(wacc[threadIdx.x >> 5], -1.0, lx, ly, lz, __dmul_rn(rho, ux), __dmul_rn(rho, uy),
                           __dmul_rn(rho, uz));
        }
    }
    if (CORR && pt.corr) {
        __syncthreads();
        if (threadIdx.x < 6) {
            const int a = threadIdx.x;
            double sum = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum = __dadd_rn(sum, wacc[w][a]);
            double *dst = (a < 3 ? pt.Fcorr : pt.Tcorr) + 3 * p + a % 3;
            *dst = __dadd_rn(*dst, sum);
        }
    }
}

template <typename T, bool CORR>
__global__ void __launch_bounds__(CORR ? 256 : kGeomThreads, CORR ? 4 : 1280 / kGeomThreads) k_refill(const Lat L, const SFrame *__restrict__ fcur,
                                                const SFrame *__restrict__ fprev, T *__restrict__ f,
                                                uint8_t *__restrict__ flag, const int32_t *__restrict__ owner,
                                                const int P, unsigned long long *__restrict__ ctr,
                                                int *__restrict__ status, const Parts pt, const uint8_t cur) {
    refill_body<T, CORR>(L, fcur, fprev, f, flag, owner, P, ctr, status, pt, cur);
}

// Batched: instance blockIdx.y; parity P is also the step parity.
template <typename T, bool CORR>
__global__ void __launch_bounds__(256, CORR ? 4 : 5) k_refill_b(const Inst *__restrict__ I, const int P) {
    const Inst &a = I[blockIdx.y];
    if ((int)blockIdx.x >= a.pt.np) return;
    refill_body<T, CORR>(a.L, a.pt.frame[P], a.pt.frame[P ^ 1], (T *)a.f, a.flag, a.owner, P, a.ctr, a.status,
                         a.pt, mark_value(P));
}

// Near set of step s+1, from the centres the geometry of step s uses.
// The far-node collisions of step s+1 run while the link kernel of step s,
// the geometry of step s+1 and the near-node collisions of step s+1 run.
// Under the A-A layout a node's collision touches only its own 19 slot
// locations, so the far collisions are safe if every node whose locations
// those other kernels touch is near:
//   links of step s: a fluid node x_f next to a solid node and x_f - c_j,
//     both within Chebyshev distance 2 of a node inside a sphere of step s;
//   refill of step s+1: nodes of step s's spheres and their neighbours
//     (distance 1);
//   marks of step s+1 (flags read by the collide kernels): nodes inside the
//     spheres at the new centres, which moved < max_step < 2 since step s,
//     hence inside the distance-2 dilation of step s's spheres.
// A node within Chebyshev distance 2 of a point inside a sphere of radius R
// centred at X has sum_a max(0, |x_a - X_a| - 2)^2 < R^2; the test below
// adds `margin` to R for the FP32 rounding of the sphere test of k_mark.
// A group (2^shift nodes along x) is tagged when any of its nodes passes.
// Thread (0, 0) also clears the counts of the near and far lists the same
// stream builds next.
__global__ void __launch_bounds__(256) k_near_mark(const Lat L, const SFrame *__restrict__ fr, const float margin,
                                                   uint8_t *__restrict__ near, const uint8_t tag, const int ngx,
                                                   const int shift, int *__restrict__ count,
                                                   int *__restrict__ far_count) {
    const int p = blockIdx.x;
    if (p == 0 && threadIdx.x == 0) {
        *count = 0;
        *far_count = 0;
    }
    const SFrame F = fr[p];
    const float Rg = F.R + margin, R2 = Rg * Rg;
    // |ox - fr| < Rg + 2 with fr in [0, 1): ox in [-(ceil(Rg) + 2), ceil(Rg) + 2]
    const int e = (int)ceilf(Rg) + 3, B = 2 * e + 1;
    for (int t = threadIdx.x; t < B * B * B; t += blockDim.x) {
        const int oz = t / (B * B) - e, oy = (t / B) % B - e, ox = t % B - e;
        const int z = F.b[2] + oz;
        if (z < 0 || z >= L.nz) continue;
        const float ax = fmaxf(0.f, fabsf((float)ox - F.fr[0]) - 2.f);
        const float ay = fmaxf(0.f, fabsf((float)oy - F.fr[1]) - 2.f);
        const float az = fmaxf(0.f, fabsf((float)oz - F.fr[2]) - 2.f);
        if (!(ax * ax + ay * ay + az * az < R2)) continue;
        const int x = wrapi(F.b[0] + ox, L.nx), y = wrapi(F.b[1] + oy, L.ny);
        near[(y + L.ny * z) * ngx + (x >> shift)] = tag;
    }
}

// Compaction of the entries tagged `tag` into list[0 .. *count) and of the
// others into far[0 .. *far_count), each ascending within each 4096-entry
// chunk (one chunk per block, one atomic per list and block; the chunks land
// in any order).  Both counts must be 0 on entry.
constexpr int kListPerThread = 16;
__global__ void __launch_bounds__(256) k_near_list(const uint8_t *__restrict__ near, const uint8_t tag,
                                                   const long long N, int *__restrict__ list,
                                                   int *__restrict__ count, int *__restrict__ far,
                                                   int *__restrict__ far_count) {
    __shared__ int warp_sum[2][8];
    __shared__ int base[2];
    const long long n0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * kListPerThread;
    unsigned bits = 0, valid = 0;
    if (n0 + kListPerThread <= N) {
        const uint4 v = *(const uint4 *)(near + n0);  // chunk starts are multiples of 16 bytes
        const unsigned t4 = 0x01010101u * tag;
        const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned m = __vcmpeq4(w[k], t4);  // 0xff in each matching byte
            bits |= (((m >> 7) & 1u) | ((m >> 14) & 2u) | ((m >> 21) & 4u) | ((m >> 28) & 8u)) << (4 * k);
        }
        valid = 0xffffu;
    } else {
        for (int k = 0; k < kListPerThread && n0 + k < N; ++k) {
            valid |= 1u << k;
            if (near[n0 + k] == tag) bits |= 1u << k;
        }
    }
    unsigned sel[2] = {bits, valid & ~bits};  // near, far
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int c[2], inc[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        c[a] = __popc(sel[a]);
        inc[a] = c[a];  // inclusive scan over the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc[a], o);
            if (lane >= o) inc[a] += v;
        }
        if (lane == 31) warp_sum[a][wid] = inc[a];
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        const int a = threadIdx.x;
        int tot = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            const int v = warp_sum[a][k];
            warp_sum[a][k] = tot;
            tot += v;
        }
        base[a] = tot ? atomicAdd(a == 0 ? count : far_count, tot) : 0;
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        int *out = a == 0 ? list : far;
        int o = base[a] + warp_sum[a][wid] + inc[a] - c[a];
        unsigned b = sel[a];
        while (b) {
            const int k = __ffs(b) - 1;
            b &= b - 1;
            out[o++] = (int)(n0 + k);
        }
    }
}

int launch_near_mark(lbm_s *h, uint8_t *near, uint8_t tag, const SFrame *frames, int *list, int *count, int *far,
                     int *far_count, cudaStream_t stream) {
    k_near_mark<<<h->pt.np, 256, 0, stream>>>(h->L, frames, 0.05f, near, tag, h->near_ngx, h->near_shift, count,
                                              far_count);
    const long long per_block = 256ll * kListPerThread;
    const long long blocks = (h->near_groups + per_block - 1) / per_block;
    k_near_list<<<(unsigned)blocks, 256, 0, stream>>>(near, tag, h->near_groups, list, count, far, far_count);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

template <bool CORR>
int mark_launch(lbm_s *h, int P, int corr) {
    const SFrame *fcur = h->pt.frame[h->steps & 1];
    const uint8_t cur = mark_value((int)(h->steps & 1));
    const dim3 g(h->pt.np);
    const int nt = CORR ? 256 : kGeomThreads;
    switch (h->precision) {
        case LBM_FP32:
            k_mark<float, CORR><<<g, nt, 0, h->stream>>>(h->L, h->pt, fcur, h->flag, h->owner,
                                                           (const float *)h->f, P, corr, cur);
            break;
        case LBM_BF16_DEV:
            k_mark<__nv_bfloat16, CORR><<<g, nt, 0, h->stream>>>(h->L, h->pt, fcur, h->flag, h->owner,
                                                                   (const __nv_bfloat16 *)h->f, P, corr, cur);
            break;
        case LBM_FP16_DEV:
            k_mark<__half, CORR><<<g, nt, 0, h->stream>>>(h->L, h->pt, fcur, h->flag, h->owner,
                                                            (const __half *)h->f, P, corr, cur);
            break;
        default: return LBM_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int launch_mark(lbm_s *h, int P, int corr) {
    return corr ? mark_launch<true>(h, P, corr) : mark_launch<false>(h, P, 0);
}

template <typename T, bool CORR>
void refill_launch(lbm_s *h, int parity) {
    const SFrame *fcur = h->pt.frame[h->steps & 1], *fprev = h->pt.frame[(h->steps + 1) & 1];
    k_refill<T, CORR><<<h->pt.np, CORR ? 256 : kGeomThreads, 0, h->stream>>>(h->L, fcur, fprev, (T *)h->f, h->flag, h->owner, parity,
                                                         h->ctr, h->status, h->pt, mark_value((int)(h->steps & 1)));
}

int launch_refill(lbm_s *h, int parity) {
    const bool c = h->pt.corr != 0;
    switch (h->precision) {
        case LBM_FP32: c ? refill_launch<float, true>(h, parity) : refill_launch<float, false>(h, parity); break;
        case LBM_BF16_DEV:
            c ? refill_launch<__nv_bfloat16, true>(h, parity) : refill_launch<__nv_bfloat16, false>(h, parity);
            break;
        case LBM_FP16_DEV:
            c ? refill_launch<__half, true>(h, parity) : refill_launch<__half, false>(h, parity);
            break;
        default: return LBM_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

// Any member with the momentum correction selects the CORR kernels (each
// instance still follows its own flag).
static bool batch_corr(const lbm_batch_s *b) {
    for (int i = 0; i < b->n; ++i)
        if (b->m[i]->pt.corr) return true;
    return false;
}

template <typename T>
void geometry_batch(const lbm_batch_s *b, bool refill, bool corr, int P) {
    const dim3 grid(b->max_np, b->n);
    if (refill) {
        if (corr) k_refill_b<T, true><<<grid, 256, 0, b->stream>>>(b->dinst, P);
        else k_refill_b<T, false><<<grid, 256, 0, b->stream>>>(b->dinst, P);
    } else {
        if (corr) k_mark_b<T, true><<<grid, 256, 0, b->stream>>>(b->dinst, P);
        else k_mark_b<T, false><<<grid, 256, 0, b->stream>>>(b->dinst, P);
    }
}

static int geometry_batch_launch(const lbm_batch_s *b, bool refill, int P) {
    if (b->max_np == 0) return LBM_OK;
    const bool c = batch_corr(b);
    switch (b->precision) {
        case LBM_FP32: geometry_batch<float>(b, refill, c, P); break;
        case LBM_BF16_DEV: geometry_batch<__nv_bfloat16>(b, refill, c, P); break;
        case LBM_FP16_DEV: geometry_batch<__half>(b, refill, c, P); break;
        default: return LBM_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int launch_mark_batch(const lbm_batch_s *b, int sp) { return geometry_batch_launch(b, false, sp); }

int launch_refill_batch(const lbm_batch_s *b, int P) { return geometry_batch_launch(b, true, P); }

}  // namespace lbm
