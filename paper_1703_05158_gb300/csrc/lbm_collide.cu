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
#include "lbm_collide_node.cuh"

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

// Stream-collide of node (x, y, z), index n, flag fl: load (A-A addressing
// of parity ODD), collide, store, and push the wall populations.
template <int ODD, typename T>
__device__ __forceinline__ void sc_node(const Lat &L, const Phys &ph, T *__restrict__ f, uint8_t *__restrict__ flag,
                                        int *__restrict__ status, const int x, const int y, const int z, const int n,
                                        const uint8_t fl) {
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

    collide_node(ph, d, status);

#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int a = ODD ? i * S + s + nb(cx(i), cy(i), cz(i)) : opp(i) * S + s;
        Store<T>::st(f + a, d[i]);
    }

    // Walls: push the halfway bounce-back population into the slot the next
    // step (parity !ODD) reads for the direction coming from the wall, from
    // the post-collision value as stored.
    if (z == 0) {
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            if (cz(k) != 1) continue;
            const float v = wall_push(k, Store<T>::rt(d[opp(k)]), ph.ulo);
            const int a = ODD ? k * S + s : opp(k) * S + s + nb(-cx(k), -cy(k), -cz(k));
            Store<T>::st(f + a, v);
        }
    }
    if (z == L.nz - 1) {
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            if (cz(k) != -1) continue;
            const float v = wall_push(k, Store<T>::rt(d[opp(k)]), ph.uhi);
            const int a = ODD ? k * S + s : opp(k) * S + s + nb(-cx(k), -cy(k), -cz(k));
            Store<T>::st(f + a, v);
        }
    }
}

// Group tags of the overlapped schedule (lbm_capi.cu): node x of row r is
// in group r * ngx + (x >> shift).
struct NearMap {
    const uint8_t *tags;
    int ngx, shift;
    uint8_t tag;
    __device__ __forceinline__ bool near(int row, int x) const { return tags[row * ngx + (x >> shift)] == tag; }
};

// MODE 0: every fluid node; 1: only nodes of groups not tagged near (the
// far nodes of the overlapped schedule).
template <int ODD, typename T, int MODE>
__global__ void __launch_bounds__(256, 4) k_stream_collide(const Lat L, const Phys ph, T *__restrict__ f,
                                                        uint8_t *__restrict__ flag, int *__restrict__ status,
                                                        const NearMap nm) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= L.nx) return;
    const int row = y + L.ny * z;
    const int n = x + L.nx * row;
    const uint8_t fl = flag[n];  // both loads issued before either is tested
    if (MODE == 1 && nm.near(row, x)) return;
    sc_node<ODD, T>(L, ph, f, flag, status, x, y, z, n, fl);
}

// The nodes of the groups in a list (the near groups of the overlapped
// schedule), *count groups, grid-stride with one thread per node, so a
// warp covers whole 32-byte sectors of each slot row; coordinates by exact
// multiply-high division.
template <int ODD, typename T>
__global__ void __launch_bounds__(256, 4) k_collide_list(const Lat L, const Phys ph, T *__restrict__ f,
                                                      uint8_t *__restrict__ flag, int *__restrict__ status,
                                                      const int *__restrict__ list, const int *__restrict__ count,
                                                      const int ngx, const int shift, const FastDiv dngx,
                                                      const FastDiv dny) {
    const int total = *count << shift;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int g = list[t >> shift];
        const int row = (int)dngx.div((unsigned)g);
        const int x = ((g - row * ngx) << shift) | (t & ((1 << shift) - 1));
        if (x >= L.nx) continue;
        const int z = (int)dny.div((unsigned)row);
        const int n = x + L.nx * row;
        sc_node<ODD, T>(L, ph, f, flag, status, x, row - z * L.ny, z, n, flag[n]);
    }
}

// Batched form: every node of every instance, one persistent launch.  Chunk
// c = (instance, first node) covers TPB consecutive nodes of one instance
// (a block's threads, coalesced); block b takes the contiguous chunk range
// [b n / G, (b + 1) n / G).  The current instance's descriptor is staged in
// shared memory (read on use, not held in registers).  MINB resident blocks
// per SM bound the registers (64 per thread at TPB * MINB = 1024, 85 at
// 768); the autotuner picks both.
template <int ODD, typename T, int TPB, int MINB>
__global__ void __launch_bounds__(TPB, MINB) k_collide_batch(const Inst *__restrict__ I,
                                                                   const int2 *__restrict__ chunks, const int nchunks) {
    __shared__ __align__(16) unsigned char si_raw[sizeof(Inst)];
    Inst &si = *reinterpret_cast<Inst *>(si_raw);
    const int c0 = (int)((long long)nchunks * blockIdx.x / gridDim.x);
    const int c1 = (int)((long long)nchunks * (blockIdx.x + 1) / gridDim.x);
    int cur = -1;
    for (int c = c0; c < c1; ++c) {
        const int2 ch = chunks[c];
        if (ch.x != cur) {
            __syncthreads();
            const unsigned *src = (const unsigned *)(I + ch.x);
            unsigned *dst = (unsigned *)&si;
            for (int w = threadIdx.x; w < (int)(sizeof(Inst) / 4); w += TPB) dst[w] = src[w];
            __syncthreads();
            cur = ch.x;
        }
        const int n = ch.y + (int)threadIdx.x;
        if (n >= (int)si.L.N) continue;
        const int row = (int)si.dnx.div((unsigned)n);
        const int z = (int)si.dny.div((unsigned)row);
        sc_node<ODD, T>(si.L, si.ph, (T *)si.f, si.flag, si.status, n - row * si.L.nx, row - z * si.L.ny, z, n,
                        si.flag[n]);
    }
}

// The same with the instances' parameters in a kernel-parameter table (up to
// kCollideTable members): no shared-memory staging, and the constants are
// read through the constant cache as in the single-instance kernel.
template <int ODD, typename T, int TPB, int MINB>
__global__ void __launch_bounds__(TPB, MINB) k_collide_batch_tab(const __grid_constant__ CollideTable tab,
                                                                  const int2 *__restrict__ chunks,
                                                                  const int nchunks) {
    const int c0 = (int)((long long)nchunks * blockIdx.x / gridDim.x);
    const int c1 = (int)((long long)nchunks * (blockIdx.x + 1) / gridDim.x);
    for (int c = c0; c < c1; ++c) {
        const int2 ch = chunks[c];
        const CInst &ci = tab.c[ch.x];
        const int n = ch.y + (int)threadIdx.x;
        if (n >= (int)ci.L.N) continue;
        const int row = (int)ci.dnx.div((unsigned)n);
        const int z = (int)ci.dny.div((unsigned)row);
        sc_node<ODD, T>(ci.L, ci.ph, (T *)ci.f, ci.flag, ci.status, n - row * ci.L.nx, row - z * ci.L.ny, z, n,
                        ci.flag[n]);
    }
}

// 16-bit storage, two nodes (x, x+1), x even, per thread: each slot pair is
// one aligned 32-bit word.  Even steps read and write the node's own words.
// Odd steps read slot opp(i) at x - c_i: for c_x(i) = 0 that is again one
// word; for c_x(i) = +-1 the pair straddles two aligned words, of which the
// needed halves are taken; the post-collision pair goes to x + c_i, as one
// word for c_x = 0 and as two 16-bit stores otherwise.  Requires even nx.
template <typename T>
struct Pack2;
template <>
struct Pack2<__nv_bfloat16> {
    static __device__ __forceinline__ float lo(unsigned w) { return __uint_as_float(w << 16); }
    static __device__ __forceinline__ float hi(unsigned w) { return __uint_as_float(w & 0xffff0000u); }
    static __device__ __forceinline__ unsigned short bits(float v) {
        return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
};
template <>
struct Pack2<__half> {
    static __device__ __forceinline__ float lo(unsigned w) {
        __half2 h;
        *reinterpret_cast<unsigned *>(&h) = w;
        return __low2float(h);
    }
    static __device__ __forceinline__ float hi(unsigned w) {
        __half2 h;
        *reinterpret_cast<unsigned *>(&h) = w;
        return __high2float(h);
    }
    static __device__ __forceinline__ unsigned short bits(float v) { return __half_as_ushort(__float2half_rn(v)); }
};

template <int ODD, typename T, int MODE>
__global__ void __launch_bounds__(128, 8) k_stream_collide2(const Lat L, const Phys ph, T *__restrict__ f,
                                                            uint8_t *__restrict__ flag, int *__restrict__ status,
                                                            const NearMap nm) {
    const int hx = L.nx >> 1;  // pairs per row
    const int xp = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (xp >= hx) return;
    const int x = 2 * xp;
    const int n = x + L.nx * (y + L.ny * z);
    const unsigned short fl2 = *(const unsigned short *)(flag + n);
    const uint8_t fla = (uint8_t)(fl2 & 0xff), flb = (uint8_t)(fl2 >> 8);
    // x even and the group size even: both nodes are in one group
    const bool sel = MODE == 0 || !nm.near(y + L.ny * z, x);
    const bool liveA = sel && !(fla & 1), liveB = sel && !(flb & 1);
    if (!liveA && !liveB) return;
    if (liveA && fla) flag[n] = 0;
    if (liveB && flb) flag[n + 1] = 0;
    const int s = n + (int)L.plane;  // storage index of node x (even)
    const int S = (int)L.S;
    const unsigned *fw = (const unsigned *)f;  // word w holds nodes 2w, 2w+1 of a slot row
    unsigned short *fh = (unsigned short *)f;
    // word offsets (in units of pairs) of the neighbouring rows / pairs
    const int wl = xp == 0 ? hx - 1 : -1, wr = xp == hx - 1 ? 1 - hx : 1;
    const int rowm = y == 0 ? hx * (L.ny - 1) : -hx, rowp = y == L.ny - 1 ? -hx * (L.ny - 1) : hx;
    const int plw = (int)(L.plane >> 1);
    auto roff = [&](int oy, int oz) { return (oy < 0 ? rowm : (oy > 0 ? rowp : 0)) + oz * plw; };
    const int sw = s >> 1;  // word index of the pair (x, x+1)
    unsigned wv[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (!ODD) {
            wv[i] = fw[(i * S >> 1) + sw];
        } else {
            // pair (x, x+1) - c_i of slot opp(i)
            const int base = (opp(i) * S >> 1) + sw + roff(-cy(i), -cz(i));
            if (cx(i) == 0) {
                wv[i] = fw[base];
            } else if (cx(i) > 0) {  // nodes x-1, x: high half of the left word, low half of this word
                const unsigned a = fw[base + wl], b = fw[base];
                wv[i] = (a >> 16) | (b << 16);
            } else {  // nodes x+1, x+2: high half of this word, low half of the right word
                const unsigned a = fw[base], b = fw[base + wr];
                wv[i] = (a >> 16) | (b << 16);
            }
        }
    }
    // collide node x, then node x+1, each result packed back into its half
    // of the word it came from (the other half still holds the other input)
    float d[Q];
    if (liveA) {
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = Pack2<T>::lo(wv[i]);
        collide_node(ph, d, status);
#pragma unroll
        for (int i = 0; i < Q; ++i) wv[i] = __byte_perm(wv[i], (unsigned)Pack2<T>::bits(d[i]), 0x3254);
    }
    if (liveB) {
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = Pack2<T>::hi(wv[i]);
        collide_node(ph, d, status);
#pragma unroll
        for (int i = 0; i < Q; ++i) wv[i] = __byte_perm(wv[i], (unsigned)Pack2<T>::bits(d[i]), 0x5410);
    }
    // write: even -> slot opp(i) of the pair; odd -> slot i at (x, x+1) + c_i
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const unsigned short oa = (unsigned short)(wv[i] & 0xffffu), ob = (unsigned short)(wv[i] >> 16);
        if (!ODD) {
            const int w = (opp(i) * S >> 1) + sw;
            if (liveA && liveB)
                ((unsigned *)f)[w] = wv[i];
            else if (liveA)
                fh[2 * w] = oa;
            else
                fh[2 * w + 1] = ob;
        } else {
            const int wbase = (i * S >> 1) + sw + roff(cy(i), cz(i));
            if (cx(i) == 0) {
                if (liveA && liveB)
                    ((unsigned *)f)[wbase] = wv[i];
                else if (liveA)
                    fh[2 * wbase] = oa;
                else
                    fh[2 * wbase + 1] = ob;
            } else if (cx(i) > 0) {  // nodes x+1 (high half of this word), x+2 (low half of the right word)
                if (liveA) fh[2 * wbase + 1] = oa;
                if (liveB) fh[2 * (wbase + wr)] = ob;
            } else {  // nodes x-1 (high half of the left word), x (low half of this word)
                if (liveA) fh[2 * (wbase + wl) + 1] = oa;
                if (liveB) fh[2 * wbase] = ob;
            }
        }
    }
    // walls: halfway bounce-back (Eqs. 19, 21 with q = 1/2) pushed into the
    // slot the next step reads, from the stored post-collision value
    if (z == 0 || z == L.nz - 1) {
        const int zw_in = z == 0 ? 1 : -1;  // c_z of the populations arriving from the wall
        const float *u = z == 0 ? ph.ulo : ph.uhi;
        const int ym = y == 0 ? L.ny - 1 : y - 1, yq = y == L.ny - 1 ? 0 : y + 1;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            if (!(side == 0 ? liveA : liveB)) continue;
            const int xs = x + side, ss = s + side;
            const int xm = xs == 0 ? L.nx - 1 : xs - 1, xq = xs == L.nx - 1 ? 0 : xs + 1;
#pragma unroll
            for (int k = 1; k < Q; ++k) {
                if (cz(k) == 0) continue;
                for (int pass = 0; pass < 2; ++pass) {
                    if ((pass == 0 ? 1 : -1) != cz(k) || zw_in != cz(k)) continue;
                    const float dk = side == 0 ? Pack2<T>::lo(wv[opp(k)]) : Pack2<T>::hi(wv[opp(k)]);
                    const float v = wall_push(k, dk, u);
                    int a;
                    if (ODD) {
                        a = k * S + ss;
                    } else {
                        const int xx = cx(k) > 0 ? xm : (cx(k) < 0 ? xq : xs);
                        const int yy = cy(k) > 0 ? ym : (cy(k) < 0 ? yq : y);
                        a = opp(k) * S + xx + L.nx * (yy + L.ny * (z - cz(k))) + (int)L.plane;
                    }
                    fh[a] = Pack2<T>::bits(v);
                }
            }
        }
    }
}

template <int ODD, typename T, int MODE>
static int launch_sc(lbm_s *h, const NearMap &nm, cudaStream_t st) {
    const int bx = h->L.nx >= 256 ? 256 : ((h->L.nx + 31) / 32) * 32;
    dim3 grid((h->L.nx + bx - 1) / bx, h->L.ny, h->L.nz);
    k_stream_collide<ODD, T, MODE><<<grid, bx, 0, st>>>(h->L, h->ph, (T *)h->f, h->flag, h->status, nm);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

template <int ODD, typename T, int MODE>
static int launch_sc2(lbm_s *h, const NearMap &nm, cudaStream_t st) {
    const int hx = h->L.nx / 2;
    const int bx = hx >= 128 ? 128 : ((hx + 31) / 32) * 32;
    dim3 grid((hx + bx - 1) / bx, h->L.ny, h->L.nz);
    k_stream_collide2<ODD, T, MODE><<<grid, bx, 0, st>>>(h->L, h->ph, (T *)h->f, h->flag, h->status, nm);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

template <int ODD, typename T>
static int launch_mode(lbm_s *h, int mode, const NearMap &nm, cudaStream_t st) {
    if constexpr (sizeof(T) == 2) {
        if ((h->L.nx % 2) == 0) {
            if (mode == 1) return launch_sc2<ODD, T, 1>(h, nm, st);
            return launch_sc2<ODD, T, 0>(h, nm, st);
        }
    }
    if (mode == 1) return launch_sc<ODD, T, 1>(h, nm, st);
    return launch_sc<ODD, T, 0>(h, nm, st);
}

template <typename T>
static int launch_type(lbm_s *h, int parity, int mode, const NearMap &nm, cudaStream_t st) {
    return parity ? launch_mode<1, T>(h, mode, nm, st) : launch_mode<0, T>(h, mode, nm, st);
}

int launch_stream_collide(lbm_s *h, int parity, int mode, const uint8_t *near, uint8_t tag, cudaStream_t stream) {
    cudaStream_t st = stream ? stream : h->stream;
    const NearMap nm{near, h->near_ngx, h->near_shift, tag};
    switch (h->precision) {
        case LBM_FP32: return launch_type<float>(h, parity, mode, nm, st);
        case LBM_BF16_DEV: return launch_type<__nv_bfloat16>(h, parity, mode, nm, st);
        case LBM_FP16_DEV: return launch_type<__half>(h, parity, mode, nm, st);
    }
    return LBM_ERR_ARG;
}

template <typename T>
static int launch_list_type(lbm_s *h, int parity, const int *list, const int *count, cudaStream_t st) {
    const FastDiv dngx((unsigned)h->near_ngx), dny((unsigned)h->L.ny);
    const int grid = h->sms * 4, ngx = h->near_ngx, sh = h->near_shift;
    if (parity)
        k_collide_list<1, T><<<grid, 256, 0, st>>>(h->L, h->ph, (T *)h->f, h->flag, h->status, list, count, ngx, sh,
                                                   dngx, dny);
    else
        k_collide_list<0, T><<<grid, 256, 0, st>>>(h->L, h->ph, (T *)h->f, h->flag, h->status, list, count, ngx, sh,
                                                   dngx, dny);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int launch_collide_list(lbm_s *h, int parity, const int *list, const int *count, cudaStream_t stream) {
    cudaStream_t st = stream ? stream : h->stream;
    switch (h->precision) {
        case LBM_FP32: return launch_list_type<float>(h, parity, list, count, st);
        case LBM_BF16_DEV: return launch_list_type<__nv_bfloat16>(h, parity, list, count, st);
        case LBM_FP16_DEV: return launch_list_type<__half>(h, parity, list, count, st);
    }
    return LBM_ERR_ARG;
}

template <int ODD, typename T, int TPB, int MINB>
static cudaError_t collide_batch_t(const lbm_batch_s *b, int grid, const int2 *chunks, int nchunks) {
    if (b->ctab)
        k_collide_batch_tab<ODD, T, TPB, MINB><<<grid, TPB, 0, b->stream>>>(*b->ctab, chunks, nchunks);
    else
        k_collide_batch<ODD, T, TPB, MINB><<<grid, TPB, 0, b->stream>>>(b->dinst, chunks, nchunks);
    return cudaGetLastError();
}

// Launch shapes of the batched collide: (threads per block, minimum resident
// blocks per SM), i.e. 64 or 85 registers per thread.
#define LBM_BATCH_SHAPES(X) X(128, 8) X(128, 6) X(256, 4) X(256, 3) X(512, 2) X(512, 1)

template <int ODD, typename T>
static cudaError_t collide_batch_p(const lbm_batch_s *b, int tpb, int minb, int grid, const int2 *chunks,
                                   int nchunks) {
#define LBM_CASE(t, m) \
    if (tpb == t && minb == m) return collide_batch_t<ODD, T, t, m>(b, grid, chunks, nchunks);
    LBM_BATCH_SHAPES(LBM_CASE)
#undef LBM_CASE
    return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t collide_batch_ty(const lbm_batch_s *b, int P, int tpb, int minb, int grid, const int2 *chunks,
                                    int nchunks) {
    return P ? collide_batch_p<1, T>(b, tpb, minb, grid, chunks, nchunks)
             : collide_batch_p<0, T>(b, tpb, minb, grid, chunks, nchunks);
}

int launch_collide_batch(const lbm_batch_s *b, int P, int tpb, int minb, int grid, const int2 *chunks, int nchunks) {
    if (nchunks == 0) return LBM_OK;
    cudaError_t e = cudaErrorInvalidValue;
    switch (b->precision) {
        case LBM_FP32: e = collide_batch_ty<float>(b, P, tpb, minb, grid, chunks, nchunks); break;
        case LBM_BF16_DEV: e = collide_batch_ty<__nv_bfloat16>(b, P, tpb, minb, grid, chunks, nchunks); break;
        case LBM_FP16_DEV: e = collide_batch_ty<__half>(b, P, tpb, minb, grid, chunks, nchunks); break;
    }
    if (e != cudaSuccess) cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : (e == cudaErrorInvalidValue ? LBM_ERR_ARG : LBM_ERR_CUDA);
}

template <int ODD, typename T, int TPB, int MINB>
static cudaError_t occ_t(int *bps, bool table) {
    return table ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_collide_batch_tab<ODD, T, TPB, MINB>, TPB, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_collide_batch<ODD, T, TPB, MINB>, TPB, 0);
}

template <typename T>
static cudaError_t occ_ty(int P, int tpb, int minb, int *bps, bool table) {
#define LBM_CASE(t, m) \
    if (tpb == t && minb == m) return P ? occ_t<1, T, t, m>(bps, table) : occ_t<0, T, t, m>(bps, table);
    LBM_BATCH_SHAPES(LBM_CASE)
#undef LBM_CASE
    return cudaErrorInvalidValue;
}

int collide_batch_occupancy(int precision, int P, int tpb, int minb, int *blocks_per_sm, bool table) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (precision) {
        case LBM_FP32: e = occ_ty<float>(P, tpb, minb, blocks_per_sm, table); break;
        case LBM_BF16_DEV: e = occ_ty<__nv_bfloat16>(P, tpb, minb, blocks_per_sm, table); break;
        case LBM_FP16_DEV: e = occ_ty<__half>(P, tpb, minb, blocks_per_sm, table); break;
    }
    if (e != cudaSuccess) cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

}  // namespace lbm
