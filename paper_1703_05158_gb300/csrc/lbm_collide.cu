// Fused collide-and-stream kernels (Sect. 2.2) on the one-array A-A layout:
// the plain step, the far / near split of the overlapped schedule and the
// batched form.  The per-node bodies are in lbm_stream.cuh.
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
#include "lbm_stream.cuh"

namespace lbm {

// Every fluid node, one thread each, one block per row segment.  Resident
// blocks per SM: the even parity fits 48 registers without spills and at 5
// blocks keeps more loads in flight (FP32 collide 0.435 -> 0.422 ms per
// step over both parities; 6 blocks at 40 registers spill and lose); the
// odd parity's shifted addressing needs 64 (at 48 it spills 112 bytes and
// the step's collide took 0.477 ms).
#ifndef LBM_SC_MINB_EVEN
#define LBM_SC_MINB_EVEN 5
#endif
#ifndef LBM_SC_MINB_ODD
#define LBM_SC_MINB_ODD 4
#endif
template <int ODD, typename T>
__global__ void __launch_bounds__(256, ODD ? LBM_SC_MINB_ODD : LBM_SC_MINB_EVEN) k_stream_collide(const Lat L, const Phys ph, T *__restrict__ f,
                                                        uint8_t *__restrict__ flag, int *__restrict__ status) {
    // a programmatic dependent (the link kernel) may launch once every block
    // has started; it waits for this grid's completion before its reads
    asm volatile("griddepcontrol.launch_dependents;");
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= L.nx) return;
    const int row = y + L.ny * z;
    const int n = x + L.nx * row;
    sc_node<ODD, T>(L, ph, f, flag, status, x, y, z, n, flag[n]);
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

// 16-bit storage: the same with one node pair per thread (sc_pair); the
// groups hold 2^shift nodes, 2^(shift - 1) pairs.  Requires even nx.
template <int ODD, typename T>
__global__ void __launch_bounds__(256, 4) k_collide_list2(const Lat L, const Phys ph, T *__restrict__ f,
                                                       uint8_t *__restrict__ flag, int *__restrict__ status,
                                                       const int *__restrict__ list, const int *__restrict__ count,
                                                       const int ngx, const int shift, const FastDiv dngx,
                                                       const FastDiv dny) {
    const int ps = shift - 1;  // pairs per group: 2^ps
    const int total = *count << ps;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int g = list[t >> ps];
        const int row = (int)dngx.div((unsigned)g);
        const int xp = ((g - row * ngx) << ps) | (t & ((1 << ps) - 1));
        if (2 * xp >= L.nx) continue;
        const int z = (int)dny.div((unsigned)row);
        sc_pair<ODD, T>(L, ph, f, flag, status, xp, row - z * L.ny, z);
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

// 16-bit storage: two nodes per thread (sc_pair).  Requires even nx.
template <int ODD, typename T>
__global__ void __launch_bounds__(128, 8) k_stream_collide2(const Lat L, const Phys ph, T *__restrict__ f,
                                                            uint8_t *__restrict__ flag, int *__restrict__ status) {
    asm volatile("griddepcontrol.launch_dependents;");  // as in k_stream_collide
    const int xp = blockIdx.x * blockDim.x + threadIdx.x;
    if (xp >= (L.nx >> 1)) return;
    sc_pair<ODD, T>(L, ph, f, flag, status, xp, blockIdx.y, blockIdx.z);
}

template <int ODD, typename T>
static int launch_sc(lbm_s *h, cudaStream_t st) {
    const int bx = h->L.nx >= 256 ? 256 : ((h->L.nx + 31) / 32) * 32;
    dim3 grid((h->L.nx + bx - 1) / bx, h->L.ny, h->L.nz);
    k_stream_collide<ODD, T><<<grid, bx, 0, st>>>(h->L, h->ph, (T *)h->f, h->flag, h->status);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

template <int ODD, typename T>
static int launch_sc2(lbm_s *h, cudaStream_t st) {
    const int hx = h->L.nx / 2;
    const int bx = hx >= 128 ? 128 : ((hx + 31) / 32) * 32;
    dim3 grid((hx + bx - 1) / bx, h->L.ny, h->L.nz);
    k_stream_collide2<ODD, T><<<grid, bx, 0, st>>>(h->L, h->ph, (T *)h->f, h->flag, h->status);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

template <int ODD, typename T>
static int launch_parity(lbm_s *h, cudaStream_t st) {
    if constexpr (sizeof(T) == 2) {
        if ((h->L.nx % 2) == 0) return launch_sc2<ODD, T>(h, st);
    }
    return launch_sc<ODD, T>(h, st);
}

template <typename T>
static int launch_type(lbm_s *h, int parity, cudaStream_t st) {
    return parity ? launch_parity<1, T>(h, st) : launch_parity<0, T>(h, st);
}

int launch_stream_collide(lbm_s *h, int parity, cudaStream_t stream) {
    cudaStream_t st = stream ? stream : h->stream;
    switch (h->precision) {
        case LBM_FP32: return launch_type<float>(h, parity, st);
        case LBM_BF16_DEV: return launch_type<__nv_bfloat16>(h, parity, st);
        case LBM_FP16_DEV: return launch_type<__half>(h, parity, st);
    }
    return LBM_ERR_ARG;
}

template <typename T>
static int launch_list_type(lbm_s *h, int parity, const int *list, const int *count, cudaStream_t st) {
    const FastDiv dngx((unsigned)h->near_ngx), dny((unsigned)h->L.ny);
    const int grid = h->sms * 4, ngx = h->near_ngx, sh = h->near_shift;
    if constexpr (sizeof(T) == 2) {
        if ((h->L.nx % 2) == 0 && sh >= 1) {  // node pairs
            if (parity)
                k_collide_list2<1, T><<<grid, 256, 0, st>>>(h->L, h->ph, (T *)h->f, h->flag, h->status, list, count,
                                                             ngx, sh, dngx, dny);
            else
                k_collide_list2<0, T><<<grid, 256, 0, st>>>(h->L, h->ph, (T *)h->f, h->flag, h->status, list, count,
                                                             ngx, sh, dngx, dny);
            return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
        }
    }
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
