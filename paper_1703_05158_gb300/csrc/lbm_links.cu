// Link kernels (Sect. 2.3): one CTA per sphere, run after the collide
// kernel of a step; the per-sphere body is in lbm_links.cuh.
#include <cmath>

#include "lbm_links.cuh"

namespace lbm {

// GI: compiled with the Galilean-invariant momentum exchange (taken where
// the handle asks for it).
// The link kernel waits on scattered DRAM accesses: five resident CTAs per
// SM (48 registers, a few bytes of spills) with two links per thread in
// flight keep more of them outstanding than four CTAs at 64 registers with
// three (0.114 against 0.117 ms per launch on 2000 spheres; six CTAs at 40
// registers spill more and lose).  A thread's links, and so the sums, are
// in the same order for any batch.
#ifndef LBM_LINK_MINB
#define LBM_LINK_MINB 5  // resident CTAs per SM the register budget is set for
#endif
#ifndef LBM_LINK_BATCH
#define LBM_LINK_BATCH 2  // links per thread whose populations are loaded together
#endif

template <typename T, bool GI>
__global__ void __launch_bounds__(256, LBM_LINK_MINB) k_links(const Lat L, const Parts pt, const SFrame *__restrict__ fcur,
                                               T *__restrict__ f,
                                               uint8_t *__restrict__ flag, const int32_t *__restrict__ owner,
                                               const int P, const int ext, const int cap, int *__restrict__ status,
                                               unsigned long long *__restrict__ ctr) {
    links_body<T, GI, LBM_LINK_BATCH>(L, pt, fcur, f, flag, owner, P, ext, cap, status, ctr, blockIdx.x);
}

// Batched: instance blockIdx.y; parity P is also the step parity.
// The batched form (its instance read through a pointer takes more
// registers): 4 CTAs per SM at 64 registers with two links in flight took
// the 64-member sweep from 3.846 to 3.407 ms per step against 3 CTAs at 80
// registers with six (3.482 with three links at 4 CTAs, 3.435 at 5 CTAs
// and 48 registers, which spill 136 bytes).
#ifndef LBM_LINK_B_MINB
#define LBM_LINK_B_MINB 4
#endif
#ifndef LBM_LINK_B_BATCH
#define LBM_LINK_B_BATCH 2
#endif
template <typename T, bool GI>
__global__ void __launch_bounds__(256, LBM_LINK_B_MINB) k_links_b(const Inst *__restrict__ I, const int P,
                                                                  const int ext, const int cap) {
    const Inst &a = I[blockIdx.y];
    if ((int)blockIdx.x >= a.pt.np) return;
    links_body<T, GI, LBM_LINK_B_BATCH>(a.L, a.pt, a.pt.frame[P], (T *)a.f, a.flag, a.owner, P, ext, cap, a.status,
                                        a.ctr, blockIdx.x);
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
static void links_launch(lbm_s *h, int parity, size_t smem, const SFrame *fcur, int ext, int cap, bool pdl) {
    if (!pdl) {
        k_links<T, GI><<<h->pt.np, 256, smem, h->stream>>>(h->L, h->pt, fcur, (T *)h->f, h->flag, h->owner, parity,
                                                           ext, cap, h->status, h->ctr);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(h->pt.np);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = h->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_links<T, GI>, h->L, h->pt, fcur, (T *)h->f, (uint8_t *)h->flag,
                       (const int32_t *)h->owner, parity, ext, cap, h->status, h->ctr);
}

template <typename T>
static void links_launch_t(lbm_s *h, int parity, size_t smem, const SFrame *fcur, int ext, int cap, bool pdl) {
    if (h->pt.gimea) links_launch<T, true>(h, parity, smem, fcur, ext, cap, pdl);
    else links_launch<T, false>(h, parity, smem, fcur, ext, cap, pdl);
}

int launch_links(lbm_s *h, int parity, bool after_collide) {
    const int ext = h->tile_ext, cap = h->link_cap;
    const size_t smem = link_smem(ext, cap);
    const SFrame *fcur = h->pt.frame[h->steps & 1];
    const bool pdl = after_collide;
    switch (h->precision) {
        case LBM_FP32: links_launch_t<float>(h, parity, smem, fcur, ext, cap, pdl); break;
        case LBM_BF16_DEV: links_launch_t<__nv_bfloat16>(h, parity, smem, fcur, ext, cap, pdl); break;
        case LBM_FP16_DEV: links_launch_t<__half>(h, parity, smem, fcur, ext, cap, pdl); break;
        default: return LBM_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int links_setup_batch(int ext, int cap) { return links_setup(ext, cap); }

// A batch with any member on the Galilean-invariant exchange takes the GI
// kernels; each instance still follows its own setting.
template <typename T>
static void links_launch_batch(const lbm_batch_s *b, int P, size_t smem, int ext, int cap) {
    bool gi = false;
    for (int i = 0; i < b->n; ++i) gi = gi || b->m[i]->pt.gimea != 0;
    const dim3 grid(b->max_np, b->n);
    if (gi) k_links_b<T, true><<<grid, 256, smem, b->stream>>>(b->dinst, P, ext, cap);
    else k_links_b<T, false><<<grid, 256, smem, b->stream>>>(b->dinst, P, ext, cap);
}

int launch_links_batch(const lbm_batch_s *b, int P) {
    if (b->max_np == 0) return LBM_OK;
    const int ext = b->ext, cap = b->cap;
    const size_t smem = link_smem(ext, cap);
    switch (b->precision) {
        case LBM_FP32: links_launch_batch<float>(b, P, smem, ext, cap); break;
        case LBM_BF16_DEV: links_launch_batch<__nv_bfloat16>(b, P, smem, ext, cap); break;
        case LBM_FP16_DEV: links_launch_batch<__half>(b, P, smem, ext, cap); break;
        default: return LBM_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

}  // namespace lbm
