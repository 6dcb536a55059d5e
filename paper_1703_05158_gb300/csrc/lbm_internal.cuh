// Internal declarations of the GB300 LBM-DEM library (not part of the ABI).
//
// Lattice: D3Q19 in the direction order of Table 1 (Sect. 2.2); weights from
// the text under Eq. (9).  Populations are stored as deviations d_i = f_i - w_i
// from the rest equilibrium (so a fluid at rest is all zeros and the moment
// sums lose no precision), one array per direction (SoA), x fastest, with one
// ghost plane below z = 0 and one above z = nz-1 for the wall bounce-back.
//
// Streaming uses the one-array A-A pattern (Bailey et al. 2009):
//   even step: node x reads its 19 slots i, collides, writes f^c_i into slot
//              opp(i) of the same node;
//   odd step:  node x reads slot opp(i) of x - c_i (= f^c_i of the neighbour),
//              collides, writes f^c_i into slot i of x + c_i.
// in_slot / post_slot below give, for each parity, where the pre-collision
// population f_k(x) of the next step is read and where the post-collision
// f^c_i(x) of a finished step sits.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbm.h"

namespace lbm {

constexpr int Q = 19;

// Table 1, direction i = 0..18.
__host__ __device__ constexpr int cx(int i) {
    constexpr int t[Q] = {0, -1, 0, 0, -1, -1, -1, -1, 0, 0, 1, 0, 0, 1, 1, 1, 1, 0, 0};
    return t[i];
}
__host__ __device__ constexpr int cy(int i) {
    constexpr int t[Q] = {0, 0, -1, 0, -1, 1, 0, 0, -1, -1, 0, 1, 0, 1, -1, 0, 0, 1, 1};
    return t[i];
}
__host__ __device__ constexpr int cz(int i) {
    constexpr int t[Q] = {0, 0, 0, -1, 0, 0, -1, 1, -1, 1, 0, 0, 1, 0, 0, 1, -1, 1, -1};
    return t[i];
}
// Opposite direction: in Table 1 the pairs are (i, i+9) for i = 1..9.
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 9 ? i + 9 : i - 9); }
// 36 w_i: 12 at rest, 2 on the axes, 1 on the diagonals.
__host__ __device__ constexpr int w36(int i) { return i == 0 ? 12 : (cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i) == 1 ? 2 : 1); }
__host__ __device__ constexpr float wf(int i) { return (float)w36(i) / 36.0f; }

// Runtime-indexed velocity components without memory: each table packed two
// bits per direction into a 64-bit constant.
__host__ __device__ constexpr unsigned long long pack_axis(int axis) {
    unsigned long long r = 0;
    for (int i = 0; i < Q; ++i)
        r |= (unsigned long long)((axis == 0 ? cx(i) : (axis == 1 ? cy(i) : cz(i))) + 1) << (2 * i);
    return r;
}
__device__ __forceinline__ int rcx(int i) { return (int)((pack_axis(0) >> (2 * i)) & 3ull) - 1; }
__device__ __forceinline__ int rcy(int i) { return (int)((pack_axis(1) >> (2 * i)) & 3ull) - 1; }
__device__ __forceinline__ int rcz(int i) { return (int)((pack_axis(2) >> (2 * i)) & 3ull) - 1; }
__device__ __forceinline__ int ropp(int i) { return i == 0 ? 0 : (i <= 9 ? i + 9 : i - 9); }
__device__ __forceinline__ int rw36(int i) {
    return i == 0 ? 12 : (rcx(i) * rcx(i) + rcy(i) * rcy(i) + rcz(i) * rcz(i) == 1 ? 2 : 1);
}

// Flag value of the solid nodes marked by a step of step parity sp (1 or
// 3, bit 0 set); the other value marks the previous step's geometry.
__host__ __device__ constexpr uint8_t mark_value(int sp) { return (uint8_t)(1 + 2 * (sp & 1)); }

// Device status bits (sticky, OR-ed by kernels).
enum : int {
    ST_DIVERGED = 1,
    ST_NBR_OVERFLOW = 2,
    ST_TIMEOUT = 4,
    ST_FAST = 8,
    ST_TILE = 16,
};

// Population storage: FP32, or a 16-bit float holding the deviation.
template <typename T>
struct Store;
template <>
struct Store<float> {
    static __device__ __forceinline__ float ld(const float *p) { return *p; }
    static __device__ __forceinline__ float ldcg(const float *p) { return __ldcg(p); }  // through L2 only
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
    static __device__ __forceinline__ float rt(float v) { return v; }  // v as stored and read back
};
template <>
struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ float ldcg(const __nv_bfloat16 *p) {
        return __uint_as_float((unsigned)__ldcg((const unsigned short *)p) << 16);
    }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float rt(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
};
template <>
struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ float ldcg(const __half *p) {
        return __half2float(__ushort_as_half(__ldcg((const unsigned short *)p)));
    }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ float rt(float v) { return __half2float(__float2half_rn(v)); }
};

// Exact unsigned division of n < 2^31 by a fixed d >= 1 (Granlund and
// Montgomery 1994, Thm. 4.2): with l = ceil(log2 d) and
// m = ceil(2^(31+l) / d) < 2^32, floor(n / d) = (n m) >> (31 + l), since
// 0 <= m d - 2^(31+l) < d <= 2^l.
struct FastDiv {
    unsigned m;
    int sh;
    FastDiv() : m(0u), sh(0) {}
    explicit FastDiv(unsigned d) {
        int l = 0;
        while ((1ull << l) < d) ++l;
        m = (unsigned)(((1ull << (31 + l)) + d - 1) / d);
        sh = 31 + l;
    }
    __device__ __forceinline__ unsigned div(unsigned n) const {
        return (unsigned)(((unsigned long long)n * m) >> sh);
    }
};

// Lattice extents.  Storage index of node (x, y, z) is x + nx*(y + ny*(z+1)):
// plane z = -1 and plane z = nz are the wall ghosts.  Slot i starts at i*S.
struct Lat {
    int nx, ny, nz;
    long long plane;  // nx*ny
    long long N;      // nx*ny*nz (flag / owner arrays, no ghosts)
    long long S;      // slot stride in elements, >= plane*(nz+2), multiple of 64
};

// Offset of the storage index of x + (ox, oy, oz) from that of x, with x and y
// periodic; z is never wrapped (the ghost planes absorb |oz| = 1 at the walls).
struct Nbr {
    int xm, xp;            // x offsets of -1 and +1
    long long ym, yp, zp;  // y offsets of -1, +1; z offset of +1
    __device__ __forceinline__ Nbr(const Lat &L, int x, int y) {
        xm = x == 0 ? L.nx - 1 : -1;
        xp = x == L.nx - 1 ? -(L.nx - 1) : 1;
        ym = y == 0 ? (long long)L.nx * (L.ny - 1) : -(long long)L.nx;
        yp = y == L.ny - 1 ? -(long long)L.nx * (L.ny - 1) : (long long)L.nx;
        zp = L.plane;
    }
    __device__ __forceinline__ long long off(int ox, int oy, int oz) const {
        return (ox < 0 ? xm : (ox > 0 ? xp : 0)) + (oy < 0 ? ym : (oy > 0 ? yp : 0)) + (long long)oz * zp;
    }
};

// Slot (element index into the population array) holding the pre-collision
// f_k(x) that the step of parity P reads; s is the storage index of x.
__device__ __forceinline__ long long in_slot(const Lat &L, const Nbr &nb, int P, int k, long long s) {
    return P == 0 ? (long long)k * L.S + s : (long long)ropp(k) * L.S + s + nb.off(-rcx(k), -rcy(k), -rcz(k));
}
// Slot holding the post-collision f^c_i(x) written by a finished step of parity P.
__device__ __forceinline__ long long post_slot(const Lat &L, const Nbr &nb, int P, int i, long long s) {
    return P == 0 ? (long long)ropp(i) * L.S + s : (long long)i * L.S + s + nb.off(rcx(i), rcy(i), rcz(i));
}

// Fluid parameters in FP32 for the kernels.
struct Phys {
    float tau0;
    float smag;  // 18 sqrt(2) C^2 (Eq. 18 with c_s^4 = 1/9)
    float g[3];
    float ulo[3], uhi[3];
};

// FP32 frame of a sphere for the lattice kernels, written once per step by
// the DEM: integer base b = floor(X), fraction (float)(X - b), radius, and
// velocity / angular velocity in FP32.  Relative coordinates of a lattice
// point x are (float)(x - b) - fr.
struct SFrame {
    int b[3];
    float fr[3];
    float R, R2;
    float V[3], W[3];
    float pad[2];
};

// Sphere state on the device.
struct Parts {
    int np;
    double *X, *V, *W, *R;         // [np][3] x3, [np]
    const uint8_t *fixed;          // [np]
    double *Fh, *Th;               // hydrodynamic load of the last step
    double *Fc;                    // contact force at the current position
    double *Fx, *Tx;               // external load
    float4 *Xf;                    // FP32 copy of centre and radius (neighbour search)
    double *Xb[2], *Vh[2];         // DEM sub-step buffers
    int *nbr, *nbr_cnt;            // neighbour lists [np][max_nbr]
    int max_nbr;
    float4 *pairA, *pairB;         // per contact candidate: (d0, c0) and (dv0, gamma), see lbm_dem.cu
    int2 *pairBM;                  // per contact candidate: (b, list position)
    int *nact;                     // [np] contact candidates of the step
    double *Xbuild;                // centres when the lists were built
    int *rebuild;                  // [2]: rebuild[s & 1] = 1 asks the neighbour pass of step s to rebuild
    SFrame *frame[2];              // frames of the centres of even / odd steps
    double kn, ce, rho_s;          // ce = -2 ln e / sqrt(pi^2 + ln^2 e)
    int substeps;
    double skin;                   // list skin: pairs within R_a + R_b + skin are listed
    double max_step;               // largest displacement allowed in one step
    int corr;                      // 1: covered / uncovered nodes exchange momentum with the sphere
    double *Fcorr, *Tcorr;         // that exchange in the current step (marks write, refill adds)
    // tangential contact law (Eqs. 2, 3), on when fric != 0
    int fric;
    double kt, mu, ct;             // ct = -2 ln e_t / sqrt(pi^2 + ln^2 e_t) (0 for e_t = 1)
    double *Tc;                    // contact torque at the current position [np][3]
    float4 *pairC;                 // per contact candidate: (spin of b at the start of the step, gamma_t)
    float4 *tdisp;                 // per list entry: tangential displacement of the contact (xyz)
    unsigned long long *tmask;     // per sphere: bit m set = list entry m was in contact
    float4 *twall;                 // [np][2]: tangential displacement against the lower / upper wall
    float ulo[3], uhi[3];          // wall velocities
    int gimea;                     // 1: Galilean-invariant momentum exchange
};

// Makes device d current for the lifetime of the object, then restores the
// caller's device.
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int d) {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceScope() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Tag of the near set used by the collisions of step s (never 0).  Step s
// uses buffer near[s & 1]; within one buffer the tags run 1..255 and the
// buffer is cleared before its tag comes back to 1, so no stale tag matches.
inline uint8_t near_tag(long long s) { return (uint8_t)(1 + (s >> 1) % 255); }

}  // namespace lbm

struct lbm_batch_s;

// Handle (opaque in the ABI).
struct lbm_s {
    lbm_batch_s *batch;      // the batch this handle belongs to (steps only through it), or null
    cudaGraphExec_t graph[2];  // one serial step from parity 0 / 1 (null: not captured)
    bool graph_stale;          // sphere count changed since the capture
    cudaStream_t side;         // branch of the step graph that builds the neighbour lists
    cudaEvent_t ev_fork, ev_nbr;
    lbm_params p;
    lbm::Lat L;
    lbm::Phys ph;
    lbm::Parts pt;
    int device;
    cudaStream_t stream;
    bool own_stream;
    int precision;
    size_t esize;  // bytes per stored population
    void *f;       // populations
    uint8_t *flag;  // 0 fluid, 1 solid, 3 solid at the previous geometry, 2 refilled (see lbm_geometry.cu)
    int32_t *owner;
    int *status;             // device status word
    int *status_host;        // pinned mirror
    unsigned *bar;           // DEM grid-barrier counter
    unsigned long long *ctr; // [0] links, [1] refilled, [2] fluid-count scratch
    int parity;              // parity of the next step
    long long steps;
    int sticky;              // first device error seen
    int dem_blocks, dem_threads;  // cooperative fallback grid
    int dem_cluster;              // CTAs of the one-cluster DEM kernel (0: use the fallback)
    int dem_mode = 0;             // LBM_DEM_AUTO, LBM_DEM_CLUSTER or LBM_DEM_GRID
    int dem_grid_blocks = 0;      // co-resident blocks of the grid form (0: unavailable)
    float4 *xbuf = nullptr;       // grid form: [2][max_particles][3] sub-step exchange buffer
    // ZIEB face on z = 0: zs = [rho, rho, H_p, H_p, v_p] (rho and H_p ping-pong by
    // step parity), zpart / zcnt = [2][zblocks] per-block sums of u_z and node counts
    int zieb = 0, zblocks = 0;
    double zA = 0.0, zV0 = 0.0, zvp = 0.0;
    double *zs = nullptr, *zpart = nullptr;
    int *zcnt = nullptr;
    // host loads staged in pinned memory (two slots, each [2][max_particles][3]:
    // force, torque) so that lbm_set_particle_load returns without waiting for
    // the stream; load_ev[k] follows the last copy out of slot k
    double *load_stage[2] = {nullptr, nullptr};
    cudaEvent_t load_ev[2] = {nullptr, nullptr};
    int load_slot = 0;
    int tile_ext;            // half width of the per-sphere link tile
    int link_cap;            // link-list capacity per sphere (shared memory)
    size_t bytes;
    // overlap of the next step's far-node collisions with the link / DEM /
    // geometry chain (see lbm_capi.cu): near-node tags per step parity
    uint8_t *near[2];
    cudaStream_t stream2;    // far-node collisions, lowest priority
    cudaStream_t chain;      // highest priority; runs lbm_step's main-stream work when the caller's stream
                             // does not have that priority (null otherwise)
    cudaEvent_t ev_join;     // hand-over between the caller's stream and `chain`
    // Tags are kept per group of 2^near_shift consecutive nodes along x (64
    // bytes of a slot row, the DRAM access granularity): group (x >>
    // near_shift) of row y + ny z is tag entry row * near_ngx + (x >> near_shift).
    int near_shift, near_ngx;
    long long near_groups;   // rows * near_ngx
    int *near_list[2];       // near groups of step parity 0 / 1, compacted
    int *near_cnt;           // [2] their counts
    int *far_list[2];        // the other groups of step parity 0 / 1, compacted
    int *far_cnt;            // [2] their counts
    int sms;                 // multiprocessors of the device
    cudaEvent_t ev_cf;                 // after the far collisions
    bool overlap;
    cudaEvent_t ev_nm[2];              // after the near marks of step parity 0 / 1
    // phase profiler: kProfEv events per step
    cudaEvent_t *ev;
    int ev_cap, ev_used;     // capacity and used count, in steps
    bool prof;
    double prof_ms[LBM_PHASES];
    long long prof_steps;
};

namespace lbm {

// What a kernel needs of one simulation; the batched kernels read one per
// instance from a device array (instance = blockIdx.y, or from a chunk
// table for the collide).
struct Inst {
    Lat L;
    Phys ph;
    Parts pt;
    void *f;
    uint8_t *flag;
    int32_t *owner;
    int *status;
    unsigned long long *ctr;
    FastDiv dnx, dny;
};

// What the batched collide needs of one instance.  Up to kCollideTable
// instances travel as one kernel-parameter table (read through the constant
// cache, like the single-instance kernel's parameters).
struct CInst {
    Lat L;
    Phys ph;
    void *f;
    uint8_t *flag;
    int *status;
    FastDiv dnx, dny;
};
constexpr int kCollideTable = 192;
struct CollideTable {
    CInst c[kCollideTable];
};
static_assert(sizeof(CollideTable) <= 32000, "kernel parameters are limited to 32764 bytes");

}  // namespace lbm

// A batch of independent simulations stepped together (lbm_batch_*).
struct lbm_batch_s {
    int n = 0;
    lbm_s **m = nullptr;          // members (their handles)
    lbm::Inst *dinst = nullptr;   // device array [n]
    int2 *chunks = nullptr;       // collide chunk table: (instance, first node), tpb nodes each
    int nchunks = 0, chunk_tpb = 0;
    int tpb = 0, minb = 0, grid = 0;  // collide launch picked by the autotuner (0: not tuned)
    int max_np = 0;               // largest sphere count of a member
    int ext = 0, cap = 0;         // link tile half width and list capacity (largest over members)
    int dem_cluster = 0;          // CTAs per instance cluster of the DEM kernel
    bool fric = false;            // a member has tangential friction: the DEM kernel that keeps its state
    lbm::CollideTable *ctab = nullptr;  // host copy of the collide's parameter table (n <= kCollideTable)
    int precision = 0, device = 0, sms = 0;
    bool dirty = true;            // descriptors / graphs to be rebuilt
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // one step from parity 0 / 1
};

// Launchers (one per translation unit).
namespace lbm {
int launch_stream_collide(lbm_s *h, int parity, cudaStream_t stream = nullptr);
// near tags of one step into `near`, the tagged groups compacted into list / *count and the
// other groups into far / *far_count
int launch_near_mark(lbm_s *h, uint8_t *near, uint8_t tag, const SFrame *frames, int *list, int *count, int *far,
                     int *far_count, cudaStream_t stream);
int launch_collide_list(lbm_s *h, int parity, const int *list, const int *count, cudaStream_t stream);
int launch_zieb(lbm_s *h, int P);  // ZIEB face after the step of parity P
int launch_wait_probe(lbm_s *h);   // a bounded device wait that runs out (self-test)
int launch_mark(lbm_s *h, int P, int corr);  // corr: momentum correction of the covered nodes
int launch_refill(lbm_s *h, int parity);
// after_collide: launched as a programmatic dependent of the collide kernel
// just before it on the stream (its node codes and link list, which read
// only the marks, overlap the collide's last blocks; the populations are
// read after the collide grid has completed).
int launch_links(lbm_s *h, int parity, bool after_collide = false);
int launch_neighbours(lbm_s *h, int force, cudaStream_t stream = nullptr);
int launch_contact(lbm_s *h);
int launch_dem(lbm_s *h);
int launch_set_populations(lbm_s *h, const double *f_dev, int parity);
int launch_get_populations(lbm_s *h, double *f_dev, int parity);
int launch_fields(lbm_s *h, float *rho, float *u, int parity);
int launch_owner(lbm_s *h, int32_t *owner);
int launch_count_fluid(lbm_s *h);
int dem_max_blocks(int threads, int *blocks_per_sm);
int dem_cluster_setup(int max_particles, bool small = false, bool fric = false);
int dem_grid_setup(bool fric, int sms);
long long dem_grid_capacity(bool fric, int blocks);
int link_capacity(double max_radius);
size_t link_smem(int ext, int cap);
int links_setup(int ext, int cap);
int settle_handle(lbm_s *h);
// batched forms (all members at step parity sp = P)
int launch_mark_batch(const lbm_batch_s *b, int sp);
int launch_refill_batch(const lbm_batch_s *b, int P);
int launch_collide_batch(const lbm_batch_s *b, int P, int tpb, int minb, int grid, const int2 *chunks, int nchunks);
int collide_batch_occupancy(int precision, int P, int tpb, int minb, int *blocks_per_sm, bool table);
int launch_links_batch(const lbm_batch_s *b, int P);
int links_setup_batch(int ext, int cap);
int launch_neighbours_batch(const lbm_batch_s *b, int sp);
int launch_dem_batch(const lbm_batch_s *b, int sp);
int dem_cluster_setup_batch(int cl, bool fric);
}  // namespace lbm
