// Per-node (FP32) and per-node-pair (16-bit) bodies of the fused
// collide-and-stream step on the one-array A-A layout (Sect. 2.2), shared by
// the collide kernels of lbm_collide.cu.
//
// Per fluid node: read the 19 pre-collision deviations d_i = f_i - w_i, form
// rho (Eq. 5) and the force-shifted velocity (Eq. 6), the Smagorinsky
// relaxation time (Eq. 18), relax (Eq. 12) with the Guo body-force source,
// and write the 19 post-collision deviations in place (A-A, so streaming is
// implicit in the addressing of the next step).  Nodes next to the z walls
// also write the halfway bounce-back value of Eqs. (19, 21) with q = 1/2
// straight into the slot the next step reads for the population arriving
// from the wall.
#pragma once

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

// 16-bit storage, the two nodes (x, x+1) = (2 xp, 2 xp + 1) of one thread:
// each slot pair is one aligned 32-bit word.  Even steps read and write the node's own words.
// Odd steps read slot opp(i) at x - c_i: for c_x(i) = 0 that is again one
// word; for c_x(i) = +-1 the pair straddles two aligned words, of which the
// needed halves are taken; the post-collision pair goes to x + c_i, as one
// word for c_x = 0 and as two 16-bit stores otherwise.  Requires even nx.
template <int ODD, typename T>
__device__ __forceinline__ void sc_pair(const Lat &L, const Phys &ph, T *__restrict__ f, uint8_t *__restrict__ flag,
                                        int *__restrict__ status, const int xp, const int y, const int z) {
    const int hx = L.nx >> 1;  // pairs per row
    const int x = 2 * xp;
    const int n = x + L.nx * (y + L.ny * z);
    const unsigned short fl2 = *(const unsigned short *)(flag + n);
    const uint8_t fla = (uint8_t)(fl2 & 0xff), flb = (uint8_t)(fl2 >> 8);
    const bool liveA = !(fla & 1), liveB = !(flb & 1);
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
    // write: even -> slot opp(i) of the pair; odd -> slot i at (x, x+1) + c_i.
    // Both nodes fluid (the common case): whole words where the pair stays
    // aligned, no per-direction tests.
    if (liveA && liveB) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (!ODD) {
                ((unsigned *)f)[(opp(i) * S >> 1) + sw] = wv[i];
            } else {
                const int wbase = (i * S >> 1) + sw + roff(cy(i), cz(i));
                if (cx(i) == 0) {
                    ((unsigned *)f)[wbase] = wv[i];
                } else if (cx(i) > 0) {  // nodes x+1 (high half of this word), x+2 (low half of the right word)
                    fh[2 * wbase + 1] = (unsigned short)(wv[i] & 0xffffu);
                    fh[2 * (wbase + wr)] = (unsigned short)(wv[i] >> 16);
                } else {  // nodes x-1 (high half of the left word), x (low half of this word)
                    fh[2 * (wbase + wl) + 1] = (unsigned short)(wv[i] & 0xffffu);
                    fh[2 * wbase] = (unsigned short)(wv[i] >> 16);
                }
            }
        }
    } else
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


}  // namespace lbm
