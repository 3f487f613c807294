// The block solves of SAP(n, m), Algorithm 1 (Sec. 2.4.1), in FP32.
//
// One CTA owns one block of the decomposition and does its whole solve:
//   r_hat_e = r_e - D_eo D_oo^{-1} r_o                  (odd-even inside the block,
//   m steps of Minimal Residual on S = D_ee - D_eo D_oo^{-1} D_oe  Sec. 2.4.5)
//   e_o = D_oo^{-1} (r_o - D_oe e_e)
//   x += e on the block's sites
// where every hop that leaves the block is dropped (the block operator is D
// restricted to the block).  The blocks of one colour touch no other block of
// that colour, so all of them run in one launch with no interaction; the MR
// dot products are CTA-local reductions, so an MR step needs no grid-wide
// synchronisation.  The block's MR residual and iterate and the odd
// intermediate live in shared memory, where the hops read their neighbours;
// links and clover blocks come from block-major FP32 copies (below), so that
// the sites of one block are contiguous and the half-steps re-read them from
// L2 in whole cache lines.
//
// The residual r = b - D x each block solve starts from is kept up to date
// block by block instead of by applying D to the whole lattice before every
// launch.  After a block's solve its residual is known: the even sites carry
// the MR residual of the Schur system (r_e - D_ee e_e - D_eo e_o equals
// r_hat_e - S e_e when e_o is reconstructed as above) and the odd sites none.
// The blocks adjacent across a face are of the other colour (an even number of
// blocks along each direction, or one block spanning it), so between two
// sweeps of a colour x changes only by the other colour's correction e', and
// the block's residual changes only through the hops that cross its faces:
//   r_B <- r_B + 1/2 sum over out-of-block neighbours of (1 -+ g_mu) W e'.
// Each launch stores its blocks' even residual and its correction e; the next
// launch of the other colour adds the face hops of e in a prologue.
#include "lq_kernels.h"
#include "spin.cuh"

namespace lq {

static constexpr int SAP_THREADS = 128;   // one thread per block site of each parity

struct SapArgs {
    Geom g;
    int b[4];                 // block extents (even, dividing the lattice)
    int bvh;                  // sites of one parity in a block (<= SAP_THREADS)
    const int4 *origin;       // lattice coordinates of the first site of each block of the colour
    const float4 *U[2];       // FP32 links by parity, lattice order (face hops)
    const float4 *Ub[2];      // the same links in block-major order (block hops)
    const float4 *Ce;         // C of the even sites, block-major
    const float4 *Ci;         // C^{-1} of the odd sites, block-major
    const float4 *rin[2];     // the blocks' residual before the face update, by parity (rin[1] null: zero)
    const float4 *eface[2];   // the other colour's last correction by parity (null: none yet)
    float4 *rout_e;           // out: the blocks' even residual after the solve
    float4 *eout[2];          // out: the blocks' correction e by parity
    float4 *x[2];             // solution by parity (x += e)
    float4 *ro;               // scratch: the odd residual between the prologue and the last half-step
    int m;                    // Minimal Residual steps
};

// local coordinates of the i-th block site of parity p (lexicographic over
// the block, the same checkerboard numbering as the lattice's)
__device__ __forceinline__ void sap_local(const SapArgs &a, int i, int p, int l[4])
{
    const int bx2 = a.b[0] >> 1;
    const int row = i / bx2;
    l[1] = row % a.b[1];
    l[2] = (row / a.b[1]) % a.b[2];
    l[3] = row / (a.b[1] * a.b[2]);
    l[0] = 2 * (i - row * bx2) + ((l[1] + l[2] + l[3] + p) & 1);
}

__device__ __forceinline__ long long sap_global_cb(const Geom &g, const int G[4])
{
    return LQ_IDX((G[0] + (long long)g.L[0] * (G[1] + (long long)g.L[1] * (G[2] + (long long)g.L[2] * G[3]))) >> 1,
                  g.Vh, B_SAP_GLOBAL);
}

// Block-major order of one parity's sites: the blocks in lexicographic order
// of their block coordinates, and inside a block its sites of that parity in
// the local checkerboard numbering of sap_local.  It is a permutation of the
// lattice's checkerboard index (every block holds bvh sites of each parity),
// so a block-major copy has the same size and row stride as the original.
__device__ __forceinline__ long long sap_block_base(const SapArgs &a, const int O[4])
{
    const int n0 = a.g.L[0] / a.b[0], n1 = a.g.L[1] / a.b[1], n2 = a.g.L[2] / a.b[2];
    const long long blk =
        O[0] / a.b[0] + (long long)n0 * (O[1] / a.b[1] + (long long)n1 * (O[2] / a.b[2] + (long long)n2 * (O[3] / a.b[3])));
    return blk * a.bvh;
}

__device__ __forceinline__ void ld_sm(const float2 *f, int i, cx<float> v[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) {
        const float2 t = f[c * SAP_THREADS + i];
        v[c] = {t.x, t.y};
    }
}

__device__ __forceinline__ void st_sm(float2 *f, int i, const cx<float> v[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) f[c * SAP_THREADS + i] = make_float2(v[c].re, v[c].im);
}

// one direction of the block-local hopping sum at the site with local
// coordinates l (parity p, global coordinates G, block-major index base + i):
// the neighbour is read from the shared-memory field `src` of the other parity
// when it lies in the block
template <int MU>
__device__ __forceinline__ void sap_hop_dir(const SapArgs &a, const float2 *src, const int l[4], const int G[4],
                                            int p, long long base, int i, cx<float> acc[12])
{
    const int ext = a.b[MU], L = a.g.L[MU];
    const bool whole = ext == L;   // the block spans the direction: the wrap stays inside
#pragma unroll
    for (int dir = 0; dir < 2; dir++) {
        const int ln = dir == 0 ? l[MU] + 1 : l[MU] - 1;
        const bool in = whole || (ln >= 0 && ln < ext);
        if (!in) continue;
        int q[4] = {l[0], l[1], l[2], l[3]};
        q[MU] = (ln + ext) % ext;
        const int nbi = (int)LQ_IDX((q[0] + a.b[0] * (q[1] + a.b[1] * (q[2] + a.b[2] * q[3]))) >> 1, a.bvh,
                                    B_SAP_LOCAL);
        cx<float> psi[12];
        ld_sm(src, nbi, psi);
        cx<float> m[9];
        float s = 1.0f;
        if (dir == 0) {
            load_link(a.Ub[p], a.g.stride, MU, LQ_IDX(base + i, a.g.Vh, B_SAP_GLOBAL), m);
            if (MU == 3 && G[3] + 1 == L) s = (float)a.g.tbc;
            hop_apply<MU, -1>(acc, psi, m, s);
        } else {   // the link of the neighbour at -mu, which lies in the block
            load_link(a.Ub[1 - p], a.g.stride, MU, LQ_IDX(base + nbi, a.g.Vh, B_SAP_GLOBAL), m);
            if (MU == 3 && G[3] == 0) s = (float)a.g.tbc;
            hop_apply<MU, +1>(acc, psi, m, s);
        }
    }
}

// acc = sum over the in-block neighbours of (1 -+ g_mu) W psi
__device__ __forceinline__ void sap_hop(const SapArgs &a, const float2 *src, const int l[4], const int G[4], int p,
                                        long long base, int i, cx<float> acc[12])
{
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = {0.0f, 0.0f};
    sap_hop_dir<0>(a, src, l, G, p, base, i, acc);
    sap_hop_dir<1>(a, src, l, G, p, base, i, acc);
    sap_hop_dir<2>(a, src, l, G, p, base, i, acc);
    sap_hop_dir<3>(a, src, l, G, p, base, i, acc);
}

// The hops across the two faces of the block normal to MU: for every site on
// a face, 1/2 (1 -+ g_mu) W e' of its neighbour outside the block is added to
// the site's residual in shared memory (smE even, smO odd).  The work items
// are the face sites, one per thread, so no lane idles on a direction its
// site does not need; a site lies on at most one of the two faces, so the
// items of one call touch distinct sites.
template <int MU>
__device__ __forceinline__ void sap_face(const SapArgs &a, const int O[4], float2 *smE, float2 *smO)
{
    const int ext = a.b[MU], L = a.g.L[MU];
    if (ext == L) return;              // the block spans the direction: no face
    const int nf = 2 * a.bvh / ext;    // sites on one face
    for (int w = threadIdx.x; w < 2 * nf; w += SAP_THREADS) {
        const int side = w >= nf;      // 0: the face at l_mu = ext - 1 (hop to +mu), 1: at l_mu = 0
        int f = w - side * nf;
        int l[4];
#pragma unroll
        for (int nu = 0; nu < 4; nu++) {
            if (nu == MU) {
                l[nu] = side ? 0 : ext - 1;
            } else {
                l[nu] = f % a.b[nu];
                f /= a.b[nu];
            }
        }
        const int G[4] = {O[0] + l[0], O[1] + l[1], O[2] + l[2], O[3] + l[3]};
        const int p = (l[0] + l[1] + l[2] + l[3]) & 1;   // block origins have even coordinates
        int Gn[4] = {G[0], G[1], G[2], G[3]};
        Gn[MU] = side ? (G[MU] == 0 ? L - 1 : G[MU] - 1) : (G[MU] + 1 == L ? 0 : G[MU] + 1);
        const long long ncb = sap_global_cb(a.g, Gn);
        cx<float> psi[12], m[9], acc[12];
        load_spinor(a.eface[1 - p], a.g.stride, ncb, psi);
#pragma unroll
        for (int k = 0; k < 12; k++) acc[k] = {0.0f, 0.0f};
        if (!side) {
            load_link(a.U[p], a.g.stride, MU, sap_global_cb(a.g, G), m);
            hop_apply<MU, -1>(acc, psi, m, (MU == 3 && G[3] + 1 == L) ? (float)a.g.tbc : 1.0f);
        } else {
            load_link(a.U[1 - p], a.g.stride, MU, ncb, m);
            hop_apply<MU, +1>(acc, psi, m, (MU == 3 && G[3] == 0) ? (float)a.g.tbc : 1.0f);
        }
        float2 *dst = p ? smO : smE;
        const int ii = (int)LQ_IDX((l[0] + a.b[0] * (l[1] + a.b[1] * (l[2] + a.b[2] * l[3]))) >> 1, a.bvh,
                                   B_SAP_LOCAL);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            float2 t = dst[c * SAP_THREADS + ii];
            t.x += 0.5f * acc[c].re;
            t.y += 0.5f * acc[c].im;
            dst[c * SAP_THREADS + ii] = t;
        }
    }
}

// sum over the CTA of three floats (all threads receive the totals)
__device__ __forceinline__ void sap_sum3(float v[3], float *sh)
{
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 3; k++) sh[warp * 3 + k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 3; k++) {
        float t = 0.0f;
        for (int w = 0; w < SAP_THREADS / 32; w++) t += sh[w * 3 + k];
        v[k] = t;
    }
}

#ifndef LQ_SAP_MINB
#define LQ_SAP_MINB 4
#endif

// The CTA asks for four resident blocks per SM (at most 128 registers, no spills); the
// MR iterate and residual live in shared memory, not in registers.  The solve
// is one loop over half-steps, each one hop into one parity followed by its
// epilogue, so that a single copy of the hop code serves all of them (the
// instruction cache holds it):
//   (face) the block's residual rin plus the face hops of e', staged in smE / smO
//   0      odd:  D_oo^{-1} r_o                               (no hop; r_o kept in ro)
//   1      even: r_hat = r_e + 1/2 H_eo (D_oo^{-1} r_o); e = 0
//   2j+2   odd:  t = D_oo^{-1} (-1/2 H_oe res)                     (MR step j)
//   2j+3   even: p = C res + 1/2 H_eo t; alpha; e += alpha res; res -= alpha p
//   2m+2   odd:  e_o = D_oo^{-1} (r_o + 1/2 H_oe e_e); x += e; store e and res
__global__ void __launch_bounds__(SAP_THREADS, LQ_SAP_MINB) sap_block_kernel(SapArgs a)
{
    __shared__ float2 smE[12 * SAP_THREADS];   // even: r_e, r_hat, then the MR residual
    __shared__ float2 smX[12 * SAP_THREADS];   // even: the MR iterate e_e
    __shared__ float2 smO[12 * SAP_THREADS];   // odd: D_oo^{-1} r_o, then t_o
    __shared__ float red[3 * (SAP_THREADS / 32)];
    const int i = threadIdx.x;
    const bool on = i < a.bvh;
    const int4 o4 = a.origin[blockIdx.x];
    const int O[4] = {o4.x, o4.y, o4.z, o4.w};
    int le[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0};
    if (on) {
        sap_local(a, i, 0, le);
        sap_local(a, i, 1, lo);
    }
    const long long st = a.g.stride;
    const long long base = sap_block_base(a, O);
    const long long sb = on ? LQ_IDX(base + i, a.g.Vh, B_SAP_GLOBAL) : 0;   // block-major index of the thread's sites
    const int last = 2 * a.m + 2;
    const bool face = a.eface[0] != nullptr;
    if (face) {
        if (on) {
            int G[4];
            cx<float> v[12];
#pragma unroll
            for (int mu = 0; mu < 4; mu++) G[mu] = O[mu] + le[mu];
            load_spinor_rw(a.rin[0], st, sap_global_cb(a.g, G), v);
            st_sm(smE, i, v);
#pragma unroll
            for (int mu = 0; mu < 4; mu++) G[mu] = O[mu] + lo[mu];
            if (a.rin[1]) load_spinor_rw(a.rin[1], st, sap_global_cb(a.g, G), v);
            else
#pragma unroll
                for (int k = 0; k < 12; k++) v[k] = {0.0f, 0.0f};
            st_sm(smO, i, v);
        }
        __syncthreads();
        sap_face<0>(a, O, smE, smO);
        __syncthreads();
        sap_face<1>(a, O, smE, smO);
        __syncthreads();
        sap_face<2>(a, O, smE, smO);
        __syncthreads();
        sap_face<3>(a, O, smE, smO);
        __syncthreads();
    }
#pragma unroll 1
    for (int ph = 0; ph <= last; ph++) {
        const int p = (ph == 1 || (ph > 1 && ph < last && (ph & 1))) ? 0 : 1;   // output parity
        int l[4], G[4];
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            l[mu] = p ? lo[mu] : le[mu];
            G[mu] = O[mu] + l[mu];
        }
        const long long cb = on ? sap_global_cb(a.g, G) : 0;
        cx<float> w[12];
        if (on && ph > 0) sap_hop(a, p ? (ph == last ? smX : smE) : smO, l, G, p, base, i, w);
        float d[3] = {0.0f, 0.0f, 0.0f};
        cx<float> pv[12];
        if (on) {
            cx<float> v[12];
            if (ph == 0) {   // r_o, kept for the last half-step
                if (face) ld_sm(smO, i, v);
                else load_spinor_rw(a.rin[1], st, cb, v);
                store_spinor(a.ro, st, cb, v);
            }
            if (p == 1) {   // odd output: D_oo^{-1} (...)
                if (ph == last) {
                    load_spinor_rw(a.ro, st, cb, v);
#pragma unroll
                    for (int k = 0; k < 12; k++) v[k] = v[k] + 0.5f * w[k];
                } else if (ph > 0) {
#pragma unroll
                    for (int k = 0; k < 12; k++) v[k] = -0.5f * w[k];
                }
                clover_apply<float>(a.Ci, st, sb, v, pv);
                if (ph < last) {
                    st_sm(smO, i, pv);
                } else {   // x += e on both parities of the site pair; store e and the residual
                    store_spinor(a.eout[1], st, cb, pv);
                    load_spinor_rw(a.x[1], st, cb, v);
#pragma unroll
                    for (int k = 0; k < 12; k++) v[k] = v[k] + pv[k];
                    store_spinor(a.x[1], st, cb, v);
                    int Ge[4];
#pragma unroll
                    for (int mu = 0; mu < 4; mu++) Ge[mu] = O[mu] + le[mu];
                    const long long cbe = sap_global_cb(a.g, Ge);
                    ld_sm(smE, i, v);
                    store_spinor(a.rout_e, st, cbe, v);
                    ld_sm(smX, i, pv);
                    store_spinor(a.eout[0], st, cbe, pv);
                    load_spinor_rw(a.x[0], st, cbe, v);
#pragma unroll
                    for (int k = 0; k < 12; k++) v[k] = v[k] + pv[k];
                    store_spinor(a.x[0], st, cbe, v);
                }
            } else if (ph == 1) {   // r_hat = r_e + 1/2 H_eo (D_oo^{-1} r_o), e = 0
                if (face) ld_sm(smE, i, v);   // r_e from the prologue
                else load_spinor_rw(a.rin[0], st, cb, v);
#pragma unroll
                for (int k = 0; k < 12; k++) v[k] = v[k] + 0.5f * w[k];
                st_sm(smE, i, v);
#pragma unroll
                for (int k = 0; k < 12; k++) v[k] = {0.0f, 0.0f};
                st_sm(smX, i, v);
            } else if (ph > 1) {   // p = C res + 1/2 H_eo t and the dot products
                ld_sm(smE, i, v);
                clover_apply<float>(a.Ce, st, sb, v, pv);
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    pv[k] = pv[k] + 0.5f * w[k];
                    d[0] = fmaf(pv[k].re, v[k].re, fmaf(pv[k].im, v[k].im, d[0]));    // Re (p, res)
                    d[1] = fmaf(pv[k].re, v[k].im, fmaf(-pv[k].im, v[k].re, d[1]));   // Im (p, res)
                    d[2] = fmaf(pv[k].re, pv[k].re, fmaf(pv[k].im, pv[k].im, d[2]));  // (p, p)
                }
            }
        }
        if (p == 0 && ph > 1) {   // the MR update after an even half-step
            sap_sum3(d, red);
            const float ar = d[2] > 0.0f ? d[0] / d[2] : 0.0f, ai = d[2] > 0.0f ? d[1] / d[2] : 0.0f;
            if (on) {
                cx<float> v[12], e[12];
                ld_sm(smE, i, v);
                ld_sm(smX, i, e);
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    e[k] = e[k] + cx<float>{ar * v[k].re - ai * v[k].im, ar * v[k].im + ai * v[k].re};
                    v[k] = v[k] - cx<float>{ar * pv[k].re - ai * pv[k].im, ar * pv[k].im + ai * pv[k].re};
                }
                st_sm(smE, i, v);
                st_sm(smX, i, e);
            }
        }
        __syncthreads();
    }
}

void sap_blocks(const Exec &e, const SapLaunch &s)
{
    if (s.count <= 0) return;
    SapArgs a;
    a.g = e.g;
    for (int mu = 0; mu < 4; mu++) a.b[mu] = s.b[mu];
    a.bvh = s.b[0] * s.b[1] * s.b[2] * s.b[3] / 2;
    a.origin = s.origin;
    for (int q = 0; q < 2; q++) {
        a.U[q] = (const float4 *)s.U[q];
        a.Ub[q] = (const float4 *)s.Ub[q];
        a.rin[q] = (const float4 *)s.rin[q];
        a.eface[q] = (const float4 *)s.eface[q];
        a.eout[q] = (float4 *)s.eout[q];
        a.x[q] = (float4 *)s.x[q];
    }
    a.Ce = (const float4 *)s.Ce;
    a.Ci = (const float4 *)s.Ci;
    a.rout_e = (float4 *)s.rout_e;
    a.ro = (float4 *)s.ro;
    a.m = s.m;
    // per block site pair: the stored residual in, links and clover once per
    // hop sweep from L1/L2, x read and written, e and the even residual
    // written; per MR step two block hops, plus the face hops (about a quarter
    // of a hop per site on 4^4 blocks, counted as such for the flops)
    const double sites = (double)s.count * a.bvh;
    const bool face = s.eface[0] != nullptr;
    Launch L_(e, K_SAP, sites * (2 * 96 + 2 * 192 + 3 * 96 + 8 * 48 + 2 * 288 + (face ? 2 * 96 : 0)),
              sites * ((2 * s.m + 2 + (face ? 0.5 : 0.0)) * (1320 + 552) + s.m * 100));
    sap_block_kernel<<<s.count, SAP_THREADS, 0, e.st>>>(a);
}

// dst[r][d] = src[r][s(d)] for the `rows` float4 rows of a parity-p FP32 field
// (row stride g.stride), d running over the block-major order of the blocks
// with extents b and s(d) the lattice checkerboard index of the same site.
// Writes are coalesced; a read touches the b0/2 consecutive sites of one
// block row.
__global__ void __launch_bounds__(256) sap_block_major_kernel(Geom g, int4 b, int bvh, int parity, int rows,
                                                              const float4 *__restrict__ src, float4 *__restrict__ dst)
{
    const long long d = blockIdx.x * 256LL + threadIdx.x;
    if (d >= g.Vh) return;
    const long long blk = d / bvh;
    const int i = (int)(d - blk * bvh);
    const int n0 = g.L[0] / b.x, n1 = g.L[1] / b.y, n2 = g.L[2] / b.z;
    const int B[4] = {(int)(blk % n0), (int)((blk / n0) % n1), (int)((blk / ((long long)n0 * n1)) % n2),
                      (int)(blk / ((long long)n0 * n1 * n2))};
    const int bx2 = b.x >> 1;
    const int row = i / bx2;
    int l[4];
    l[1] = row % b.y;
    l[2] = (row / b.y) % b.z;
    l[3] = row / (b.y * b.z);
    l[0] = 2 * (i - row * bx2) + ((l[1] + l[2] + l[3] + parity) & 1);
    const int G[4] = {B[0] * b.x + l[0], B[1] * b.y + l[1], B[2] * b.z + l[2], B[3] * b.w + l[3]};
    const long long s = LQ_IDX((G[0] + (long long)g.L[0] * (G[1] + (long long)g.L[1] * (G[2] + (long long)g.L[2] * G[3]))) >> 1,
                               g.Vh, B_SAP_GLOBAL);
    for (int r = 0; r < rows; r++) dst[r * g.stride + d] = src[r * g.stride + s];
}

void sap_block_major(const Exec &e, const int b[4], int parity, int rows, const void *src, void *dst)
{
    const Geom &g = e.g;
    if (g.Vh == 0) return;
    Launch L_(e, K_LAYOUT, (double)g.Vh * rows * 32);
    const int bvh = b[0] * b[1] * b[2] * b[3] / 2;
    sap_block_major_kernel<<<(unsigned)((g.Vh + 255) / 256), 256, 0, e.st>>>(
        g, make_int4(b[0], b[1], b[2], b[3]), bvh, parity, rows, (const float4 *)src, (float4 *)dst);
}

}  // namespace lq
