// The fused hopping kernels of the odd-even Wilson-clover operator.
//
// One thread per output site of one parity.  For each of the eight
// directions the neighbour spinor is spin-projected onto a half spinor with
// (1 -+ g_mu), multiplied by the link (U_mu(x) forward, U_mu(x-mu)^+ backward)
// and reconstructed into the 12-component accumulator; the epilogue then
// applies the site-diagonal clover block (C or C^{-1}) and whatever BLAS-1
// step the mode fuses.  Together the two launches
//   K1: t_o = D_oo^{-1} D_oe x_e      (HOP_K1 on odd sites)
//   K2: y_e = D_ee x_e - D_eo t_o     (HOP_K2 on even sites)
// apply the Schur complement D_S of Eq. 3; HOP_RICH fuses the Richardson
// update x_e += omega (b_e - D_S x_e) of Algorithm 4 into K2.
// The spin projection and transport of one hop live in spin.cuh.
#include <type_traits>

#include "bf16.cuh"
#include "lq_kernels.h"
#include "spin.cuh"

namespace lq {

#define LQ_HOP_THREADS 128
static_assert(LQ_HOP_THREADS == kHopBlock, "hopping block size");
// minimum resident blocks per SM asked of the single-right-hand-side kernels.
// Unset leaves the register allocation to the compiler's default for
// 128-thread blocks, which differs from an explicit 1 (that one lets the
// kernels grow to about 160 registers).
#ifdef LQ_HOP_MINB
#define LQ_HOP_BOUNDS __launch_bounds__(LQ_HOP_THREADS, LQ_HOP_MINB)
#else
#define LQ_HOP_BOUNDS __launch_bounds__(LQ_HOP_THREADS)
#endif

// one hop: acc += (1 -+ g_mu) W psi(nb), W = U_mu(x) (SIGN -1) or U_mu(x-mu)^+ (SIGN +1);
// `bsign` is the fermion boundary factor of this hop
template <int MU, int SIGN, typename R, typename SV, typename LV>
__device__ __forceinline__ void hop_dir(cx<R> acc[12], const SV *__restrict__ psi, const LV *__restrict__ U,
                                        long long link_site, long long nb, long long stride, R bsign)
{
    cx<R> p[12];
    load_spinor(psi, stride, nb, p);
    cx<R> m[9];
    load_link(U, stride, MU, link_site, m);
    hop_apply<MU, SIGN>(acc, p, m, bsign);
}

template <typename R>
struct HopArgs {
    typedef typename St<R>::vec V;
    const V *in;
    const V *in2;
    const V *b;
    V *out;
    const V *Uout;   // links of the output parity: forward links U_mu(x)
    const V *Uin;    // links of the input parity: backward links U_mu(x - mu)
    const V *clov;
    const V *clov2;  // HOP_RECON_RES: C of the output parity
    V *out2;         // HOP_RECON_RES: the residual
    R omega;
    int pout;
    int nrhs;        // right-hand sides sharing the links and clover of this launch
    long long fs;    // distance between consecutive right-hand sides' fields, in vectors
};


// SV, LV, CV: storage vectors of the spinors, links and clover blocks (the same
// type for FP64, FP32 and df64; BF16 spinors and links with FP32 clover)
template <typename R, int MODE, typename SV, typename LV, typename CV>
__device__ __forceinline__ void hop_body(const Geom &g, const LV *Uout, const LV *Uin, const CV *clov, R omega,
                                         const SV *in, const SV *in2, const SV *bv, SV *out, long long s,
                                         const Coords &c, const CV *clov2 = nullptr, SV *out2 = nullptr)
{
    const long long st = g.stride;
    cx<R> acc[12];
#pragma unroll
    for (int i = 0; i < 12; i++) acc[i] = {R(0), R(0)};
    const R one = R(1);

    // x direction: the neighbour changes x, so its cb index is recomputed
    {
        const long long base = c.row * g.Lxh;
        const int xp = (c.x + 1 == g.L[0]) ? 0 : c.x + 1;
        const int xm = (c.x == 0) ? g.L[0] - 1 : c.x - 1;
        const long long nf = LQ_IDX(base + (xp >> 1), g.Vh, B_HOP_NB), nb = LQ_IDX(base + (xm >> 1), g.Vh, B_HOP_NB);
        hop_dir<0, -1>(acc, in, Uout, s, nf, st, one);
        hop_dir<0, +1>(acc, in, Uin, nb, nb, st, one);
    }
    // y, z, t: x is unchanged, so the cb index moves by a fixed stride
    {
        const long long d = g.Lxh;
        const long long nf = LQ_IDX((c.y + 1 == g.L[1]) ? s - (long long)(g.L[1] - 1) * d : s + d, g.Vh, B_HOP_NB);
        const long long nb = LQ_IDX((c.y == 0) ? s + (long long)(g.L[1] - 1) * d : s - d, g.Vh, B_HOP_NB);
        hop_dir<1, -1>(acc, in, Uout, s, nf, st, one);
        hop_dir<1, +1>(acc, in, Uin, nb, nb, st, one);
    }
    {
        const long long d = (long long)g.Lxh * g.L[1];
        const long long nf = LQ_IDX((c.z + 1 == g.L[2]) ? s - (long long)(g.L[2] - 1) * d : s + d, g.Vh, B_HOP_NB);
        const long long nb = LQ_IDX((c.z == 0) ? s + (long long)(g.L[2] - 1) * d : s - d, g.Vh, B_HOP_NB);
        hop_dir<2, -1>(acc, in, Uout, s, nf, st, one);
        hop_dir<2, +1>(acc, in, Uin, nb, nb, st, one);
    }
    {
        const long long d = (long long)g.Lxh * g.L[1] * g.L[2];
        const bool last = (c.t + 1 == g.L[3]), first = (c.t == 0);
        const long long nf = LQ_IDX(last ? s - (long long)(g.L[3] - 1) * d : s + d, g.Vh, B_HOP_NB);
        const long long nb = LQ_IDX(first ? s + (long long)(g.L[3] - 1) * d : s - d, g.Vh, B_HOP_NB);
        const R tb = R(g.tbc);
        hop_dir<3, -1>(acc, in, Uout, s, nf, st, last ? tb : one);
        hop_dir<3, +1>(acc, in, Uin, nb, nb, st, first ? tb : one);
    }

    cx<R> v[12];
    if (MODE == HOP_K1) {
#pragma unroll
        for (int i = 0; i < 12; i++) acc[i] = R(-0.5) * acc[i];
        clover_apply<R>(clov, st, s, acc, v);
    } else if (MODE == HOP_K2 || MODE == HOP_RICH || MODE == HOP_FULL || MODE == HOP_RES) {
        cx<R> x[12];
        load_spinor_rw(in2, st, s, x);
        clover_apply<R>(clov, st, s, x, v);
        const R f = (MODE == HOP_FULL || MODE == HOP_RES) ? R(-0.5) : R(0.5);
#pragma unroll
        for (int i = 0; i < 12; i++) v[i] = v[i] + f * acc[i];
        if (MODE == HOP_RICH) {
            cx<R> bb[12];
            load_spinor(bv, st, s, bb);
#pragma unroll
            for (int i = 0; i < 12; i++) v[i] = x[i] + omega * (bb[i] - v[i]);
        }
        if (MODE == HOP_RES) {
            cx<R> bb[12];
            load_spinor(bv, st, s, bb);
#pragma unroll
            for (int i = 0; i < 12; i++) v[i] = bb[i] - v[i];
        }
    } else {   // HOP_PREP, HOP_RECON, HOP_RECON_RES
        cx<R> y[12];
        load_spinor_rw(in2, st, s, y);
#pragma unroll
        for (int i = 0; i < 12; i++) y[i] = y[i] + R(0.5) * acc[i];
        if (MODE == HOP_RECON || MODE == HOP_RECON_RES) {
            clover_apply<R>(clov, st, s, y, v);
            if (MODE == HOP_RECON_RES) {   // the parity's residual u - C x_o of the x_o just formed
                cx<R> w[12];
                clover_apply<R>(clov2, st, s, v, w);
#pragma unroll
                for (int i = 0; i < 12; i++) w[i] = y[i] - w[i];
                store_spinor(out2, st, s, w);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 12; i++) v[i] = y[i];
        }
    }
    store_spinor(out, st, s, v);
}

// One thread per output site.  The batched form (MULTI) loops over the
// right-hand sides, so each site's links and clover block come from DRAM once
// and from the caches for the other right-hand sides; it is a separate
// instantiation so that the single right-hand-side kernel keeps its registers.
// Two right-hand sides per thread (K1 and K2 of the batched hop): each link is
// loaded once and transports both neighbour spinors.
template <int MU, int SIGN>
__device__ __forceinline__ void hop_dir2(cx<float> acc0[12], cx<float> acc1[12], const float4 *__restrict__ psi0,
                                         const float4 *__restrict__ psi1, const float4 *__restrict__ U,
                                         long long link_site, long long nb, long long stride, float bsign)
{
    cx<float> m[9];
    load_link(U, stride, MU, link_site, m);
    cx<float> p[12];
    load_spinor(psi0, stride, nb, p);
    hop_apply<MU, SIGN>(acc0, p, m, bsign);
    load_spinor(psi1, stride, nb, p);
    hop_apply<MU, SIGN>(acc1, p, m, bsign);
}

template <int MODE>
__device__ __forceinline__ void hop_body2(const Geom &g, const float4 *Uout, const float4 *Uin, const float4 *clov,
                                          const float4 *in0, const float4 *in1, const float4 *in20,
                                          const float4 *in21, float4 *out0, float4 *out1, bool two, long long s,
                                          const Coords &c)
{
    const long long st = g.stride;
    cx<float> a0[12], a1[12];
#pragma unroll
    for (int i = 0; i < 12; i++) a0[i] = a1[i] = {0.0f, 0.0f};
    {
        const long long base = c.row * g.Lxh;
        const int xp = (c.x + 1 == g.L[0]) ? 0 : c.x + 1;
        const int xm = (c.x == 0) ? g.L[0] - 1 : c.x - 1;
        const long long nf = LQ_IDX(base + (xp >> 1), g.Vh, B_HOP_NB), nb = LQ_IDX(base + (xm >> 1), g.Vh, B_HOP_NB);
        hop_dir2<0, -1>(a0, a1, in0, in1, Uout, s, nf, st, 1.0f);
        hop_dir2<0, +1>(a0, a1, in0, in1, Uin, nb, nb, st, 1.0f);
    }
    {
        const long long d = g.Lxh;
        const long long nf = LQ_IDX((c.y + 1 == g.L[1]) ? s - (long long)(g.L[1] - 1) * d : s + d, g.Vh, B_HOP_NB);
        const long long nb = LQ_IDX((c.y == 0) ? s + (long long)(g.L[1] - 1) * d : s - d, g.Vh, B_HOP_NB);
        hop_dir2<1, -1>(a0, a1, in0, in1, Uout, s, nf, st, 1.0f);
        hop_dir2<1, +1>(a0, a1, in0, in1, Uin, nb, nb, st, 1.0f);
    }
    {
        const long long d = (long long)g.Lxh * g.L[1];
        const long long nf = LQ_IDX((c.z + 1 == g.L[2]) ? s - (long long)(g.L[2] - 1) * d : s + d, g.Vh, B_HOP_NB);
        const long long nb = LQ_IDX((c.z == 0) ? s + (long long)(g.L[2] - 1) * d : s - d, g.Vh, B_HOP_NB);
        hop_dir2<2, -1>(a0, a1, in0, in1, Uout, s, nf, st, 1.0f);
        hop_dir2<2, +1>(a0, a1, in0, in1, Uin, nb, nb, st, 1.0f);
    }
    {
        const long long d = (long long)g.Lxh * g.L[1] * g.L[2];
        const bool last = (c.t + 1 == g.L[3]), first = (c.t == 0);
        const long long nf = LQ_IDX(last ? s - (long long)(g.L[3] - 1) * d : s + d, g.Vh, B_HOP_NB);
        const long long nb = LQ_IDX(first ? s + (long long)(g.L[3] - 1) * d : s - d, g.Vh, B_HOP_NB);
        const float tb = (float)g.tbc;
        hop_dir2<3, -1>(a0, a1, in0, in1, Uout, s, nf, st, last ? tb : 1.0f);
        hop_dir2<3, +1>(a0, a1, in0, in1, Uin, nb, nb, st, first ? tb : 1.0f);
    }
    cx<float> v[12], x[12];
    if (MODE == HOP_K1) {
#pragma unroll
        for (int i = 0; i < 12; i++) a0[i] = -0.5f * a0[i];
        clover_apply<float>(clov, st, s, a0, v);
        store_spinor(out0, st, s, v);
        if (two) {
#pragma unroll
            for (int i = 0; i < 12; i++) a1[i] = -0.5f * a1[i];
            clover_apply<float>(clov, st, s, a1, v);
            store_spinor(out1, st, s, v);
        }
    } else {   // HOP_K2
        load_spinor_rw(in20, st, s, x);
        clover_apply<float>(clov, st, s, x, v);
#pragma unroll
        for (int i = 0; i < 12; i++) v[i] = v[i] + 0.5f * a0[i];
        store_spinor(out0, st, s, v);
        if (two) {
            load_spinor_rw(in21, st, s, x);
            clover_apply<float>(clov, st, s, x, v);
#pragma unroll
            for (int i = 0; i < 12; i++) v[i] = v[i] + 0.5f * a1[i];
            store_spinor(out1, st, s, v);
        }
    }
}

template <typename R, int MODE>
__global__ void LQ_HOP_BOUNDS hop_kernel(Geom g, HopArgs<R> k)
{
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
    const Coords c = cb_coords(g, s, k.pout);
    if constexpr (std::is_same<R, float>::value)   // links and clover read once: no L1 allocation
        hop_body<R, MODE>(g, (const F4S *)k.Uout, (const F4S *)k.Uin, (const F4S *)k.clov, k.omega, k.in, k.in2,
                          k.b, k.out, s, c);
    else
        hop_body<R, MODE>(g, k.Uout, k.Uin, k.clov, k.omega, k.in, k.in2, k.b, k.out, s, c, k.clov2, k.out2);
}

// The same for FP32 K2 and its Richardson form, asked to fit six blocks per SM
// (80 registers, a few bytes of spills): measured on GB300 on 32^3 x 64, K2
// moves from 0.89 to 0.93 of the copy bandwidth this way, while K1 (78
// registers unbounded) gains nothing.
template <typename R, int MODE>
__global__ void __launch_bounds__(LQ_HOP_THREADS, 6) hop_kernel_occ(Geom g, HopArgs<R> k)
{
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
    const Coords c = cb_coords(g, s, k.pout);
    hop_body<R, MODE>(g, (const F4S *)k.Uout, (const F4S *)k.Uin, (const F4S *)k.clov, k.omega, k.in, k.in2, k.b,
                      k.out, s, c);
}


// BF16 spinors and links, FP32 clover and arithmetic (all modes)
struct HopArgsBF {
    const BfS4 *in, *in2, *b;
    BfS4 *out;
    const BfL2 *Uout, *Uin;
    const F4S *clov;   // FP32 clover blocks, read once
    float omega;
    int pout;
};
template <int MODE>
__global__ void LQ_HOP_BOUNDS hop_kernel_bf(Geom g, HopArgsBF k)
{
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
    const Coords c = cb_coords(g, s, k.pout);
    hop_body<float, MODE>(g, k.Uout, k.Uin, k.clov, k.omega, k.in, k.in2, k.b, k.out, s, c);
}

template <int MODE>
static void launch_hop_bf(const Exec &e, const HopCall &c)
{
    HopArgsBF k;
    k.in = (const BfS4 *)c.in;
    k.in2 = (const BfS4 *)c.in2;
    k.b = (const BfS4 *)c.b;
    k.out = (BfS4 *)c.out;
    k.Uout = (const BfL2 *)c.U[c.pout];
    k.Uin = (const BfL2 *)c.U[1 - c.pout];
    k.clov = (const F4S *)c.clov;
    k.omega = (float)c.omega;
    k.pout = c.pout;
    hop_kernel_bf<MODE><<<(unsigned)((e.g.Vh + LQ_HOP_THREADS - 1) / LQ_HOP_THREADS), LQ_HOP_THREADS, 0, e.st>>>(e.g, k);
}

// The batched hop over the right-hand sides of several lattices of different
// sizes in one persistent launch: each block walks the work table, an entry
// naming a lattice, a block of blockDim.x consecutive sites and the first of
// blockDim.y right-hand sides.  Entries of the same sites follow one another, so
// a site's links and clover block reach L1/L2 once for all its right-hand sides.
#ifdef LQ_GROUP_MINB
#define LQ_GROUP_BOUNDS __launch_bounds__(LQ_HOP_THREADS, LQ_GROUP_MINB)
#else
#define LQ_GROUP_BOUNDS __launch_bounds__(LQ_HOP_THREADS)
#endif
template <int MODE, int RPT>
__global__ void LQ_GROUP_BOUNDS hop_group_kernel(const LatDesc *__restrict__ d,
                                                                   const int4 *__restrict__ tiles, int ntiles,
                                                                   const float4 *in, const float4 *in2, float4 *out)
{
    constexpr int pout = MODE == HOP_K1 ? 1 : 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 w = __ldg(tiles + t);
        const LatDesc *L = d + w.x;
        const Geom g = L->g;
        const long long s = (long long)w.y * blockDim.x + threadIdx.x;
        const int r = w.z + RPT * threadIdx.y;   // the thread's first right-hand side
        if (s >= g.Vh || r >= L->nrhs) continue;
        const Coords c = cb_coords(g, s, pout);
        const long long o = L->off + r * L->fs;
        if (RPT == 1) {
            hop_body<float, MODE>(g, L->U[pout], L->U[1 - pout], L->clov[pout], 0.0f, in + o,
                                  in2 ? in2 + o : nullptr, (const float4 *)nullptr, out + o, s, c);
        } else {
            // the second right-hand side, when it exists (else the first is read twice, stored once)
            const bool two = r + 1 < L->nrhs;
            const long long o1 = two ? o + L->fs : o;
            hop_body2<MODE>(g, L->U[pout], L->U[1 - pout], L->clov[pout], in + o, in + o1,
                            in2 ? in2 + o : nullptr, in2 ? in2 + o1 : nullptr, out + o, out + o1, two, s, c);
        }
    }
}

// The batched hop with a site block's links and clover blocks staged in shared
// memory once for every right-hand side of its lattice.  A tile is (lattice,
// block of S consecutive sites); the block has S x (128 / S) threads, thread
// (x, y) owns site x of the block and walks right-hand sides y, y + 128/S, ...
// Staging: for every site of the block, the four forward links U_mu(x), the
// four backward links U_mu(x - mu) (read at the neighbour's index in the other
// parity's link array) and the two packed clover blocks of the output parity:
// 12 + 12 + 18 float4, laid out [entry][site] so that a warp's reads of one
// entry are consecutive.  The links and clover thus cross DRAM once per site,
// whatever the number of right-hand sides, and each right-hand side costs only
// its spinor traffic.
constexpr int kTileEntries = 42;   // float4 entries staged per site
constexpr int kTileFwd = 0, kTileBwd = 12, kTileClov = 24;

__device__ __forceinline__ void tile_link(const float4 *sm, int S, int e0, int x, cx<float> m[9])
{
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float4 t = sm[(e0 + k) * S + x];
        m[2 * k] = {t.x, t.y};
        m[2 * k + 1] = {t.z, t.w};
    }
    m[6] = cconj(cmul(m[1], m[5]) - cmul(m[2], m[4]));
    m[7] = cconj(cmul(m[2], m[3]) - cmul(m[0], m[5]));
    m[8] = cconj(cmul(m[0], m[4]) - cmul(m[1], m[3]));
}

// y = C x with both packed blocks of the site read from the staged entries
__device__ __forceinline__ void tile_clover(const float4 *sm, int S, int x, const cx<float> in[12], cx<float> y[12])
{
#pragma unroll
    for (int blk = 0; blk < 2; blk++) {
        float a[36];
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const float4 t = sm[(kTileClov + blk * 9 + k) * S + x];
            a[4 * k] = t.x;
            a[4 * k + 1] = t.y;
            a[4 * k + 2] = t.z;
            a[4 * k + 3] = t.w;
        }
        herm6_apply<float>(a, in + 6 * blk, y + 6 * blk);
    }
}

template <int MU, int SIGN>
__device__ __forceinline__ void tile_hop(cx<float> acc[12], const float4 *__restrict__ psi, long long st, int nb,
                                         const float4 *sm, int S, int x, float bsign)
{
    cx<float> p[12];
    load_spinor(psi, st, nb, p);
    cx<float> m[9];
    tile_link(sm, S, (SIGN < 0 ? kTileFwd : kTileBwd) + 3 * MU, x, m);
    hop_apply<MU, SIGN>(acc, p, m, bsign);
}

template <int MODE, int S>
__global__ void __launch_bounds__(LQ_HOP_THREADS, 5) hop_tile_kernel(const LatDesc *__restrict__ d,
                                                                     const int4 *__restrict__ tiles, int ntiles,
                                                                     const float4 *in, const float4 *in2, float4 *out)
{
    static_assert(MODE == HOP_K1 || MODE == HOP_K2, "K1 or K2");
    constexpr int R = LQ_HOP_THREADS / S;   // right-hand-side lanes
    constexpr int pout = MODE == HOP_K1 ? 1 : 0;
    extern __shared__ float4 tile_sm[];
    // after the staged entries: the eight neighbour indices of each site and its
    // two time-boundary factors, [10][S] words (kept here rather than in
    // registers across the loop over right-hand sides)
    int *tile_nb = reinterpret_cast<int *>(tile_sm + kTileEntries * S);
    float *tile_bc = reinterpret_cast<float *>(tile_nb + 8 * S);
    const int x = threadIdx.x, y = threadIdx.y;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 w = __ldg(tiles + t);
        const LatDesc *L = d + w.x;
        const Geom g = L->g;
        const long long st = g.stride;
        const long long s = (long long)w.y * S + x;
        const bool valid = s < g.Vh;
        // neighbour checkerboard indices (forward, backward per direction) and
        // the time-boundary factors; Vh < 2^31, so they fit an int
        int nf[4], nb[4];
        float tf = 1.0f, tb = 1.0f;
        if (valid) {
            const Coords c = cb_coords(g, s, pout);
            const long long base = c.row * g.Lxh;
            const int xp = (c.x + 1 == g.L[0]) ? 0 : c.x + 1;
            const int xm = (c.x == 0) ? g.L[0] - 1 : c.x - 1;
            nf[0] = (int)LQ_IDX(base + (xp >> 1), g.Vh, B_TILE_NB);
            nb[0] = (int)LQ_IDX(base + (xm >> 1), g.Vh, B_TILE_NB);
            long long dd = g.Lxh;
            const int co[3] = {c.y, c.z, c.t};
#pragma unroll
            for (int mu = 1; mu < 4; mu++) {
                const int ext = g.L[mu], q = co[mu - 1];
                nf[mu] = (int)LQ_IDX((q + 1 == ext) ? s - (long long)(ext - 1) * dd : s + dd, g.Vh, B_TILE_NB);
                nb[mu] = (int)LQ_IDX((q == 0) ? s + (long long)(ext - 1) * dd : s - dd, g.Vh, B_TILE_NB);
                dd *= ext;
            }
            if (c.t + 1 == g.L[3]) tf = (float)g.tbc;
            if (c.t == 0) tb = (float)g.tbc;
        }
        __syncthreads();   // the previous tile's reads of the staged entries are done
        if (valid) {
            const F4S *Uo = (const F4S *)L->U[pout];
            const F4S *Ui = (const F4S *)L->U[1 - pout];
            const F4S *Cl = (const F4S *)L->clov[pout];
            for (int e = y; e < kTileEntries; e += R) {
                const F4S *src;
                if (e < kTileBwd) src = Uo + e * st + s;
                else if (e < kTileClov) {
                    const int mu = (e - kTileBwd) / 3;   // selected, not indexed: nb stays in registers
                    const int n = mu == 0 ? nb[0] : mu == 1 ? nb[1] : mu == 2 ? nb[2] : nb[3];
                    src = Ui + (long long)(e - kTileBwd) * st + n;
                } else {
                    src = Cl + (long long)(e - kTileClov) * st + s;
                }
                tile_sm[e * S + x] = ldg(src);
            }
            if (y == 0) {
#pragma unroll
                for (int mu = 0; mu < 4; mu++) {
                    tile_nb[(2 * mu) * S + x] = nf[mu];
                    tile_nb[(2 * mu + 1) * S + x] = nb[mu];
                }
                tile_bc[x] = tf;
                tile_bc[S + x] = tb;
            }
        }
        __syncthreads();
        if (!valid) continue;
        for (int r = y; r < L->nrhs; r += R) {
            const long long o = L->off + r * L->fs;
            const float4 *pin = in + o;
            cx<float> acc[12];
#pragma unroll
            for (int i = 0; i < 12; i++) acc[i] = {0.0f, 0.0f};
            tile_hop<0, -1>(acc, pin, st, tile_nb[0 * S + x], tile_sm, S, x, 1.0f);
            tile_hop<0, +1>(acc, pin, st, tile_nb[1 * S + x], tile_sm, S, x, 1.0f);
            tile_hop<1, -1>(acc, pin, st, tile_nb[2 * S + x], tile_sm, S, x, 1.0f);
            tile_hop<1, +1>(acc, pin, st, tile_nb[3 * S + x], tile_sm, S, x, 1.0f);
            tile_hop<2, -1>(acc, pin, st, tile_nb[4 * S + x], tile_sm, S, x, 1.0f);
            tile_hop<2, +1>(acc, pin, st, tile_nb[5 * S + x], tile_sm, S, x, 1.0f);
            tile_hop<3, -1>(acc, pin, st, tile_nb[6 * S + x], tile_sm, S, x, tile_bc[x]);
            tile_hop<3, +1>(acc, pin, st, tile_nb[7 * S + x], tile_sm, S, x, tile_bc[S + x]);
            cx<float> v[12];
            if (MODE == HOP_K1) {
#pragma unroll
                for (int i = 0; i < 12; i++) acc[i] = -0.5f * acc[i];
                tile_clover(tile_sm, S, x, acc, v);
            } else {
                cx<float> xs[12];
                load_spinor_rw(in2 + o, st, s, xs);
                tile_clover(tile_sm, S, x, xs, v);
#pragma unroll
                for (int i = 0; i < 12; i++) v[i] = v[i] + 0.5f * acc[i];
            }
            store_spinor(out + o, st, s, v);
        }
    }
}

// ---------------------------------------------------------------------------
// df64 variant.  Each df64 operation is a chain of several FP32 instructions,
// so the fully unrolled eight-direction body of hop_kernel would not fit the
// instruction cache.  Here the eight hops share one loop body: the spin
// projection and reconstruction of direction d are the table entries
//   h0 = psi_0 + i^qa psi_pa,  h1 = psi_1 + i^qb psi_(5-pa)
//   acc_2 += i^qc u_ra,        acc_3 += i^qd u_(1-ra)
// (the same identities as `project` / `reconstruct` above, with s = -1 for the
// forward and +1 for the backward hop), and the backward link enters as U^+.
// ---------------------------------------------------------------------------
// y += A x for one packed Hermitian 6x6 block A (reals 0..5 the diagonal,
// then the strictly lower entries), read one entry at a time as the product
// needs it; the six sums are lazily normalised (dl_*) and left unnormalised.
__device__ __forceinline__ void herm6_fma_df(const df2 *__restrict__ Cb, long long stride, const cx<df64> x[6],
                                             cx<df64> y[6])
{
#pragma unroll
    for (int k = 0; k < 3; k++) {   // the diagonal: reals 2k, 2k+1
        const df2 t = ldg(Cb + k * stride);
        const df64 d0(t.rh, t.rl), d1(t.ih, t.il);
        dl_fma(y[2 * k].re, d0, x[2 * k].re);
        dl_fma(y[2 * k].im, d0, x[2 * k].im);
        dl_fma(y[2 * k + 1].re, d1, x[2 * k + 1].re);
        dl_fma(y[2 * k + 1].im, d1, x[2 * k + 1].im);
    }
#pragma unroll
    for (int i = 1; i < 6; i++)
#pragma unroll
        for (int j = 0; j < i; j++) {
            const cx<df64> l = df2_cx(ldg(Cb + (3 + tri(i, j)) * stride));
            dl_cfma(y[i], l, x[j]);    // lower entry
            dl_cfmac(y[j], l, x[i]);   // its conjugate above the diagonal
        }
}

__device__ __forceinline__ cx<df64> rot_i(cx<df64> z, int q)   // i^q z
{
    const cx<df64> a = (q & 1) ? cx<df64>{-z.im, z.re} : z;
    return (q & 2) ? cx<df64>{-a.re, -a.im} : a;
}

template <int MODE>
__device__ __forceinline__ void hop_df_body(const Geom &g, const HopArgs<df64> &k, const df2 *in, const df2 *in2,
                                            const df2 *bv, df2 *out, df2 *out2, long long s, const Coords &c)
{
    // per direction d = 2 mu + (backward): the partner of h0 is psi_3 for x, y
    // and psi_2 for z, t (acc_2 takes u_1 resp. u_0); the i-powers
    //   qa = {1,3,0,2,1,3,2,0}, qb = {1,3,2,0,3,1,2,0},
    //   qc = {3,1,2,0,3,1,2,0}, qd = {3,1,0,2,1,3,2,0}
    // are packed two bits per direction (no local-memory tables).  The
    // neighbour's components and the link's entries are read as the
    // projection and the product use them, and every sum is lazily normalised
    // (dl_*): acc is renormalised once, after the eight directions.
    constexpr unsigned QA = 11661u, QB = 10029u, QC = 10023u, QD = 11655u;
    const long long st = g.stride;
    cx<df64> acc[12];
#pragma unroll
    for (int i = 0; i < 12; i++) acc[i] = {df64(0.0f, 0.0f), df64(0.0f, 0.0f)};

    // the neighbour's checkerboard index in direction d, and whether the time
    // boundary flips the sign of the hop
    auto neighbour = [&](int d, bool &flip) {
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        flip = false;
        if (mu == 0) {
            const int xn = fwd ? (c.x + 1 == g.L[0] ? 0 : c.x + 1) : (c.x == 0 ? g.L[0] - 1 : c.x - 1);
            return (long long)LQ_IDX(c.row * g.Lxh + (xn >> 1), g.Vh, B_DF_NB);
        }
        const int coord = mu == 1 ? c.y : mu == 2 ? c.z : c.t;
        const int ext = g.L[mu];
        const long long dd = mu == 1 ? (long long)g.Lxh
                           : mu == 2 ? (long long)g.Lxh * g.L[1] : (long long)g.Lxh * g.L[1] * g.L[2];
        if (mu == 3) flip = g.tbc < 0 && (fwd ? coord + 1 == ext : coord == 0);
        if (fwd) return (long long)LQ_IDX((coord + 1 == ext) ? s - (long long)(ext - 1) * dd : s + dd, g.Vh, B_DF_NB);
        return (long long)LQ_IDX((coord == 0) ? s + (long long)(ext - 1) * dd : s - dd, g.Vh, B_DF_NB);
    };

#pragma unroll 1
    for (int d = 0; d < 8; d++) {
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        bool flip;
        const long long nb = neighbour(d, flip);
        const df2 *pn = in + nb;
        const int pa = d < 4 ? 3 : 2;
        const int qa = (QA >> (2 * d)) & 3, qb = (QB >> (2 * d)) & 3;
        cx<df64> h[6];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            h[a] = df2_cx(ldg(pn + a * st));
            dl_cadd(h[a], rot_i(df2_cx(ldg(pn + (pa == 3 ? 9 + a : 6 + a) * st)), qa));
            h[3 + a] = df2_cx(ldg(pn + (3 + a) * st));
            dl_cadd(h[3 + a], rot_i(df2_cx(ldg(pn + (pa == 3 ? 6 + a : 9 + a) * st)), qb));
        }
        const df2 *Um = (fwd ? k.Uout : k.Uin) + (long long)mu * 9 * st + (fwd ? s : nb);
        const int ra = d < 4 ? 1 : 0;
        const int qc = (QC >> (2 * d)) & 3, qd = (QD >> (2 * d)) & 3;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            // row a of U (forward) or of U^+ (backward): entries m[a*3+b] or conj(m[b*3+a])
            cx<df64> e[3];
#pragma unroll
            for (int b = 0; b < 3; b++) {
                const cx<df64> t = df2_cx(ldg(Um + (fwd ? a * 3 + b : b * 3 + a) * st));
                e[b] = fwd ? t : cx<df64>{t.re, dl_neg(t.im)};
            }
            cx<df64> u0 = dl_cmul(e[0], h[0]), u1 = dl_cmul(e[0], h[3]);
            dl_cfma(u0, e[1], h[1]);
            dl_cfma(u1, e[1], h[4]);
            dl_cfma(u0, e[2], h[2]);
            dl_cfma(u1, e[2], h[5]);
            if (flip) {
                u0 = {dl_neg(u0.re), dl_neg(u0.im)};
                u1 = {dl_neg(u1.re), dl_neg(u1.im)};
            }
            dl_cadd(acc[a], u0);
            dl_cadd(acc[3 + a], u1);
            dl_cadd(acc[6 + a], rot_i(ra ? u1 : u0, qc));
            dl_cadd(acc[9 + a], rot_i(ra ? u0 : u1, qd));
        }
    }
#pragma unroll
    for (int i = 0; i < 12; i++) acc[i] = dl_cnorm(acc[i]);

    // the site term, one 6x6 clover block (spins 0,1 then 2,3) at a time: six
    // components of the output are formed and stored per block (register
    // arrays are selected by the block, never indexed by it)
#pragma unroll 1
    for (int blk = 0; blk < 2; blk++) {
        const long long o = (long long)blk * 6 * st + s;
        const df2 *Cb = k.clov + (long long)blk * 18 * st + s;
        cx<df64> a6[6], y[6];
#pragma unroll
        for (int i = 0; i < 6; i++) a6[i] = blk ? acc[6 + i] : acc[i];
        if (MODE == HOP_K1) {   // y = C (-1/2 acc)
#pragma unroll
            for (int i = 0; i < 6; i++) {
                a6[i] = {dl_scale2(a6[i].re, -0.5f), dl_scale2(a6[i].im, -0.5f)};
                y[i] = {df64(0.0f, 0.0f), df64(0.0f, 0.0f)};
            }
            herm6_fma_df(Cb, st, a6, y);
#pragma unroll
            for (int i = 0; i < 6; i++) y[i] = dl_cnorm(y[i]);
        } else if (MODE == HOP_K2 || MODE == HOP_RICH || MODE == HOP_FULL || MODE == HOP_RES) {   // y = C x +- 1/2 acc
            const float f = (MODE == HOP_FULL || MODE == HOP_RES) ? -0.5f : 0.5f;
            cx<df64> x6[6];
#pragma unroll
            for (int i = 0; i < 6; i++) {
                x6[i] = df2_cx(in2[o + i * st]);
                y[i] = {dl_scale2(a6[i].re, f), dl_scale2(a6[i].im, f)};
            }
            herm6_fma_df(Cb, st, x6, y);
#pragma unroll
            for (int i = 0; i < 6; i++) y[i] = dl_cnorm(y[i]);
            if (MODE == HOP_RICH) {   // x + omega (b - D x)
#pragma unroll
                for (int i = 0; i < 6; i++) y[i] = x6[i] + k.omega * (df2_cx(ldg(bv + o + i * st)) - y[i]);
            }
            if (MODE == HOP_RES) {   // b - D x
#pragma unroll
                for (int i = 0; i < 6; i++) y[i] = df2_cx(ldg(bv + o + i * st)) - y[i];
            }
        } else {   // y = in2 + 1/2 acc, and for the reconstruction C^{-1} of that
#pragma unroll
            for (int i = 0; i < 6; i++) {
                cx<df64> t = df2_cx(in2[o + i * st]);
                dl_cadd(t, {dl_scale2(a6[i].re, 0.5f), dl_scale2(a6[i].im, 0.5f)});
                a6[i] = dl_cnorm(t);
            }
            if (MODE == HOP_RECON || MODE == HOP_RECON_RES) {
#pragma unroll
                for (int i = 0; i < 6; i++) y[i] = {df64(0.0f, 0.0f), df64(0.0f, 0.0f)};
                herm6_fma_df(Cb, st, a6, y);
#pragma unroll
                for (int i = 0; i < 6; i++) y[i] = dl_cnorm(y[i]);
                if (MODE == HOP_RECON_RES) {   // the parity's residual u - C x_o of the x_o just formed
                    cx<df64> z[6];
#pragma unroll
                    for (int i = 0; i < 6; i++) z[i] = {df64(0.0f, 0.0f), df64(0.0f, 0.0f)};
                    herm6_fma_df(k.clov2 + (long long)blk * 18 * st + s, st, y, z);
#pragma unroll
                    for (int i = 0; i < 6; i++) out2[o + i * st] = cx_df2(a6[i] - dl_cnorm(z[i]));
                }
            } else {
#pragma unroll
                for (int i = 0; i < 6; i++) y[i] = a6[i];
            }
        }
#pragma unroll
        for (int i = 0; i < 6; i++) out[o + i * st] = cx_df2(y[i]);
    }
}

#ifndef LQ_DF_MINB
#define LQ_DF_MINB 1
#endif
template <int MODE>
__global__ void __launch_bounds__(128, MODE == HOP_RECON_RES ? 3 : LQ_DF_MINB) hop_df_kernel(const __grid_constant__ Geom g,
                                                     const __grid_constant__ HopArgs<df64> k)
{
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
    const Coords c = cb_coords(g, s, k.pout);
#pragma unroll 1
    for (int r = 0; r < k.nrhs; r++) {
        const long long o = r * k.fs;
        hop_df_body<MODE>(g, k, k.in + o, k.in2 ? k.in2 + o : nullptr, k.b ? k.b + o : nullptr, k.out + o,
                          k.out2 ? k.out2 + o : nullptr, s, c);
    }
}

template <typename R>
__global__ void __launch_bounds__(256) clover_mul_kernel(Geom g, const typename St<R>::vec *__restrict__ C,
                                                         const typename St<R>::vec *in, typename St<R>::vec *out)
{
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
    cx<R> x[12], y[12];
    load_spinor_rw(in, g.stride, s, x);
    clover_apply<R>(C, g.stride, s, x, y);
    store_spinor(out, g.stride, s, y);
}

template <typename R, int MODE>
static void launch_hop(const Exec &e, const HopCall &c)
{
    typedef typename St<R>::vec V;
    HopArgs<R> k;
    k.in = (const V *)c.in;
    k.in2 = (const V *)c.in2;
    k.b = (const V *)c.b;
    k.out = (V *)c.out;
    k.Uout = (const V *)c.U[c.pout];
    k.Uin = (const V *)c.U[1 - c.pout];
    k.clov = (const V *)c.clov;
    k.clov2 = (const V *)c.clov2;
    k.out2 = (V *)c.out2;
    k.omega = R(c.omega);
    k.pout = c.pout;
    k.nrhs = c.nrhs;
    k.fs = (long long)St<R>::SPINOR_VECS * e.g.stride;
    const unsigned blocks = (unsigned)((e.g.Vh + LQ_HOP_THREADS - 1) / LQ_HOP_THREADS);
    if constexpr (std::is_same<R, df64>::value)
        hop_df_kernel<MODE><<<blocks, 128, 0, e.st>>>(e.g, k);
    else
    {
        // several right-hand sides of FP64 or FP32 fields: one launch each (the
        // batched FP32 solve uses the work-table kernel instead)
        for (int r = 0; r < c.nrhs; r++) {
            HopArgs<R> kr = k;
            const long long o = r * k.fs;
            kr.in = k.in + o;
            kr.in2 = k.in2 ? k.in2 + o : nullptr;
            kr.b = k.b ? k.b + o : nullptr;
            kr.out = k.out + o;
            kr.out2 = k.out2 ? k.out2 + o : nullptr;
            if constexpr (std::is_same<R, float>::value && (MODE == HOP_K2 || MODE == HOP_RICH))
                hop_kernel_occ<R, MODE><<<blocks, LQ_HOP_THREADS, 0, e.st>>>(e.g, kr);
            else
                hop_kernel<R, MODE><<<blocks, LQ_HOP_THREADS, 0, e.st>>>(e.g, kr);
        }
    }
}

// algorithmic bytes per output site of one hopping launch (FP64 and df64 share
// the 8-byte-per-real layout)
static double hop_site_bytes(int mode, int prec, int nrhs)
{
    const bool wide = prec == P64 || prec == PDF;
    const double sp = wide ? 192.0 : prec == P16 ? 48.0 : 96.0;   // spinor
    const double lk = wide ? 144.0 : prec == P16 ? 24.0 : 48.0;   // link (18 / 12 reals)
    const double cl = wide ? 576.0 : 288.0;                       // 72-real clover pair (FP32 for BF16)
    double once = 8 * lk, per = sp + sp;            // links; neighbours and output per rhs
    switch (mode) {
    case HOP_K1: once += cl; break;
    case HOP_K2: case HOP_FULL: once += cl; per += sp; break;
    case HOP_RICH: once += cl; per += 2 * sp; break;
    case HOP_PREP: per += sp; break;
    case HOP_RECON: once += cl; per += sp; break;
    case HOP_RES: once += cl; per += 2 * sp; break;                  // x, b
    case HOP_RECON_RES: once += 2 * cl; per += 2 * sp; break;        // C^{-1} and C; b in, x and r out
    }
    return once + nrhs * per;
}

static int hop_class(int mode, int prec)
{
    if (prec == P16) return mode == HOP_K1 ? K_HOP_K1_BF16 : (mode == HOP_K2 || mode == HOP_RICH) ? K_HOP_K2_BF16 : K_HOP_OTHER;
    if (mode == HOP_K1) return prec == P64 ? K_HOP_K1_F64 : prec == P32 ? K_HOP_K1_F32 : K_HOP_K1_DF;
    if (mode == HOP_K2 || mode == HOP_RICH) return prec == P64 ? K_HOP_K2_F64 : prec == P32 ? K_HOP_K2_F32 : K_HOP_K2_DF;
    return K_HOP_OTHER;
}

// algorithmic flops per site: 1320 for the eight hops (projection 12, two
// SU(3) mat-vecs 132, accumulation 24, per direction, less the first
// accumulation), 552 per clover-block pair, 24 per spinor add / scale
static const double c_hop_flops[8] = {1320 + 552, 1320 + 552 + 24, 1320 + 552 + 24 + 48,
                                      1320 + 552 + 24, 1320 + 24, 1320 + 24 + 552,
                                      1320 + 552 + 48, 1320 + 24 + 2 * 552 + 24};

double hop_bytes(int mode, int prec, int nrhs, double sites) { return sites * hop_site_bytes(mode, prec, nrhs); }
double hop_flops(int mode, double site_rhs) { return site_rhs * c_hop_flops[mode]; }

// dynamic shared memory of the staged batched hop with S sites per tile
static size_t tile_smem(int S) { return (size_t)kTileEntries * S * sizeof(float4) + 10 * S * sizeof(int); }

int hop_group_resident(int rpt, int spt)
{
    int a = 0, b = 0;
    if (rpt == 0) {
        if (spt == 64) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, hop_tile_kernel<HOP_K1, 64>, LQ_HOP_THREADS, tile_smem(64));
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, hop_tile_kernel<HOP_K2, 64>, LQ_HOP_THREADS, tile_smem(64));
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, hop_tile_kernel<HOP_K1, 32>, LQ_HOP_THREADS, tile_smem(32));
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, hop_tile_kernel<HOP_K2, 32>, LQ_HOP_THREADS, tile_smem(32));
        }
    } else if (rpt == 2) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, hop_group_kernel<HOP_K1, 2>, LQ_HOP_THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, hop_group_kernel<HOP_K2, 2>, LQ_HOP_THREADS, 0);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, hop_group_kernel<HOP_K1, 1>, LQ_HOP_THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, hop_group_kernel<HOP_K2, 1>, LQ_HOP_THREADS, 0);
    }
    const int r = a < b ? a : b;
    return r < 1 ? 1 : r;
}

void hop_group(const Exec &e, int mode, const LatDesc *desc, const int4 *tiles, int ntiles, int grid, int spt,
               int rpt, const void *in, const void *in2, void *out, double bytes, double flops)
{
    Launch L_(e, mode == HOP_K1 ? K_HOP_K1_F32 : K_HOP_K2_F32, bytes, flops);
    const dim3 block(spt, LQ_HOP_THREADS / spt);
    const float4 *i1 = (const float4 *)in, *i2 = (const float4 *)in2;
    float4 *o = (float4 *)out;
    if (rpt == 0) {   // staged links and clover, every right-hand side of the tile's lattice
        const size_t sm = tile_smem(spt);
        if (spt == 64) {
            if (mode == HOP_K1) hop_tile_kernel<HOP_K1, 64><<<grid, block, sm, e.st>>>(desc, tiles, ntiles, i1, i2, o);
            else hop_tile_kernel<HOP_K2, 64><<<grid, block, sm, e.st>>>(desc, tiles, ntiles, i1, i2, o);
        } else {
            if (mode == HOP_K1) hop_tile_kernel<HOP_K1, 32><<<grid, block, sm, e.st>>>(desc, tiles, ntiles, i1, i2, o);
            else hop_tile_kernel<HOP_K2, 32><<<grid, block, sm, e.st>>>(desc, tiles, ntiles, i1, i2, o);
        }
        return;
    }
    if (mode == HOP_K1 && rpt == 2) hop_group_kernel<HOP_K1, 2><<<grid, block, 0, e.st>>>(desc, tiles, ntiles, i1, i2, o);
    else if (mode == HOP_K1) hop_group_kernel<HOP_K1, 1><<<grid, block, 0, e.st>>>(desc, tiles, ntiles, i1, i2, o);
    else if (rpt == 2) hop_group_kernel<HOP_K2, 2><<<grid, block, 0, e.st>>>(desc, tiles, ntiles, i1, i2, o);
    else hop_group_kernel<HOP_K2, 1><<<grid, block, 0, e.st>>>(desc, tiles, ntiles, i1, i2, o);
}

void hop(const Exec &e, const HopCall &c)
{
#define LQ_CASE(M)                                                              \
    case M:                                                                     \
        if (c.prec == P64) launch_hop<double, M>(e, c);                         \
        else if (c.prec == P32) launch_hop<float, M>(e, c);                     \
        else if (c.prec == P16) launch_hop_bf<M>(e, c);                         \
        else launch_hop<df64, M>(e, c);                                         \
        break;
    // df64 keeps the right-hand sides of a site in one thread (links and clover
    // counted once); FP64 and FP32 launch once per right-hand side
    const double site_bytes = c.prec == PDF ? hop_site_bytes(c.mode, c.prec, c.nrhs)
                                            : c.nrhs * hop_site_bytes(c.mode, c.prec, 1);
    Launch L_(e, hop_class(c.mode, c.prec), (double)e.g.Vh * site_bytes, (double)e.g.Vh * c_hop_flops[c.mode] * c.nrhs);
    switch (c.mode) {
        LQ_CASE(HOP_K1)
        LQ_CASE(HOP_K2)
        LQ_CASE(HOP_RICH)
        LQ_CASE(HOP_FULL)
        LQ_CASE(HOP_PREP)
        LQ_CASE(HOP_RECON)
    case HOP_RES:   // FP64 and df64 only (the solve's full residual)
        if (c.prec == P64) launch_hop<double, HOP_RES>(e, c);
        else if (c.prec == PDF) launch_hop<df64, HOP_RES>(e, c);
        break;
    case HOP_RECON_RES:
        if (c.prec == P64) launch_hop<double, HOP_RECON_RES>(e, c);
        else if (c.prec == PDF) launch_hop<df64, HOP_RECON_RES>(e, c);
        break;
    }
#undef LQ_CASE
}

void clover_mul(const Exec &e, int prec, const void *clov, const void *in, void *out)
{
    Launch L_(e, K_HOP_OTHER, (double)e.g.Vh * (prec != P32 ? 192.0 * 2 + 576.0 : 96.0 * 2 + 288.0),
              (double)e.g.Vh * 552);
    const unsigned blocks = (unsigned)((e.g.Vh + 255) / 256);
    if (prec == P64)
        clover_mul_kernel<double><<<blocks, 256, 0, e.st>>>(e.g, (const double2 *)clov, (const double2 *)in,
                                                           (double2 *)out);
    else if (prec == P32)
        clover_mul_kernel<float><<<blocks, 256, 0, e.st>>>(e.g, (const float4 *)clov, (const float4 *)in,
                                                          (float4 *)out);
    else
        clover_mul_kernel<df64><<<blocks, 256, 0, e.st>>>(e.g, (const df2 *)clov, (const df2 *)in, (df2 *)out);
}

}  // namespace lq
