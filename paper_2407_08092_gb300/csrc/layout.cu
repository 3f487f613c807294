// Layout kernels: natural complex-double fields <-> internal checkerboarded
// structure-of-arrays fields, precision conversion and the gamma_5 multiply.
// (Sec. 2.4.5: odd-even reordering; the internal order is even sites first,
// each parity in lexicographic order.)
#include "lq_kernels.h"

namespace lq {

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ df2 to_df2(double2 v)
{
    const df64 r = df_split(v.x), i = df_split(v.y);
    return df2{r.hi, r.lo, i.hi, i.lo};
}
__device__ __forceinline__ double2 from_df2(df2 v) { return make_double2(df_join(v.rh, v.rl), df_join(v.ih, v.il)); }

// parity of lattice site lex (32-bit arithmetic: a lattice of 2^31 sites
// would not fit one spinor field in HBM, and lq_create rejects it)
__device__ __forceinline__ int lex_parity(const Geom &g, long long lex)
{
    unsigned r = (unsigned)lex;
    const unsigned c0 = r % (unsigned)g.L[0];
    r /= (unsigned)g.L[0];
    const unsigned c1 = r % (unsigned)g.L[1];
    r /= (unsigned)g.L[1];
    const unsigned c2 = r % (unsigned)g.L[2], c3 = r / (unsigned)g.L[2];
    return (int)((c0 + c1 + c2 + c3) & 1u);
}

// The natural fields are row-major [site][components] arrays of complex
// doubles; the internal ones are component-major per parity.  Each CTA moves
// a tile of TS consecutive natural rows through shared memory, so both the
// natural rows and every internal component are read and written in
// contiguous runs.  On a full lattice the rows lex0 .. lex0 + TS - 1 (lex0 a
// multiple of TS) hold TS/2 sites of each parity with consecutive
// checkerboard indices lex0/2 .. lex0/2 + TS/2 - 1: rows 2j and 2j + 1 share
// index lex0/2 + j and have opposite parities (the lattice extents are even).
constexpr int TS = 64;            // natural rows per tile
constexpr int TT = 128;           // threads per tile
constexpr int TPAD = 13;          // double2 slots per tile row of a spinor (12 + 1 against bank conflicts)

// internal vector k of a site from its 12 complex components, and back
template <int PR> struct Vec;
template <> struct Vec<P64> {
    static constexpr int N = 12;
    typedef double2 T;
    static __device__ __forceinline__ T from(const double2 *row, int k) { return row[k]; }
    static __device__ __forceinline__ void to(T v, double2 *row, int k) { row[k] = v; }
};
template <> struct Vec<PDF> {
    static constexpr int N = 12;
    typedef df2 T;
    static __device__ __forceinline__ T from(const double2 *row, int k) { return to_df2(row[k]); }
    static __device__ __forceinline__ void to(T v, double2 *row, int k) { row[k] = from_df2(v); }
};
template <> struct Vec<P32> {
    static constexpr int N = 6;   // two complex components per float4
    typedef float4 T;
    static __device__ __forceinline__ T from(const double2 *row, int k)
    {
        const double2 a = row[2 * k], b = row[2 * k + 1];
        return make_float4(d2f_bits(a.x), d2f_bits(a.y), d2f_bits(b.x), d2f_bits(b.y));
    }
    static __device__ __forceinline__ void to(T v, double2 *row, int k)
    {
        row[2 * k] = make_double2(f2d_bits(v.x), f2d_bits(v.y));
        row[2 * k + 1] = make_double2(f2d_bits(v.z), f2d_bits(v.w));
    }
};

// row of the tile and internal site index of output item j of parity p
// (FULL: lattice rows split by parity; else: a field of one parity, row = site)
template <bool FULL>
__device__ __forceinline__ int tile_row(const unsigned char *par, int j, int p)
{
    return FULL ? 2 * j + (par[j] != p) : j;
}

// shared-memory slot of tile row r: with FULL the rows are stored de-interleaved
// by parity (row r at (r & 1) * TS/2 + r / 2), so that the rows 2j + b that
// consecutive j read sit in consecutive slots, and TPAD = 13 spreads eight
// consecutive slots over all eight 16-byte bank groups
template <bool FULL>
__device__ __forceinline__ int tile_slot(int r)
{
    return FULL ? (r & 1) * (TS / 2) + (r >> 1) : r;
}

// natural [n][12] c128 -> internal field(s): f0 (FULL: even sites), f1 (odd sites)
template <int PR, bool FULL>
__global__ void __launch_bounds__(TT) import_tile_kernel(Geom g, const double2 *__restrict__ nat,
                                                         typename Vec<PR>::T *f0, typename Vec<PR>::T *f1)
{
    __shared__ double2 tile[TS][TPAD];
    __shared__ unsigned char par[TS / 2];
    const long long n = FULL ? g.V : g.Vh;
    const long long r0 = (long long)blockIdx.x * TS;
    const int rows = (int)(n - r0 < TS ? n - r0 : TS);
    for (int i = threadIdx.x; i < rows * 12; i += TT) tile[tile_slot<FULL>(i / 12)][i % 12] = __ldg(nat + r0 * 12 + i);
    if (FULL && threadIdx.x < TS / 2 && 2 * (int)threadIdx.x < rows) par[threadIdx.x] = lex_parity(g, r0 + 2 * threadIdx.x);
    __syncthreads();
    constexpr int NV = Vec<PR>::N, PER = FULL ? TS / 2 : TS;
    const long long s0 = FULL ? r0 / 2 : r0;
    if (rows == TS) {   // a whole tile: every index split below is by a constant
#pragma unroll
        for (int w = threadIdx.x; w < (FULL ? 2 : 1) * NV * PER; w += TT) {
            const int j = w % PER, pk = w / PER, p = pk / NV, k = pk % NV;
            typename Vec<PR>::T *f = p ? f1 : f0;
            f[k * g.stride + LQ_IDX(s0 + j, g.Vh, B_LAYOUT)] =
                Vec<PR>::from(tile[tile_slot<FULL>(LQ_IDX(tile_row<FULL>(par, j, p), rows, B_LAYOUT))], k);
        }
    } else {            // the last, partial tile (rows is even on a full lattice)
        const int per = FULL ? rows / 2 : rows;
        for (int w = threadIdx.x; w < (FULL ? 2 : 1) * NV * per; w += TT) {
            const int j = w % per, pk = w / per, p = pk / NV, k = pk % NV;
            typename Vec<PR>::T *f = p ? f1 : f0;
            f[k * g.stride + LQ_IDX(s0 + j, g.Vh, B_LAYOUT)] =
                Vec<PR>::from(tile[tile_slot<FULL>(LQ_IDX(tile_row<FULL>(par, j, p), rows, B_LAYOUT))], k);
        }
    }
}

// internal field(s) -> natural [n][12] c128
template <int PR, bool FULL>
__global__ void __launch_bounds__(TT) export_tile_kernel(Geom g, const typename Vec<PR>::T *__restrict__ f0,
                                                         const typename Vec<PR>::T *__restrict__ f1, double2 *nat)
{
    __shared__ double2 tile[TS][TPAD];
    __shared__ unsigned char par[TS / 2];
    const long long n = FULL ? g.V : g.Vh;
    const long long r0 = (long long)blockIdx.x * TS;
    const int rows = (int)(n - r0 < TS ? n - r0 : TS);
    if (FULL && threadIdx.x < TS / 2 && 2 * (int)threadIdx.x < rows) par[threadIdx.x] = lex_parity(g, r0 + 2 * threadIdx.x);
    __syncthreads();
    constexpr int NV = Vec<PR>::N, PER = FULL ? TS / 2 : TS;
    const long long s0 = FULL ? r0 / 2 : r0;
    if (rows == TS) {
#pragma unroll
        for (int w = threadIdx.x; w < (FULL ? 2 : 1) * NV * PER; w += TT) {
            const int j = w % PER, pk = w / PER, p = pk / NV, k = pk % NV;
            const typename Vec<PR>::T *f = p ? f1 : f0;
            Vec<PR>::to(f[k * g.stride + LQ_IDX(s0 + j, g.Vh, B_LAYOUT)],
                        tile[tile_slot<FULL>(LQ_IDX(tile_row<FULL>(par, j, p), rows, B_LAYOUT))], k);
        }
    } else {
        const int per = FULL ? rows / 2 : rows;
        for (int w = threadIdx.x; w < (FULL ? 2 : 1) * NV * per; w += TT) {
            const int j = w % per, pk = w / per, p = pk / NV, k = pk % NV;
            const typename Vec<PR>::T *f = p ? f1 : f0;
            Vec<PR>::to(f[k * g.stride + LQ_IDX(s0 + j, g.Vh, B_LAYOUT)],
                        tile[tile_slot<FULL>(LQ_IDX(tile_row<FULL>(par, j, p), rows, B_LAYOUT))], k);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < rows * 12; i += TT) nat[r0 * 12 + i] = tile[tile_slot<FULL>(i / 12)][i % 12];
}

// gauge links: U_nat[lex][mu][3][3] c128 -> per parity U64 [mu][9][stride]
// double2, U32 [mu][3][stride] float4 (rows 0 and 1: 12 reals) and Udf
// [mu][9][stride] df2; a tile of TL lattice rows (36 complex numbers each)
constexpr int TL = 32;
constexpr int LPAD = 37;
__global__ void __launch_bounds__(TT) import_links_kernel(Geom g, const double2 *__restrict__ U, double2 *U64e,
                                                          double2 *U64o, float4 *U32e, float4 *U32o, df2 *Udfe,
                                                          df2 *Udfo)
{
    // tile rows are stored de-interleaved, row r at slot (r & 1) * TL/2 + r / 2, so
    // that the rows 2j + b that consecutive j read below sit in consecutive slots
    // (distinct shared-memory banks) whatever b
    __shared__ double2 tile[TL][LPAD];
    __shared__ unsigned char par[TL / 2];
    const long long r0 = (long long)blockIdx.x * TL;
    const int rows = (int)(g.V - r0 < TL ? g.V - r0 : TL);
    for (int i = threadIdx.x; i < rows * 36; i += TT) {
        const int r = i / 36;
        tile[(r & 1) * (TL / 2) + (r >> 1)][i % 36] = __ldg(U + r0 * 36 + i);
    }
    if (threadIdx.x < TL / 2 && 2 * (int)threadIdx.x < rows) par[threadIdx.x] = lex_parity(g, r0 + 2 * threadIdx.x);
    __syncthreads();
    const long long s0 = r0 / 2;
    // entry k = mu * 9 + e of link mu: its FP64 copy (only when asked for), its
    // df64 split, and for the first two rows (e < 6) the FP32 value, which is the
    // split's high part: the half (e & 1) of float4 mu * 3 + e / 2 of the
    // 12-real FP32 link
    auto put = [&](int j, int pk) {
        const int p = pk / 36, k = pk % 36;
        const int r = (int)LQ_IDX(tile_row<true>(par, j, p), rows, B_LAYOUT);
        const double2 *row = tile[(r & 1) * (TL / 2) + (r >> 1)];
        const long long s = LQ_IDX(s0 + j, g.Vh, B_LAYOUT);
        if (U64e) (p ? U64o : U64e)[k * g.stride + s] = row[k];
        const df2 d = to_df2(row[k]);
        (p ? Udfo : Udfe)[k * g.stride + s] = d;
        const int mu = k / 9, e = k % 9;
        if (e < 6) {
            float2 *f = reinterpret_cast<float2 *>(p ? U32o : U32e);
            f[((mu * 3 + e / 2) * g.stride + s) * 2 + (e & 1)] = make_float2(d.rh, d.ih);
        }
    };
    if (rows == TL) {   // a whole tile: w splits by constants
        for (int w = threadIdx.x; w < 2 * 36 * (TL / 2); w += TT) put(w % (TL / 2), w / (TL / 2));
    } else {
        const int per = rows / 2;
        for (int w = threadIdx.x; w < 2 * 36 * per; w += TT) put(w % per, w / per);
    }
}

void import_links(const Exec &e, const void *U_nat, void *U64[2], void *U32[2], void *Udf[2])
{
    Launch L_(e, K_LAYOUT, (double)e.g.V * 4 * (144 + (U64 ? 144 : 0) + 48 + 144));
    import_links_kernel<<<nblk(e.g.V, TL), TT, 0, e.st>>>(e.g, (const double2 *)U_nat,
                                                          U64 ? (double2 *)U64[0] : nullptr,
                                                          U64 ? (double2 *)U64[1] : nullptr, (float4 *)U32[0],
                                                          (float4 *)U32[1], (df2 *)Udf[0], (df2 *)Udf[1]);
}

// ---- spinors ----------------------------------------------------------------
template <int PR, bool FULL>
static void import_t(const Exec &e, const void *nat, void *f0, void *f1)
{
    typedef typename Vec<PR>::T T;
    const long long n = FULL ? e.g.V : e.g.Vh;
    import_tile_kernel<PR, FULL><<<nblk(n, TS), TT, 0, e.st>>>(e.g, (const double2 *)nat, (T *)f0, (T *)f1);
}
template <int PR, bool FULL>
static void export_t(const Exec &e, const void *f0, const void *f1, void *nat)
{
    typedef typename Vec<PR>::T T;
    const long long n = FULL ? e.g.V : e.g.Vh;
    export_tile_kernel<PR, FULL><<<nblk(n, TS), TT, 0, e.st>>>(e.g, (const T *)f0, (const T *)f1, (double2 *)nat);
}

void import_half(const Exec &e, int prec, const void *nat, void *f)
{
    if (prec == P16) {
        bf16_import_half(e, nat, f);
        return;
    }
    Launch L_(e, K_LAYOUT, (double)e.g.Vh * (192 + (prec == P32 ? 96 : 192)));
    if (prec == PDF) import_t<PDF, false>(e, nat, f, nullptr);
    else if (prec == P64) import_t<P64, false>(e, nat, f, nullptr);
    else import_t<P32, false>(e, nat, f, nullptr);
}

void export_half(const Exec &e, int prec, const void *f, void *nat)
{
    if (prec == P16) {
        bf16_export_half(e, f, nat);
        return;
    }
    Launch L_(e, K_LAYOUT, (double)e.g.Vh * (192 + (prec == P32 ? 96 : 192)));
    if (prec == PDF) export_t<PDF, false>(e, f, nullptr, nat);
    else if (prec == P64) export_t<P64, false>(e, f, nullptr, nat);
    else export_t<P32, false>(e, f, nullptr, nat);
}

void import_full(const Exec &e, int prec, const void *nat, void *fe, void *fo)
{
    Launch L_(e, K_LAYOUT, (double)e.g.V * (192 + (prec == P32 ? 96 : 192)));
    if (prec == PDF) import_t<PDF, true>(e, nat, fe, fo);
    else if (prec == P64) import_t<P64, true>(e, nat, fe, fo);
    else import_t<P32, true>(e, nat, fe, fo);
}

void export_full(const Exec &e, int prec, const void *fe, const void *fo, void *nat)
{
    Launch L_(e, K_LAYOUT, (double)e.g.V * (192 + (prec == P32 ? 96 : 192)));
    if (prec == PDF) export_t<PDF, true>(e, fe, fo, nat);
    else if (prec == P64) export_t<P64, true>(e, fe, fo, nat);
    else export_t<P32, true>(e, fe, fo, nat);
}

// ---- conversion and gamma_5 -------------------------------------------------
__global__ void d2f_kernel(Geom g, const double2 *__restrict__ in, float4 *out)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        double2 a = __ldg(in + (2 * k) * g.stride + s), b = __ldg(in + (2 * k + 1) * g.stride + s);
        out[k * g.stride + s] = make_float4(d2f_bits(a.x), d2f_bits(a.y), d2f_bits(b.x), d2f_bits(b.y));
    }
}
__global__ void f2d_kernel(Geom g, const float4 *__restrict__ in, double2 *out)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        float4 t = __ldg(in + k * g.stride + s);
        out[(2 * k) * g.stride + s] = make_double2(f2d_bits(t.x), f2d_bits(t.y));
        out[(2 * k + 1) * g.stride + s] = make_double2(f2d_bits(t.z), f2d_bits(t.w));
    }
}

__global__ void d2df_kernel(Geom g, const double2 *__restrict__ in, df2 *out)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int c = 0; c < 12; c++) out[c * g.stride + s] = to_df2(__ldg(in + c * g.stride + s));
}
__global__ void df2d_kernel(Geom g, const df2 *__restrict__ in, double2 *out)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int c = 0; c < 12; c++) out[c * g.stride + s] = from_df2(ldg(in + c * g.stride + s));
}
// FP32 -> df64 is exact (lo = 0); df64 -> FP32 rounds hi + lo once
__global__ void f2df_kernel(Geom g, const float4 *__restrict__ in, df2 *out)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const float4 t = __ldg(in + k * g.stride + s);
        out[(2 * k) * g.stride + s] = df2{t.x, 0.0f, t.y, 0.0f};
        out[(2 * k + 1) * g.stride + s] = df2{t.z, 0.0f, t.w, 0.0f};
    }
}
__global__ void df2f_kernel(Geom g, const df2 *__restrict__ in, float4 *out)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const df2 a = ldg(in + (2 * k) * g.stride + s), b = ldg(in + (2 * k + 1) * g.stride + s);
        out[k * g.stride + s] = make_float4(__fadd_rn(a.rh, a.rl), __fadd_rn(a.ih, a.il), __fadd_rn(b.rh, b.rl),
                                            __fadd_rn(b.ih, b.il));
    }
}

void convert(const Exec &e, int from, const void *in, int to, void *out)
{
    if (from == P16 || to == P16) {
        bf16_convert(e, from, in, to, out);
        return;
    }
    if (from == to) {
        copy(e, from, in, out);
        return;
    }
    const double bytes = (double)e.g.Vh * ((from == P32 ? 96 : 192) + (to == P32 ? 96 : 192));
    Launch L_(e, K_LAYOUT, bytes);
    const unsigned b = nblk(e.g.Vh, 256);
    if (from == P64 && to == P32) d2f_kernel<<<b, 256, 0, e.st>>>(e.g, (const double2 *)in, (float4 *)out);
    else if (from == P32 && to == P64) f2d_kernel<<<b, 256, 0, e.st>>>(e.g, (const float4 *)in, (double2 *)out);
    else if (from == P64 && to == PDF) d2df_kernel<<<b, 256, 0, e.st>>>(e.g, (const double2 *)in, (df2 *)out);
    else if (from == PDF && to == P64) df2d_kernel<<<b, 256, 0, e.st>>>(e.g, (const df2 *)in, (double2 *)out);
    else if (from == P32 && to == PDF) f2df_kernel<<<b, 256, 0, e.st>>>(e.g, (const float4 *)in, (df2 *)out);
    else df2f_kernel<<<b, 256, 0, e.st>>>(e.g, (const df2 *)in, (float4 *)out);
}

// gamma_5 = diag(1, 1, -1, -1): negate the components of spins 2 and 3
// (the last half of the vectors of a site in either precision); in place, the
// first half is left untouched
__global__ void gamma5_d_kernel(Geom g, const double2 *in, double2 *out)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int k = in == out ? 6 : 0; k < 12; k++) {
        double2 t = in[k * g.stride + s];
        if (k >= 6) t = make_double2(-t.x, -t.y);
        out[k * g.stride + s] = t;
    }
}
__global__ void gamma5_f_kernel(Geom g, const float4 *in, float4 *out)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int k = in == out ? 3 : 0; k < 6; k++) {
        float4 t = in[k * g.stride + s];
        if (k >= 3) t = make_float4(-t.x, -t.y, -t.z, -t.w);
        out[k * g.stride + s] = t;
    }
}

__global__ void gamma5_df_kernel(Geom g, const float4 *in, float4 *out)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int k = in == out ? 6 : 0; k < 12; k++) {
        float4 t = in[k * g.stride + s];
        if (k >= 6) t = make_float4(-t.x, -t.y, -t.z, -t.w);
        out[k * g.stride + s] = t;
    }
}

void gamma5(const Exec &e, int prec, const void *in, void *out)
{
    if (prec == P16) {
        bf16_gamma5(e, in, out);
        return;
    }
    Launch L_(e, K_LAYOUT, (double)e.g.Vh * (in == out ? 1 : 2) * (prec == P32 ? 96 : 192));
    if (prec == PDF) {
        gamma5_df_kernel<<<nblk(e.g.Vh, 256), 256, 0, e.st>>>(e.g, (const float4 *)in, (float4 *)out);
        return;
    }
    if (prec == P64)
        gamma5_d_kernel<<<nblk(e.g.Vh, 256), 256, 0, e.st>>>(e.g, (const double2 *)in, (double2 *)out);
    else
        gamma5_f_kernel<<<nblk(e.g.Vh, 256), 256, 0, e.st>>>(e.g, (const float4 *)in, (float4 *)out);
}

}  // namespace lq
