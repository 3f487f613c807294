// Internal definitions of the GB300 odd-even Wilson-clover library.
//
// Internal layout (never visible through the C ABI)
// -------------------------------------------------
// Sites of one parity are numbered by the checkerboard index cb = lex/2
// (Lx even), so a half spinor in natural order is already in cb order.  Every
// per-site quantity is stored structure-of-arrays over cb with a padded
// stride (a multiple of 64 sites), in 16-byte vectors so that a warp reads
// 512 contiguous bytes per component:
//
//   spinor   FP64: [12][stride] double2        (component = spin*3 + colour)
//            FP32: [ 6][stride] float4         (two components per float4)
//   links    FP64: [4 mu][9][stride] double2   (full 3x3, row-major)
//            FP32: [4 mu][3][stride] float4    (rows 0 and 1; row 2 = conj(r0 x r1))
//   clover   [2 blocks][36 reals][stride] as 18 double2 (FP64) or 9 float4 (FP32):
//            the 6x6 Hermitian block packed as 6 real diagonal entries, then the
//            15 strictly-lower complex entries (1,0),(2,0),(2,1),(3,0),...,(5,4).
//
// Links, clover and spinors exist once per parity; the link array of parity p
// holds U_mu(x) for the sites x of parity p.  The fermion time boundary sign is
// applied inside the hopping kernels (not folded into the links), so the same
// link copies serve the clover term and both precisions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lq {

struct Geom {
    int L[4];
    int Lxh;          // Lx / 2
    int tbc;          // +1 / -1
    long long V;      // sites
    long long Vh;     // sites per parity
    long long stride; // padded Vh
};

// ---------------------------------------------------------------------------
// Index checks of the checked build (compiled with -DLQ_BOUNDS).
// LQ_IDX(i, n, code) is i when 0 <= i < n.  Otherwise the checked build
// records the violation -- a count and the code of the first one, in device
// flags of the translation unit -- and yields 0, so that the access stays
// inside the buffer and nothing traps or faults; lq_bounds_check reads and
// clears the flags of every translation unit.  The normal build compiles
// LQ_IDX(i, n, code) to i.
// ---------------------------------------------------------------------------
enum BoundsSite : unsigned {
    B_HOP_SITE = 1,   // output site of a hopping kernel
    B_HOP_NB,         // neighbour index of the FP64 / FP32 / BF16 hopping kernels
    B_DF_NB,          // neighbour index of the df64 hopping kernel
    B_TILE_NB,        // neighbour index of the batched hopping kernels
    B_SAP_LOCAL,      // block-local (shared-memory) index of the SAP kernel
    B_SAP_GLOBAL,     // lattice index of the SAP kernel
    B_LEX,            // lexicographic site of the clover and force kernels
    B_LAYOUT          // natural / internal index of the layout kernels
};
#ifdef LQ_BOUNDS
static __device__ unsigned int lq_bounds_count_tu;
static __device__ unsigned int lq_bounds_first_tu;
__device__ __forceinline__ long long lq_idx_checked(long long i, long long n, unsigned code)
{
    if (i >= 0 && i < n) return i;
    if (atomicAdd(&lq_bounds_count_tu, 1u) == 0u) lq_bounds_first_tu = code;
    return 0;
}
#define LQ_IDX(i, n, code) ::lq::lq_idx_checked((long long)(i), (long long)(n), (code))
// host: every translation unit registers a reader of its flags
void bounds_register(unsigned (*read_clear)(unsigned *first));
#if !defined(__CUDA_ARCH__)
static unsigned lq_bounds_read_clear_tu(unsigned *first)
{
    unsigned n = 0, f = 0, z = 0;
    cudaMemcpyFromSymbol(&n, lq_bounds_count_tu, sizeof n);
    cudaMemcpyFromSymbol(&f, lq_bounds_first_tu, sizeof f);
    cudaMemcpyToSymbol(lq_bounds_count_tu, &z, sizeof z);
    cudaMemcpyToSymbol(lq_bounds_first_tu, &z, sizeof z);
    *first = f;
    return n;
}
static const int lq_bounds_registered_tu = (bounds_register(&lq_bounds_read_clear_tu), 0);
#endif
#else
#define LQ_IDX(i, n, code) (i)
#endif

// ---------------------------------------------------------------------------
// double-float ("df64") arithmetic: an unevaluated sum hi + lo of two floats,
// |lo| <= ulp(hi)/2, carrying about 48 significand bits.  GB300 executes FP32
// at 64 times its FP64 rate, so FP64-accurate work runs faster in this form.
// Built from the error-free transformations of Knuth (TwoSum), Dekker 1971
// (Fast2Sum, and the double-length add/multiply built on them) and the FMA
// form of the exact product (p = a*b, e = fma(a, b, -p)).  The explicit _rn
// intrinsics keep the compiler from contracting or reordering these steps.
// ---------------------------------------------------------------------------
struct df64 {
    float hi, lo;
    __host__ __device__ df64() {}
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ df64(double d)
    {
        hi = (float)d;
        lo = (float)(d - (double)hi);
    }
};

// s + e == a + b exactly, for |a| >= |b| (Dekker)
__device__ __forceinline__ df64 df_fast2sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// s + e == a + b exactly (Knuth)
__device__ __forceinline__ df64 df_2sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return df64(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
// p + e == a * b exactly (FMA)
__device__ __forceinline__ df64 df_2prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return df64(p, __fmaf_rn(a, b, -p));
}
__device__ __forceinline__ df64 operator+(df64 a, df64 b)
{
    df64 s = df_2sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return df_fast2sum(s.hi, s.lo);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b)
{
    df64 p = df_2prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return df_fast2sum(p.hi, p.lo);
}
// a * b + c with one rounding of the combined low parts
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c)
{
    df64 p = df_2prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    df64 s = df_2sum(p.hi, c.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(p.lo, c.lo));
    return df_fast2sum(s.hi, s.lo);
}
// keep the float and double fma overloads visible next to the df64 one, so
// that templates never route FP64 or FP32 arithmetic through df64
using ::fma;

__device__ __forceinline__ df64 operator/(df64 a, df64 b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const df64 r = a - b * df64(q1, 0.0f);
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return df_fast2sum(q1, q2);
}
__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
// Conversions between double and df64 / float with integer bit operations
// (GB300's FP64 pipe, which float <-> double conversions and double adds
// use, runs at 1/64 of the FP32 rate, so field import and export would
// otherwise be bound by it).  For a normal double d with exponent e and 53-bit
// significand m: hi = m's top 24 bits rounded to nearest even, and the
// remainder m - hi, an integer R with |R| <= 2^28 in units of 2^(e-52), gives
// lo = RN(R) 2^(e-52) -- the same values as hi = (float)d, lo = (float)(d - hi).
// Zero, subnormal, very small or very large magnitudes and non-finite values
// take the FP64 route, kept out of line: inlined, the compiler evaluates it for
// every value and selects (four FP64-pipe operations per double, which then
// bound the link import).
static __device__ __noinline__ df64 df_split_rare(double d) { return df64(d); }
static __device__ __noinline__ double f2d_rare(float x) { return (double)x; }

__device__ __forceinline__ df64 df_split(double d)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7FF) - 1023;
    if (e < -74 || e > 126) return df_split_rare(d);
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    unsigned q = (unsigned)(m >> 29);             // 2^23 <= q < 2^24
    int R = (int)(m & 0x1FFFFFFFull);             // 0 <= R < 2^29
    if (R > (1 << 28) || (R == (1 << 28) && (q & 1u))) {
        q += 1;
        R -= 1 << 29;
    }
    int eh = e;
    if (q == (1u << 24)) {
        q >>= 1;
        eh += 1;
    }
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const float hi = __uint_as_float(sign | ((unsigned)(eh + 127) << 23) | (q & 0x7FFFFFu));
    const float scale = __uint_as_float((unsigned)(e - 52 + 127) << 23);   // 2^(e-52), normal for e >= -74
    return df64(hi, __int2float_rn(sign ? -R : R) * scale);
}
// (float)d, rounded to nearest even
__device__ __forceinline__ float d2f_bits(double d) { return df_split(d).hi; }
// (double)x, exact
__device__ __forceinline__ double f2d_bits(float x)
{
    const unsigned b = __float_as_uint(x);
    const unsigned E = (b >> 23) & 0xFFu;
    if (E == 0u && (b & 0x7FFFFFu) == 0u) return __longlong_as_double((long long)((unsigned long long)b << 32));
    if (E == 0u || E == 0xFFu) return f2d_rare(x);
    return __longlong_as_double((long long)(((unsigned long long)(b & 0x80000000u) << 32) |
                                            ((unsigned long long)(E + 896u) << 52) |
                                            ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}
// hi + lo as a double (one FP64 add)
__device__ __forceinline__ double df_join(float hi, float lo) { return f2d_bits(hi) + f2d_bits(lo); }

__device__ __forceinline__ bool df_positive(df64 a) { return a.hi > 0.0f || (a.hi == 0.0f && a.lo > 0.0f); }
__device__ __forceinline__ double df_to_double(df64 a) { return (double)a.hi + (double)a.lo; }
// hi + lo rounded to FP32: one float add, which rounds the exact sum once
__device__ __forceinline__ float df_to_float(df64 a) { return a.hi + a.lo; }

// ---------------------------------------------------------------------------
// Lazily normalised df64 sums (compensated dot product in the manner of Ogita,
// Rump and Oishi's Dot2): each term a * b is split exactly into p + e (the
// FMA product error plus the two cross terms of the low parts), p enters the
// running high part through TwoSum, and every error term is gathered in the
// low part without renormalising.  A sum of n terms then costs 12 FP32
// instructions per term instead of the 15 of a normalised df64 fma, and is
// renormalised once (dl_norm, TwoSum, exact for any high/low ordering).  The
// low part grows to at most a few units in the last place of the high part,
// so the result keeps the df64 accuracy for the short sums of a hopping term.
// ---------------------------------------------------------------------------
__device__ __forceinline__ df64 dl_prod(df64 a, df64 b)   // a * b, unnormalised
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    return df64(p, __fmaf_rn(a.lo, b.hi, e));
}
__device__ __forceinline__ void dl_add(df64 &s, df64 x)   // s += x
{
    const float t = __fadd_rn(s.hi, x.hi);
    const float bb = __fsub_rn(t, s.hi);
    const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bb)), __fsub_rn(x.hi, bb));
    s.hi = t;
    s.lo = __fadd_rn(s.lo, __fadd_rn(err, x.lo));
}
__device__ __forceinline__ void dl_fma(df64 &s, df64 a, df64 b)   // s += a * b
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float t = __fadd_rn(s.hi, p);
    const float bb = __fsub_rn(t, s.hi);
    const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    s.hi = t;
    s.lo = __fadd_rn(s.lo, __fadd_rn(err, e));
}
__device__ __forceinline__ df64 dl_norm(df64 s) { return df_2sum(s.hi, s.lo); }
__device__ __forceinline__ df64 dl_neg(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 dl_scale2(df64 a, float f) { return df64(f * a.hi, f * a.lo); }   // f a power of 2

// ---------------------------------------------------------------------------
// complex arithmetic
// ---------------------------------------------------------------------------
template <typename R>
struct cx {
    R re, im;
};

// complex forms of the lazily normalised df64 sums above
__device__ __forceinline__ cx<df64> dl_cmul(cx<df64> a, cx<df64> b)   // a * b
{
    cx<df64> s = {dl_prod(a.re, b.re), dl_prod(a.re, b.im)};
    dl_fma(s.re, dl_neg(a.im), b.im);
    dl_fma(s.im, a.im, b.re);
    return s;
}
__device__ __forceinline__ void dl_cfma(cx<df64> &s, cx<df64> a, cx<df64> b)   // s += a * b
{
    dl_fma(s.re, a.re, b.re);
    dl_fma(s.re, dl_neg(a.im), b.im);
    dl_fma(s.im, a.re, b.im);
    dl_fma(s.im, a.im, b.re);
}
__device__ __forceinline__ void dl_cfmac(cx<df64> &s, cx<df64> a, cx<df64> b)   // s += conj(a) * b
{
    dl_fma(s.re, a.re, b.re);
    dl_fma(s.re, a.im, b.im);
    dl_fma(s.im, a.re, b.im);
    dl_fma(s.im, dl_neg(a.im), b.re);
}
__device__ __forceinline__ void dl_cadd(cx<df64> &s, cx<df64> x)
{
    dl_add(s.re, x.re);
    dl_add(s.im, x.im);
}
__device__ __forceinline__ cx<df64> dl_cnorm(cx<df64> s) { return {dl_norm(s.re), dl_norm(s.im)}; }

template <typename R>
__device__ __forceinline__ cx<R> mk(R a, R b) { return cx<R>{a, b}; }
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a) { return {-a.re, -a.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }
// a * b
template <typename R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b)
{
    return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
// conj(a) * b
template <typename R>
__device__ __forceinline__ cx<R> cmulc(cx<R> a, cx<R> b)
{
    return {fma(a.re, b.re, a.im * b.im), fma(a.re, b.im, -a.im * b.re)};
}
// acc + a * b
template <typename R>
__device__ __forceinline__ cx<R> cfma(cx<R> a, cx<R> b, cx<R> acc)
{
    return {fma(a.re, b.re, fma(-a.im, b.im, acc.re)), fma(a.re, b.im, fma(a.im, b.re, acc.im))};
}
// acc + conj(a) * b
template <typename R>
__device__ __forceinline__ cx<R> cfmac(cx<R> a, cx<R> b, cx<R> acc)
{
    return {fma(a.re, b.re, fma(a.im, b.im, acc.re)), fma(a.re, b.im, fma(-a.im, b.re, acc.im))};
}
// i * a, -i * a
template <typename R>
__device__ __forceinline__ cx<R> ti(cx<R> a) { return {-a.im, a.re}; }
template <typename R>
__device__ __forceinline__ cx<R> tmi(cx<R> a) { return {a.im, -a.re}; }
template <typename R>
__device__ __forceinline__ cx<R> cconj(cx<R> a) { return {a.re, -a.im}; }

// ---------------------------------------------------------------------------
// storage traits: 16-byte vectors per precision
// ---------------------------------------------------------------------------
template <typename R>
struct St;

template <>
struct St<double> {
    typedef double2 vec;               // one complex per vector
    static constexpr int SPINOR_VECS = 12;
    static constexpr int CLOVER_VECS = 18;  // per 6x6 block
    static constexpr int LINK_VECS = 9;     // 18-real links
};

template <>
struct St<float> {
    typedef float4 vec;                // two complexes per vector
    static constexpr int SPINOR_VECS = 6;
    static constexpr int CLOVER_VECS = 9;
    static constexpr int LINK_VECS = 3;     // 12-real compressed links
};

// one df64 complex (or a pair of df64 reals) in 16 bytes: the df64 layouts
// mirror the FP64 ones vector for vector
struct __align__(16) df2 {
    float rh, rl, ih, il;
};

template <>
struct St<df64> {
    typedef df2 vec;                   // one complex per vector
    static constexpr int SPINOR_VECS = 12;
    static constexpr int CLOVER_VECS = 18;
    static constexpr int LINK_VECS = 9;     // 18-real links
};

template <typename R>
__host__ __device__ constexpr long long spinor_elems(long long stride)
{
    return (long long)St<R>::SPINOR_VECS * stride;   // in vectors
}

// read-only cached vector loads
__device__ __forceinline__ double2 ldg(const double2 *p) { return __ldg(p); }
__device__ __forceinline__ float4 ldg(const float4 *p) { return __ldg(p); }
// A float4 of data that a launch reads once (links, clover blocks of the
// single-right-hand-side hopping kernels): loaded without allocating in L1, so
// that L1 keeps the neighbour spinors that eight sites each read.  Measured on
// GB300: FP32 K1 and K2 move from 0.93 to 0.95 (32^3 x 64) and from 0.97 to
// 1.02 (48^3 x 96) of the copy bandwidth; the batched kernels, whose tiles
// share links through L1, keep cached loads.
struct __align__(16) F4S {
    float4 v;
};
__device__ __forceinline__ float4 ldg(const F4S *p)
{
    float4 r;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
        : "l"(p));
    return r;
}
__device__ __forceinline__ df2 ldg(const df2 *p)
{
    const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    return df2{t.x, t.y, t.z, t.w};
}
__device__ __forceinline__ cx<df64> df2_cx(df2 t) { return {df64(t.rh, t.rl), df64(t.ih, t.il)}; }
__device__ __forceinline__ df2 cx_df2(cx<df64> v) { return df2{v.re.hi, v.re.lo, v.im.hi, v.im.lo}; }

__device__ __forceinline__ void load_spinor(const df2 *__restrict__ p, long long stride, long long s,
                                            cx<df64> v[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) v[c] = df2_cx(ldg(p + c * stride + s));
}
__device__ __forceinline__ void load_spinor_rw(const df2 *p, long long stride, long long s, cx<df64> v[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) v[c] = df2_cx(p[c * stride + s]);
}
__device__ __forceinline__ void store_spinor(df2 *p, long long stride, long long s, const cx<df64> v[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) p[c * stride + s] = cx_df2(v[c]);
}
__device__ __forceinline__ void load_link(const df2 *__restrict__ U, long long stride, int mu, long long s,
                                          cx<df64> m[9])
{
#pragma unroll
    for (int k = 0; k < 9; k++) m[k] = df2_cx(ldg(U + (mu * 9 + k) * stride + s));
}
__device__ __forceinline__ void load_block(const df2 *__restrict__ C, long long stride, int blk, long long s,
                                           df64 r[36])
{
#pragma unroll
    for (int k = 0; k < 18; k++) {
        const df2 t = ldg(C + (blk * 18 + k) * stride + s);
        r[2 * k] = df64(t.rh, t.rl);
        r[2 * k + 1] = df64(t.ih, t.il);
    }
}

__device__ __forceinline__ void load_spinor(const double2 *__restrict__ p, long long stride,
                                            long long s, cx<double> v[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) {
        double2 t = ldg(p + c * stride + s);
        v[c] = {t.x, t.y};
    }
}
__device__ __forceinline__ void load_spinor(const float4 *__restrict__ p, long long stride,
                                            long long s, cx<float> v[12])
{
#pragma unroll
    for (int k = 0; k < 6; k++) {
        float4 t = ldg(p + k * stride + s);
        v[2 * k] = {t.x, t.y};
        v[2 * k + 1] = {t.z, t.w};
    }
}
// plain (coherent) loads, for vectors the same kernel also writes
__device__ __forceinline__ void load_spinor_rw(const double2 *p, long long stride, long long s,
                                               cx<double> v[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) {
        double2 t = p[c * stride + s];
        v[c] = {t.x, t.y};
    }
}
__device__ __forceinline__ void load_spinor_rw(const float4 *p, long long stride, long long s,
                                               cx<float> v[12])
{
#pragma unroll
    for (int k = 0; k < 6; k++) {
        float4 t = p[k * stride + s];
        v[2 * k] = {t.x, t.y};
        v[2 * k + 1] = {t.z, t.w};
    }
}
__device__ __forceinline__ void store_spinor(double2 *p, long long stride, long long s,
                                             const cx<double> v[12])
{
#pragma unroll
    for (int c = 0; c < 12; c++) p[c * stride + s] = make_double2(v[c].re, v[c].im);
}
__device__ __forceinline__ void store_spinor(float4 *p, long long stride, long long s,
                                             const cx<float> v[12])
{
#pragma unroll
    for (int k = 0; k < 6; k++)
        p[k * stride + s] = make_float4(v[2 * k].re, v[2 * k].im, v[2 * k + 1].re, v[2 * k + 1].im);
}

// ---------------------------------------------------------------------------
// links
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_link(const double2 *__restrict__ U, long long stride, int mu,
                                          long long s, cx<double> m[9])
{
#pragma unroll
    for (int k = 0; k < 9; k++) {
        double2 t = ldg(U + (mu * 9 + k) * stride + s);
        m[k] = {t.x, t.y};
    }
}
template <typename P>   // const float4 (cached) or const F4S (read once)
__device__ __forceinline__ void load_link_f(const P *__restrict__ U, long long stride, int mu, long long s,
                                            cx<float> m[9])
{
#pragma unroll
    for (int k = 0; k < 3; k++) {
        float4 t = ldg(U + (mu * 3 + k) * stride + s);
        m[2 * k] = {t.x, t.y};
        m[2 * k + 1] = {t.z, t.w};
    }
    // SU(3): third row = conj(row0 x row1)
    m[6] = cconj(cmul(m[1], m[5]) - cmul(m[2], m[4]));
    m[7] = cconj(cmul(m[2], m[3]) - cmul(m[0], m[5]));
    m[8] = cconj(cmul(m[0], m[4]) - cmul(m[1], m[3]));
}
__device__ __forceinline__ void load_link(const float4 *__restrict__ U, long long stride, int mu, long long s,
                                          cx<float> m[9])
{
    load_link_f(U, stride, mu, s, m);
}
__device__ __forceinline__ void load_link(const F4S *__restrict__ U, long long stride, int mu, long long s,
                                          cx<float> m[9])
{
    load_link_f(U, stride, mu, s, m);
}

// ---------------------------------------------------------------------------
// clover blocks (packed Hermitian 6x6)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_block(const double2 *__restrict__ C, long long stride, int blk,
                                           long long s, double r[36])
{
#pragma unroll
    for (int k = 0; k < 18; k++) {
        double2 t = ldg(C + (blk * 18 + k) * stride + s);
        r[2 * k] = t.x;
        r[2 * k + 1] = t.y;
    }
}
template <typename P>
__device__ __forceinline__ void load_block_f(const P *__restrict__ C, long long stride, int blk, long long s,
                                             float r[36])
{
#pragma unroll
    for (int k = 0; k < 9; k++) {
        float4 t = ldg(C + (blk * 9 + k) * stride + s);
        r[4 * k] = t.x;
        r[4 * k + 1] = t.y;
        r[4 * k + 2] = t.z;
        r[4 * k + 3] = t.w;
    }
}
__device__ __forceinline__ void load_block(const float4 *__restrict__ C, long long stride, int blk, long long s,
                                           float r[36])
{
    load_block_f(C, stride, blk, s, r);
}
__device__ __forceinline__ void load_block(const F4S *__restrict__ C, long long stride, int blk, long long s,
                                           float r[36])
{
    load_block_f(C, stride, blk, s, r);
}

// index of the packed strictly-lower entry (i, j), i > j
__host__ __device__ constexpr int tri(int i, int j) { return i * (i - 1) / 2 + j; }

// y = A x for a packed Hermitian 6x6 block A
template <typename R>
__device__ __forceinline__ void herm6_apply(const R a[36], const cx<R> x[6], cx<R> y[6])
{
#pragma unroll
    for (int i = 0; i < 6; i++) y[i] = a[i] * x[i];
#pragma unroll
    for (int i = 1; i < 6; i++)
#pragma unroll
        for (int j = 0; j < i; j++) {
            const int k = 6 + 2 * tri(i, j);
            cx<R> l = {a[k], a[k + 1]};
            y[i] = cfma(l, x[j], y[i]);    // lower entry
            y[j] = cfmac(l, x[i], y[j]);   // its conjugate above the diagonal
        }
}

// y = C x for a full site (both blocks); x, y are 12-component spinors
template <typename R, typename V>
__device__ __forceinline__ void clover_apply(const V *__restrict__ C, long long stride, long long s,
                                             const cx<R> x[12], cx<R> y[12])
{
#pragma unroll
    for (int blk = 0; blk < 2; blk++) {
        R a[36];
        load_block(C, stride, blk, s, a);
        herm6_apply<R>(a, x + 6 * blk, y + 6 * blk);
    }
}

// ---------------------------------------------------------------------------
// site coordinates from the checkerboard index
// ---------------------------------------------------------------------------
struct Coords {
    int x, y, z, t;
    long long row;   // y + Ly*(z + Lz*t)
};

__device__ __forceinline__ Coords cb_coords(const Geom &g, long long s, int parity)
{
    Coords c;
    long long row = s / g.Lxh;
    int xh = (int)(s - row * g.Lxh);
    c.row = row;
    c.y = (int)(row % g.L[1]);
    long long r2 = row / g.L[1];
    c.z = (int)(r2 % g.L[2]);
    c.t = (int)(r2 / g.L[2]);
    c.x = 2 * xh + ((c.y + c.z + c.t + parity) & 1);
    return c;
}

// ---------------------------------------------------------------------------
// launch bookkeeping and errors (host)
// ---------------------------------------------------------------------------
struct Counters {
    long long launches = 0;
    double bytes = 0.0;
};

}  // namespace lq
