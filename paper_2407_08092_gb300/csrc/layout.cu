// Layout kernels: natural complex-double fields <-> internal checkerboarded
// structure-of-arrays fields, precision conversion and the gamma_5 multiply.
// (Sec. 2.4.5: odd-even reordering; the internal order is even sites first,
// each parity in lexicographic order.)
#include "lq_kernels.h"

namespace lq {

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// one thread per (site, mu): U_nat[lex][mu][9] -> U64[p][mu][9][stride], U32[p][mu][3][stride]
__device__ __forceinline__ df2 to_df2(double2 v)
{
    const df64 r(v.x), i(v.y);
    return df2{r.hi, r.lo, i.hi, i.lo};
}
__device__ __forceinline__ double2 from_df2(df2 v)
{
    return make_double2((double)v.rh + (double)v.rl, (double)v.ih + (double)v.il);
}

__global__ void import_links_kernel(Geom g, const double2 *__restrict__ U, double2 *U64e, double2 *U64o,
                                    float4 *U32e, float4 *U32o, df2 *Udfe, df2 *Udfo)
{
    long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= 4 * g.V) return;
    const long long lex = id >> 2;
    const int mu = (int)(id & 3);
    long long r = lex;
    int c0 = (int)(r % g.L[0]); r /= g.L[0];
    int c1 = (int)(r % g.L[1]); r /= g.L[1];
    int c2 = (int)(r % g.L[2]); int c3 = (int)(r / g.L[2]);
    const int parity = (c0 + c1 + c2 + c3) & 1;
    const long long cb = lex >> 1;
    double2 m[9];
#pragma unroll
    for (int k = 0; k < 9; k++) m[k] = __ldg(U + id * 9 + k);
    double2 *d = parity ? U64o : U64e;
#pragma unroll
    for (int k = 0; k < 9; k++) d[(mu * 9 + k) * g.stride + cb] = m[k];
    float4 *f = parity ? U32o : U32e;
#pragma unroll
    for (int k = 0; k < 3; k++)
        f[(mu * 3 + k) * g.stride + cb] = make_float4((float)m[2 * k].x, (float)m[2 * k].y,
                                                       (float)m[2 * k + 1].x, (float)m[2 * k + 1].y);
    df2 *q = parity ? Udfo : Udfe;
#pragma unroll
    for (int k = 0; k < 9; k++) q[(mu * 9 + k) * g.stride + cb] = to_df2(m[k]);
}

void import_links(const Exec &e, const void *U_nat, void *U64[2], void *U32[2], void *Udf[2])
{
    Launch L_(e, K_LAYOUT, (double)e.g.V * 4 * (144 + 144 + 48 + 144));
    import_links_kernel<<<nblk(4 * e.g.V, 256), 256, 0, e.st>>>(
        e.g, (const double2 *)U_nat, (double2 *)U64[0], (double2 *)U64[1], (float4 *)U32[0], (float4 *)U32[1],
        (df2 *)Udf[0], (df2 *)Udf[1]);
}

// ---- spinors ----------------------------------------------------------------
// natural [n][12] c128 rows -> internal component-major field
template <typename R>
__global__ void import_half_kernel(Geom g, const double2 *__restrict__ nat, typename St<R>::vec *f);

template <>
__global__ void import_half_kernel<double>(Geom g, const double2 *__restrict__ nat, double2 *f)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int c = 0; c < 12; c++) f[c * g.stride + s] = __ldg(nat + s * 12 + c);
}
template <>
__global__ void import_half_kernel<float>(Geom g, const double2 *__restrict__ nat, float4 *f)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        double2 a = __ldg(nat + s * 12 + 2 * k), b = __ldg(nat + s * 12 + 2 * k + 1);
        f[k * g.stride + s] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
    }
}

template <typename R>
__global__ void export_half_kernel(Geom g, const typename St<R>::vec *__restrict__ f, double2 *nat);

template <>
__global__ void export_half_kernel<double>(Geom g, const double2 *__restrict__ f, double2 *nat)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int c = 0; c < 12; c++) nat[s * 12 + c] = __ldg(f + c * g.stride + s);
}
template <>
__global__ void export_half_kernel<float>(Geom g, const float4 *__restrict__ f, double2 *nat)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        float4 t = __ldg(f + k * g.stride + s);
        nat[s * 12 + 2 * k] = make_double2(t.x, t.y);
        nat[s * 12 + 2 * k + 1] = make_double2(t.z, t.w);
    }
}

__global__ void import_half_df_kernel(Geom g, const double2 *__restrict__ nat, df2 *f)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int c = 0; c < 12; c++) f[c * g.stride + s] = to_df2(__ldg(nat + s * 12 + c));
}
__global__ void export_half_df_kernel(Geom g, const df2 *__restrict__ f, double2 *nat)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int c = 0; c < 12; c++) nat[s * 12 + c] = from_df2(ldg(f + c * g.stride + s));
}

__device__ __forceinline__ int lex_parity(const Geom &g, long long lex)
{
    long long r = lex;
    int c0 = (int)(r % g.L[0]); r /= g.L[0];
    int c1 = (int)(r % g.L[1]); r /= g.L[1];
    int c2 = (int)(r % g.L[2]); int c3 = (int)(r / g.L[2]);
    return (c0 + c1 + c2 + c3) & 1;
}

template <typename R>
__global__ void import_full_kernel(Geom g, const double2 *__restrict__ nat, typename St<R>::vec *fe,
                                   typename St<R>::vec *fo)
{
    long long lex = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (lex >= g.V) return;
    const long long cb = lex >> 1;
    typename St<R>::vec *f = lex_parity(g, lex) ? fo : fe;
    if constexpr (sizeof(R) == 8) {
#pragma unroll
        for (int c = 0; c < 12; c++) f[c * g.stride + cb] = __ldg(nat + lex * 12 + c);
    } else {
#pragma unroll
        for (int k = 0; k < 6; k++) {
            double2 a = __ldg(nat + lex * 12 + 2 * k), b = __ldg(nat + lex * 12 + 2 * k + 1);
            f[k * g.stride + cb] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
        }
    }
}

template <typename R>
__global__ void export_full_kernel(Geom g, const typename St<R>::vec *__restrict__ fe,
                                   const typename St<R>::vec *__restrict__ fo, double2 *nat)
{
    long long lex = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (lex >= g.V) return;
    const long long cb = lex >> 1;
    const typename St<R>::vec *f = lex_parity(g, lex) ? fo : fe;
    if constexpr (sizeof(R) == 8) {
#pragma unroll
        for (int c = 0; c < 12; c++) nat[lex * 12 + c] = __ldg(f + c * g.stride + cb);
    } else {
#pragma unroll
        for (int k = 0; k < 6; k++) {
            float4 t = __ldg(f + k * g.stride + cb);
            nat[lex * 12 + 2 * k] = make_double2(t.x, t.y);
            nat[lex * 12 + 2 * k + 1] = make_double2(t.z, t.w);
        }
    }
}

__global__ void import_full_df_kernel(Geom g, const double2 *__restrict__ nat, df2 *fe, df2 *fo)
{
    long long lex = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (lex >= g.V) return;
    const long long cb = lex >> 1;
    df2 *f = lex_parity(g, lex) ? fo : fe;
#pragma unroll
    for (int c = 0; c < 12; c++) f[c * g.stride + cb] = to_df2(__ldg(nat + lex * 12 + c));
}
__global__ void export_full_df_kernel(Geom g, const df2 *__restrict__ fe, const df2 *__restrict__ fo, double2 *nat)
{
    long long lex = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (lex >= g.V) return;
    const long long cb = lex >> 1;
    const df2 *f = lex_parity(g, lex) ? fo : fe;
#pragma unroll
    for (int c = 0; c < 12; c++) nat[lex * 12 + c] = from_df2(ldg(f + c * g.stride + cb));
}

void import_half(const Exec &e, int prec, const void *nat, void *f)
{
    if (prec == P16) {
        bf16_import_half(e, nat, f);
        return;
    }
    Launch L_(e, K_LAYOUT, (double)e.g.Vh * (192 + (prec == P32 ? 96 : 192)));
    if (prec == PDF) {
        import_half_df_kernel<<<nblk(e.g.Vh, 256), 256, 0, e.st>>>(e.g, (const double2 *)nat, (df2 *)f);
        return;
    }
    if (prec == P64)
        import_half_kernel<double><<<nblk(e.g.Vh, 256), 256, 0, e.st>>>(e.g, (const double2 *)nat, (double2 *)f);
    else
        import_half_kernel<float><<<nblk(e.g.Vh, 256), 256, 0, e.st>>>(e.g, (const double2 *)nat, (float4 *)f);
}

void export_half(const Exec &e, int prec, const void *f, void *nat)
{
    if (prec == P16) {
        bf16_export_half(e, f, nat);
        return;
    }
    Launch L_(e, K_LAYOUT, (double)e.g.Vh * (192 + (prec == P32 ? 96 : 192)));
    if (prec == PDF) {
        export_half_df_kernel<<<nblk(e.g.Vh, 256), 256, 0, e.st>>>(e.g, (const df2 *)f, (double2 *)nat);
        return;
    }
    if (prec == P64)
        export_half_kernel<double><<<nblk(e.g.Vh, 256), 256, 0, e.st>>>(e.g, (const double2 *)f, (double2 *)nat);
    else
        export_half_kernel<float><<<nblk(e.g.Vh, 256), 256, 0, e.st>>>(e.g, (const float4 *)f, (double2 *)nat);
}

void import_full(const Exec &e, int prec, const void *nat, void *fe, void *fo)
{
    Launch L_(e, K_LAYOUT, (double)e.g.V * (192 + (prec == P32 ? 96 : 192)));
    if (prec == PDF) {
        import_full_df_kernel<<<nblk(e.g.V, 256), 256, 0, e.st>>>(e.g, (const double2 *)nat, (df2 *)fe, (df2 *)fo);
        return;
    }
    if (prec == P64)
        import_full_kernel<double><<<nblk(e.g.V, 256), 256, 0, e.st>>>(e.g, (const double2 *)nat, (double2 *)fe,
                                                                       (double2 *)fo);
    else
        import_full_kernel<float><<<nblk(e.g.V, 256), 256, 0, e.st>>>(e.g, (const double2 *)nat, (float4 *)fe,
                                                                      (float4 *)fo);
}

void export_full(const Exec &e, int prec, const void *fe, const void *fo, void *nat)
{
    Launch L_(e, K_LAYOUT, (double)e.g.V * (192 + (prec == P32 ? 96 : 192)));
    if (prec == PDF) {
        export_full_df_kernel<<<nblk(e.g.V, 256), 256, 0, e.st>>>(e.g, (const df2 *)fe, (const df2 *)fo, (double2 *)nat);
        return;
    }
    if (prec == P64)
        export_full_kernel<double><<<nblk(e.g.V, 256), 256, 0, e.st>>>(e.g, (const double2 *)fe,
                                                                       (const double2 *)fo, (double2 *)nat);
    else
        export_full_kernel<float><<<nblk(e.g.V, 256), 256, 0, e.st>>>(e.g, (const float4 *)fe,
                                                                      (const float4 *)fo, (double2 *)nat);
}

// ---- conversion and gamma_5 -------------------------------------------------
__global__ void d2f_kernel(Geom g, const double2 *__restrict__ in, float4 *out)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        double2 a = __ldg(in + (2 * k) * g.stride + s), b = __ldg(in + (2 * k + 1) * g.stride + s);
        out[k * g.stride + s] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
    }
}
__global__ void f2d_kernel(Geom g, const float4 *__restrict__ in, double2 *out)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        float4 t = __ldg(in + k * g.stride + s);
        out[(2 * k) * g.stride + s] = make_double2(t.x, t.y);
        out[(2 * k + 1) * g.stride + s] = make_double2(t.z, t.w);
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
// (the last half of the vectors of a site in either precision)
__global__ void gamma5_d_kernel(Geom g, const double2 *in, double2 *out)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int k = 0; k < 12; k++) {
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
    for (int k = 0; k < 6; k++) {
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
    for (int k = 0; k < 12; k++) {
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
    Launch L_(e, K_LAYOUT, (double)e.g.Vh * 2 * (prec == P32 ? 96 : 192));
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
