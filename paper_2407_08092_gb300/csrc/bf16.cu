// BF16 fields: conversion to and from the other internal precisions and the
// natural layout, gamma5, axpby, and the BF16 copy of the 12-real links.
// Arithmetic is FP32; stores round to nearest BF16.  Only the sites below V/2
// are written, so the zero padding of a field stays zero.
#include <type_traits>

#include "bf16.cuh"
#include "lq_kernels.h"

namespace lq {

static inline unsigned nb256(long long n) { return (unsigned)((n + 255) / 256); }

__device__ __forceinline__ void to_f(const cx<double> a[12], cx<float> v[12])
{
#pragma unroll
    for (int k = 0; k < 12; k++) v[k] = {(float)a[k].re, (float)a[k].im};
}
__device__ __forceinline__ void to_f(const cx<df64> a[12], cx<float> v[12])
{
#pragma unroll
    for (int k = 0; k < 12; k++) v[k] = {df_to_float(a[k].re), df_to_float(a[k].im)};
}

// any internal precision -> BF16
template <typename V, typename R>
__global__ void to_bf16_kernel(Geom g, const V *__restrict__ in, BfS4 *out)
{
    const long long s = blockIdx.x * 256LL + threadIdx.x;
    if (s >= g.Vh) return;
    cx<R> a[12];
    load_spinor(in, g.stride, s, a);
    cx<float> v[12];
    if constexpr (std::is_same<R, float>::value) {
#pragma unroll
        for (int k = 0; k < 12; k++) v[k] = a[k];
    } else {
        to_f(a, v);
    }
    store_spinor(out, g.stride, s, v);
}

// BF16 -> FP64, FP32 or df64 (exact: a BF16 value is a float)
__global__ void bf16_to_d_kernel(Geom g, const BfS4 *__restrict__ in, double2 *out)
{
    const long long s = blockIdx.x * 256LL + threadIdx.x;
    if (s >= g.Vh) return;
    cx<float> v[12];
    load_spinor(in, g.stride, s, v);
    cx<double> d[12];
#pragma unroll
    for (int k = 0; k < 12; k++) d[k] = {(double)v[k].re, (double)v[k].im};
    store_spinor(out, g.stride, s, d);
}
__global__ void bf16_to_f_kernel(Geom g, const BfS4 *__restrict__ in, float4 *out)
{
    const long long s = blockIdx.x * 256LL + threadIdx.x;
    if (s >= g.Vh) return;
    cx<float> v[12];
    load_spinor(in, g.stride, s, v);
    store_spinor(out, g.stride, s, v);
}
__global__ void bf16_to_df_kernel(Geom g, const BfS4 *__restrict__ in, df2 *out)
{
    const long long s = blockIdx.x * 256LL + threadIdx.x;
    if (s >= g.Vh) return;
    cx<float> v[12];
    load_spinor(in, g.stride, s, v);
    cx<df64> d[12];
#pragma unroll
    for (int k = 0; k < 12; k++) d[k] = {df64(v[k].re, 0.0f), df64(v[k].im, 0.0f)};
    store_spinor(out, g.stride, s, d);
}

// natural [Vh][12] c128 <-> BF16 field of one parity
__global__ void bf16_import_half_kernel(Geom g, const double2 *__restrict__ nat, BfS4 *f)
{
    const long long s = blockIdx.x * 256LL + threadIdx.x;
    if (s >= g.Vh) return;
    cx<float> v[12];
#pragma unroll
    for (int k = 0; k < 12; k++) {
        const double2 t = nat[s * 12 + k];
        v[k] = {(float)t.x, (float)t.y};
    }
    store_spinor(f, g.stride, s, v);
}
__global__ void bf16_export_half_kernel(Geom g, const BfS4 *__restrict__ f, double2 *nat)
{
    const long long s = blockIdx.x * 256LL + threadIdx.x;
    if (s >= g.Vh) return;
    cx<float> v[12];
    load_spinor(f, g.stride, s, v);
#pragma unroll
    for (int k = 0; k < 12; k++) nat[s * 12 + k] = make_double2((double)v[k].re, (double)v[k].im);
}

// out = g5 in: spins 2, 3 (components 6..11) negated
__global__ void bf16_gamma5_kernel(Geom g, const BfS4 *in, BfS4 *out)
{
    const long long s = blockIdx.x * 256LL + threadIdx.x;
    if (s >= g.Vh) return;
    cx<float> v[12];
    load_spinor_rw(in, g.stride, s, v);
#pragma unroll
    for (int k = 6; k < 12; k++) v[k] = -v[k];
    store_spinor(out, g.stride, s, v);
}

// y = a x + b y over nfields consecutive fields (complex a, b)
__global__ void bf16_axpby_kernel(Geom g, int nfields, float ar, float ai, const BfS4 *x, float br, float bi,
                                  BfS4 *y)
{
    const long long id = blockIdx.x * 256LL + threadIdx.x;
    if (id >= g.Vh * nfields) return;
    const long long f = id / g.Vh, s = id - f * g.Vh;
    const long long o = f * 3 * g.stride;
    cx<float> xv[12], yv[12];
    load_spinor_rw(x + o, g.stride, s, xv);
    load_spinor_rw(y + o, g.stride, s, yv);
    const cx<float> a = {ar, ai}, b = {br, bi};
#pragma unroll
    for (int k = 0; k < 12; k++) yv[k] = cmul(a, xv[k]) + cmul(b, yv[k]);
    store_spinor(y + o, g.stride, s, yv);
}

// FP32 12-real links [4][3][stride] float4 -> BF16 [4][3][stride] BfL2
__global__ void links_to_bf16_kernel(Geom g, const float4 *__restrict__ U32, BfL2 *U16)
{
    const long long id = blockIdx.x * 256LL + threadIdx.x;
    if (id >= 12 * g.Vh) return;
    const long long v = id / g.Vh, s = id - v * g.Vh;   // v = mu * 3 + k
    const float4 t = U32[v * g.stride + s];
    BfL2 o;
    o.c[0] = __float22bfloat162_rn(make_float2(t.x, t.y));
    o.c[1] = __float22bfloat162_rn(make_float2(t.z, t.w));
    U16[v * g.stride + s] = o;
}

void bf16_convert(const Exec &e, int from, const void *in, int to, void *out)
{
    const double other = (from == P16 ? to : from) == P32 ? 96.0 : 192.0;
    Launch L_(e, K_LAYOUT, (double)e.g.Vh * (48.0 + other));
    const unsigned b = nb256(e.g.Vh);
    if (to == P16) {
        if (from == P64) to_bf16_kernel<double2, double><<<b, 256, 0, e.st>>>(e.g, (const double2 *)in, (BfS4 *)out);
        else if (from == P32) to_bf16_kernel<float4, float><<<b, 256, 0, e.st>>>(e.g, (const float4 *)in, (BfS4 *)out);
        else if (from == PDF) to_bf16_kernel<df2, df64><<<b, 256, 0, e.st>>>(e.g, (const df2 *)in, (BfS4 *)out);
        else copy_bytes(e, in, out, spinor_bytes(e.g, P16));
    } else if (to == P64) {
        bf16_to_d_kernel<<<b, 256, 0, e.st>>>(e.g, (const BfS4 *)in, (double2 *)out);
    } else if (to == P32) {
        bf16_to_f_kernel<<<b, 256, 0, e.st>>>(e.g, (const BfS4 *)in, (float4 *)out);
    } else {
        bf16_to_df_kernel<<<b, 256, 0, e.st>>>(e.g, (const BfS4 *)in, (df2 *)out);
    }
}

void bf16_import_half(const Exec &e, const void *nat, void *f)
{
    Launch L_(e, K_LAYOUT, (double)e.g.Vh * (192 + 48));
    bf16_import_half_kernel<<<nb256(e.g.Vh), 256, 0, e.st>>>(e.g, (const double2 *)nat, (BfS4 *)f);
}

void bf16_export_half(const Exec &e, const void *f, void *nat)
{
    Launch L_(e, K_LAYOUT, (double)e.g.Vh * (192 + 48));
    bf16_export_half_kernel<<<nb256(e.g.Vh), 256, 0, e.st>>>(e.g, (const BfS4 *)f, (double2 *)nat);
}

void bf16_gamma5(const Exec &e, const void *in, void *out)
{
    Launch L_(e, K_LAYOUT, (double)e.g.Vh * 2 * 48);
    bf16_gamma5_kernel<<<nb256(e.g.Vh), 256, 0, e.st>>>(e.g, (const BfS4 *)in, (BfS4 *)out);
}

void bf16_axpby(const Exec &e, double ar, double ai, const void *x, double br, double bi, void *y, int nfields)
{
    Launch L_(e, K_AXPY_F32, 3.0 * nfields * e.g.Vh * 48, (double)nfields * e.g.Vh * 12 * 14);
    bf16_axpby_kernel<<<nb256(e.g.Vh * nfields), 256, 0, e.st>>>(e.g, nfields, (float)ar, (float)ai,
                                                                  (const BfS4 *)x, (float)br, (float)bi, (BfS4 *)y);
}

void links_to_bf16(const Exec &e, const void *U32, void *U16)
{
    Launch L_(e, K_LAYOUT, (double)e.g.Vh * 4 * (48 + 24));
    links_to_bf16_kernel<<<nb256(12 * e.g.Vh), 256, 0, e.st>>>(e.g, (const float4 *)U32, (BfL2 *)U16);
}

}  // namespace lq
