// BF16 storage of spinors and links (FP32 arithmetic): the low-precision
// storage of the mixed-precision scheme.  Values are converted to FP32 on
// load and rounded to nearest on store (cuda_bf16 intrinsics); the clover
// blocks stay FP32.
//
//   spinor  [3][stride] BfS4: 4 complex per 16-byte vector (components 4k..4k+3)
//   links   [4 mu][3][stride] BfL2: rows 0 and 1 as 6 complex, 2 per 8-byte
//           vector (row 2 = conj(r0 x r1), as for the FP32 links)
//
// Bytes per site of one D_S apply: K1 576 (8 links x 24, the FP32 inverse
// 288, 2 spinors x 48), K2 624.
#pragma once

#include <cuda_bf16.h>

#include "lq_internal.cuh"

namespace lq {

struct __align__(16) BfS4 {
    __nv_bfloat162 c[4];
};
struct __align__(8) BfL2 {
    __nv_bfloat162 c[2];
};

__device__ __forceinline__ cx<float> bf_cx(__nv_bfloat162 v)
{
    const float2 f = __bfloat1622float2(v);
    return {f.x, f.y};
}
__device__ __forceinline__ __nv_bfloat162 cx_bf(cx<float> v) { return __float22bfloat162_rn(make_float2(v.re, v.im)); }

__device__ __forceinline__ BfS4 ldg(const BfS4 *p)
{
    const uint4 t = __ldg(reinterpret_cast<const uint4 *>(p));
    return *reinterpret_cast<const BfS4 *>(&t);
}
// BF16 links are read once per launch: loaded without L1 allocation, like the
// FP32 links of the single-right-hand-side kernels
__device__ __forceinline__ BfL2 ldg(const BfL2 *p)
{
    uint2 t;
    asm("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(t.x), "=r"(t.y) : "l"(p));
    return *reinterpret_cast<const BfL2 *>(&t);
}

__device__ __forceinline__ void load_spinor(const BfS4 *__restrict__ p, long long stride, long long s, cx<float> v[12])
{
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const BfS4 t = ldg(p + k * stride + s);
#pragma unroll
        for (int j = 0; j < 4; j++) v[4 * k + j] = bf_cx(t.c[j]);
    }
}
__device__ __forceinline__ void load_spinor_rw(const BfS4 *p, long long stride, long long s, cx<float> v[12])
{
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const BfS4 t = p[k * stride + s];
#pragma unroll
        for (int j = 0; j < 4; j++) v[4 * k + j] = bf_cx(t.c[j]);
    }
}
__device__ __forceinline__ void store_spinor(BfS4 *p, long long stride, long long s, const cx<float> v[12])
{
#pragma unroll
    for (int k = 0; k < 3; k++) {
        BfS4 t;
#pragma unroll
        for (int j = 0; j < 4; j++) t.c[j] = cx_bf(v[4 * k + j]);
        p[k * stride + s] = t;
    }
}
__device__ __forceinline__ void load_link(const BfL2 *__restrict__ U, long long stride, int mu, long long s,
                                          cx<float> m[9])
{
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const BfL2 t = ldg(U + (mu * 3 + k) * stride + s);
        m[2 * k] = bf_cx(t.c[0]);
        m[2 * k + 1] = bf_cx(t.c[1]);
    }
    // SU(3): third row = conj(row0 x row1)
    m[6] = cconj(cmul(m[1], m[5]) - cmul(m[2], m[4]));
    m[7] = cconj(cmul(m[2], m[3]) - cmul(m[0], m[5]));
    m[8] = cconj(cmul(m[0], m[4]) - cmul(m[1], m[3]));
}

}  // namespace lq
