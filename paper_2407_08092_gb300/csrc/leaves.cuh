// The plaquette leaves of the clover term (Sec. 2.3), shared by the clover
// build and the fermion force: plane numbering, the link factors of the four
// leaves of a plane, link access by lattice coordinates and the packed form of
// an anti-Hermitian 3x3 matrix.
#pragma once

#include "lq_internal.cuh"

namespace lq {

template <typename R>
struct M3 {
    cx<R> a[9];
};

// Planes (mu, nu), mu < nu, numbered xy, xz, yz, xt, yt, zt.
static __constant__ int c_pmu[6] = {0, 0, 1, 0, 1, 2};
static __constant__ int c_pnu[6] = {1, 2, 2, 3, 3, 3};

// The 16 link factors of the four leaves of plane (mu, nu), leaf by leaf (all
// four run mu -> nu, i.e. with the same orientation, and start and end at x):
//   leaf 1: U_mu(x)       U_nu(x+mu)        U_mu(x+nu)^+     U_nu(x)^+
//   leaf 2: U_nu(x)       U_mu(x-mu+nu)^+   U_nu(x-mu)^+     U_mu(x-mu)
//   leaf 3: U_mu(x-mu)^+  U_nu(x-mu-nu)^+   U_mu(x-mu-nu)    U_nu(x-nu)
//   leaf 4: U_nu(x-nu)^+  U_mu(x-nu)        U_nu(x+mu-nu)    U_mu(x)^+
// as the site offset along mu and nu, whether the link points along nu, and
// whether it enters as U^+.  Walking this table lets one inlined 3x3 product
// serve every product of a leaf (df64 code stays small enough for the
// instruction cache).
static __constant__ signed char c_ldmu[16] = {0, 1, 0, 0, 0, -1, -1, -1, -1, -1, -1, 0, 0, 0, 1, 0};
static __constant__ signed char c_ldnu[16] = {0, 0, 1, 0, 0, 1, 0, 0, 0, -1, -1, -1, -1, -1, -1, 0};
static __constant__ unsigned char c_lnu[16] = {0, 1, 0, 1, 1, 0, 1, 0, 0, 1, 0, 1, 1, 0, 1, 0};
static __constant__ unsigned char c_ldag[16] = {0, 0, 1, 1, 0, 1, 1, 0, 1, 1, 0, 0, 1, 0, 0, 1};

__device__ __forceinline__ long long lex_of(const Geom &g, const int c[4])
{
    return LQ_IDX(c[0] + (long long)g.L[0] * (c[1] + (long long)g.L[1] * (c[2] + (long long)g.L[2] * c[3])), g.V,
                  B_LEX);
}

__device__ __forceinline__ void lex_coords(const Geom &g, long long lex, int c[4])
{
    long long r = lex;
    c[0] = (int)(r % g.L[0]); r /= g.L[0];
    c[1] = (int)(r % g.L[1]); r /= g.L[1];
    c[2] = (int)(r % g.L[2]); c[3] = (int)(r / g.L[2]);
}

// the link U_mu at coordinates c, read from the internal per-parity copies
template <typename R>
__device__ __forceinline__ M3<R> link_at(const Geom &g, const typename St<R>::vec *Ue,
                                         const typename St<R>::vec *Uo, const int c[4], int mu)
{
    const int parity = (c[0] + c[1] + c[2] + c[3]) & 1;
    M3<R> m;
    load_link(parity ? Uo : Ue, g.stride, mu, lex_of(g, c) >> 1, m.a);
    return m;
}

template <typename R>
__device__ __forceinline__ M3<R> dagger(const M3<R> &m)
{
    M3<R> d;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) d.a[a * 3 + b] = cconj(m.a[b * 3 + a]);
    return d;
}

template <typename R>
__device__ __forceinline__ M3<R> mat_mul(const M3<R> &A, const M3<R> &B)
{
    M3<R> P;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            cx<R> acc = cmul(A.a[a * 3], B.a[b]);
            acc = cfma(A.a[a * 3 + 1], B.a[3 + b], acc);
            acc = cfma(A.a[a * 3 + 2], B.a[6 + b], acc);
            P.a[a * 3 + b] = acc;
        }
    return P;
}

// df64: each entry is a lazily normalised compensated sum of its three
// complex products (dl_*), renormalised once
template <>
__device__ __forceinline__ M3<df64> mat_mul<df64>(const M3<df64> &A, const M3<df64> &B)
{
    M3<df64> P;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            cx<df64> acc = dl_cmul(A.a[a * 3], B.a[b]);
            dl_cfma(acc, A.a[a * 3 + 1], B.a[3 + b]);
            dl_cfma(acc, A.a[a * 3 + 2], B.a[6 + b]);
            P.a[a * 3 + b] = dl_cnorm(acc);
        }
    return P;
}

// An anti-Hermitian 3x3 matrix A is stored as 9 reals, as df64 pairs in
// [plane][9][V] float2: Im A_aa (a = 0, 1, 2), then A_01, A_02, A_12 (re, im).
__device__ __forceinline__ M3<df64> load_antiherm(const float2 *__restrict__ base, long long V, long long lex, int p)
{
    df64 v[9];
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const float2 t = __ldg(base + ((long long)p * 9 + k) * V + lex);
        v[k] = df64(t.x, t.y);
    }
    const df64 z(0.0f, 0.0f);
    M3<df64> A;
    A.a[0] = {z, v[0]};
    A.a[4] = {z, v[1]};
    A.a[8] = {z, v[2]};
    A.a[1] = {v[3], v[4]};
    A.a[2] = {v[5], v[6]};
    A.a[5] = {v[7], v[8]};
    A.a[3] = {-v[3], v[4]};   // A_ba = -conj(A_ab)
    A.a[6] = {-v[5], v[6]};
    A.a[7] = {-v[7], v[8]};
    return A;
}

__device__ __forceinline__ void store_antiherm(float2 *base, long long V, long long lex, int p, const df64 v[9])
{
#pragma unroll
    for (int k = 0; k < 9; k++) base[((long long)p * 9 + k) * V + lex] = make_float2(v[k].hi, v[k].lo);
}

}  // namespace lq
