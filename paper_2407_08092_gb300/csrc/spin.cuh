// Spin projection and colour transport of one hop of the Wilson operator,
// shared by the hopping kernels (global-memory neighbours) and the SAP block
// kernel (shared-memory neighbours).
//
// Projection identities (chiral basis, upper = spins 0,1):
//   (1 - s g_k) psi = (h, s(-i s_k) h)  with h = psi_u + s i s_k psi_l   (k = 1,2,3)
//   (1 - s g_4) psi = (h, -s h)         with h = psi_u - s psi_l
// where s = +1 for the forward and -1 for the backward hop.
#pragma once

#include "lq_internal.cuh"

namespace lq {

// half spinor h[hs*3 + a] from the full spinor p[s*3 + a]; SIGN = -1 projects
// with (1 - g_mu) (forward hop), SIGN = +1 with (1 + g_mu) (backward hop)
template <int MU, int SIGN, typename R>
__device__ __forceinline__ void project(const cx<R> p[12], cx<R> h[6])
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const cx<R> p0 = p[a], p1 = p[3 + a], p2 = p[6 + a], p3 = p[9 + a];
        if (MU == 0) {
            h[a] = SIGN < 0 ? p0 + ti(p3) : p0 - ti(p3);
            h[3 + a] = SIGN < 0 ? p1 + ti(p2) : p1 - ti(p2);
        } else if (MU == 1) {
            h[a] = SIGN < 0 ? p0 + p3 : p0 - p3;
            h[3 + a] = SIGN < 0 ? p1 - p2 : p1 + p2;
        } else if (MU == 2) {
            h[a] = SIGN < 0 ? p0 + ti(p2) : p0 - ti(p2);
            h[3 + a] = SIGN < 0 ? p1 - ti(p3) : p1 + ti(p3);
        } else {
            h[a] = SIGN < 0 ? p0 - p2 : p0 + p2;
            h[3 + a] = SIGN < 0 ? p1 - p3 : p1 + p3;
        }
    }
}

// acc += the full spinor reconstructed from the transported half spinor u
template <int MU, int SIGN, typename R>
__device__ __forceinline__ void reconstruct(cx<R> acc[12], const cx<R> u[6])
{
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const cx<R> u0 = u[a], u1 = u[3 + a];
        acc[a] = acc[a] + u0;
        acc[3 + a] = acc[3 + a] + u1;
        if (MU == 0) {
            acc[6 + a] = SIGN < 0 ? acc[6 + a] + tmi(u1) : acc[6 + a] + ti(u1);
            acc[9 + a] = SIGN < 0 ? acc[9 + a] + tmi(u0) : acc[9 + a] + ti(u0);
        } else if (MU == 1) {
            acc[6 + a] = SIGN < 0 ? acc[6 + a] - u1 : acc[6 + a] + u1;
            acc[9 + a] = SIGN < 0 ? acc[9 + a] + u0 : acc[9 + a] - u0;
        } else if (MU == 2) {
            acc[6 + a] = SIGN < 0 ? acc[6 + a] + tmi(u0) : acc[6 + a] + ti(u0);
            acc[9 + a] = SIGN < 0 ? acc[9 + a] + ti(u1) : acc[9 + a] + tmi(u1);
        } else {
            acc[6 + a] = SIGN < 0 ? acc[6 + a] - u0 : acc[6 + a] + u0;
            acc[9 + a] = SIGN < 0 ? acc[9 + a] - u1 : acc[9 + a] + u1;
        }
    }
}

// acc += bsign (1 -+ g_mu) W p for a loaded neighbour spinor p and link m:
// W = m (SIGN -1, forward hop) or m^+ (SIGN +1, backward hop)
template <int MU, int SIGN, typename R>
__device__ __forceinline__ void hop_apply(cx<R> acc[12], const cx<R> p[12], const cx<R> m[9], R bsign)
{
    cx<R> h[6];
    project<MU, SIGN>(p, h);
    cx<R> u[6];
#pragma unroll
    for (int hs = 0; hs < 2; hs++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            cx<R> t;
            if (SIGN < 0) {
                t = cmul(m[a * 3 + 0], h[hs * 3 + 0]);
                t = cfma(m[a * 3 + 1], h[hs * 3 + 1], t);
                t = cfma(m[a * 3 + 2], h[hs * 3 + 2], t);
            } else {
                t = cmulc(m[0 * 3 + a], h[hs * 3 + 0]);
                t = cfmac(m[1 * 3 + a], h[hs * 3 + 1], t);
                t = cfmac(m[2 * 3 + a], h[hs * 3 + 2], t);
            }
            u[hs * 3 + a] = bsign * t;
        }
    reconstruct<MU, SIGN>(acc, u);
}

}  // namespace lq
