// Clover term on the device: build from the gauge field, LDL^+ inverse of the
// 6x6 Hermitian blocks, FP32 copies and natural-layout export.
//
// C(x) = (4 + m0) + c_sw (i/4) sum_{mu != nu} sigma_mu_nu F_mu_nu(x)
// (Sec. 2.3, Wilson-clover; the 6x6 block structure is the one Sec. 2.4.5
// relies on for D_oo^{-1}).  With the chiral basis the sum splits into
//   C_+ = a + (i c_sw/2) [[G3, G1 - i G2], [G1 + i G2, -G3]]   (spins 0,1)
//   C_- = the same with the time-plane terms negated           (spins 2,3)
// where, with F_ab the field strength of plane (a,b) (0..3 = x,y,z,t):
//   G1 = -F_yz +- F_xt,  G2 = F_xz +- F_yt,  G3 = -F_xy +- F_zt.
// This follows from sigma_jk = -eps_jkl diag(s_l, s_l) and
// sigma_j4 = diag(s_j, -s_j) for the basis g_k = [[0,-i s_k],[i s_k,0]],
// g_4 = [[0,1],[1,0]].
#include "lq_kernels.h"

namespace lq {

struct M3 {
    cx<double> a[9];
};

__device__ __forceinline__ M3 m3_load(const double2 *__restrict__ U, long long site, int mu)
{
    M3 m;
    const double2 *p = U + (site * 4 + mu) * 9;
#pragma unroll
    for (int k = 0; k < 9; k++) {
        double2 t = __ldg(p + k);
        m.a[k] = {t.x, t.y};
    }
    return m;
}

// A * B, A^+ * B, A * B^+
__device__ __forceinline__ M3 mm(const M3 &A, const M3 &B)
{
    M3 C;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cx<double> acc = cmul(A.a[i * 3], B.a[j]);
            acc = cfma(A.a[i * 3 + 1], B.a[3 + j], acc);
            acc = cfma(A.a[i * 3 + 2], B.a[6 + j], acc);
            C.a[i * 3 + j] = acc;
        }
    return C;
}
__device__ __forceinline__ M3 mdm(const M3 &A, const M3 &B)
{
    M3 C;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cx<double> acc = cmulc(A.a[i], B.a[j]);
            acc = cfmac(A.a[3 + i], B.a[3 + j], acc);
            acc = cfmac(A.a[6 + i], B.a[6 + j], acc);
            C.a[i * 3 + j] = acc;
        }
    return C;
}
__device__ __forceinline__ M3 mmd(const M3 &A, const M3 &B)
{
    M3 C;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cx<double> acc = cmul(A.a[i * 3], cconj(B.a[j * 3]));
            acc = cfma(A.a[i * 3 + 1], cconj(B.a[j * 3 + 1]), acc);
            acc = cfma(A.a[i * 3 + 2], cconj(B.a[j * 3 + 2]), acc);
            C.a[i * 3 + j] = acc;
        }
    return C;
}

__device__ __forceinline__ long long lex_of(const Geom &g, const int c[4])
{
    return c[0] + (long long)g.L[0] * (c[1] + (long long)g.L[1] * (c[2] + (long long)g.L[2] * c[3]));
}

__device__ __forceinline__ long long shifted(const Geom &g, const int c0[4], int mu, int dmu, int nu,
                                             int dnu)
{
    int c[4] = {c0[0], c0[1], c0[2], c0[3]};
    c[mu] = (c[mu] + dmu + g.L[mu]) % g.L[mu];
    c[nu] = (c[nu] + dnu + g.L[nu]) % g.L[nu];
    return lex_of(g, c);
}

// F = (Q - Q^+)/8 for the plane (mu, nu) at site c
__device__ void field_strength(const Geom &g, const double2 *__restrict__ U, const int c[4], int mu,
                               int nu, M3 &F)
{
    const long long x = lex_of(g, c);
    const long long xpm = shifted(g, c, mu, 1, nu, 0), xpn = shifted(g, c, mu, 0, nu, 1);
    const long long xmm = shifted(g, c, mu, -1, nu, 0), xmn = shifted(g, c, mu, 0, nu, -1);
    const long long xmmpn = shifted(g, c, mu, -1, nu, 1), xmmmn = shifted(g, c, mu, -1, nu, -1);
    const long long xpmmn = shifted(g, c, mu, 1, nu, -1);
    M3 Q, T;
    // +mu +nu -mu -nu
    T = mm(m3_load(U, x, mu), m3_load(U, xpm, nu));
    T = mmd(T, m3_load(U, xpn, mu));
    Q = mmd(T, m3_load(U, x, nu));
    // +nu -mu -nu +mu
    T = mmd(m3_load(U, x, nu), m3_load(U, xmmpn, mu));
    T = mmd(T, m3_load(U, xmm, nu));
    T = mm(T, m3_load(U, xmm, mu));
#pragma unroll
    for (int k = 0; k < 9; k++) Q.a[k] = Q.a[k] + T.a[k];
    // -mu -nu +mu +nu:  U_mu(x-mu)^+ U_nu(x-mu-nu)^+ = (U_nu(x-mu-nu) U_mu(x-mu))^+
    T = mm(m3_load(U, xmmmn, nu), m3_load(U, xmm, mu));
    T = mdm(T, m3_load(U, xmmmn, mu));
    T = mm(T, m3_load(U, xmn, nu));
#pragma unroll
    for (int k = 0; k < 9; k++) Q.a[k] = Q.a[k] + T.a[k];
    // -nu +mu +nu -mu
    T = mdm(m3_load(U, xmn, nu), m3_load(U, xmn, mu));
    T = mm(T, m3_load(U, xpmmn, nu));
    T = mmd(T, m3_load(U, x, mu));
#pragma unroll
    for (int k = 0; k < 9; k++) Q.a[k] = Q.a[k] + T.a[k];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            cx<double> q = Q.a[i * 3 + j], qt = cconj(Q.a[j * 3 + i]);
            F.a[i * 3 + j] = 0.125 * (q - qt);
        }
}

__global__ void __launch_bounds__(128) clover_build_kernel(Geom g, const double2 *__restrict__ U,
                                                           double csw, double m0, double2 *Ce,
                                                           double2 *Co)
{
    long long lex = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (lex >= g.V) return;
    int c[4];
    {
        long long r = lex;
        c[0] = (int)(r % g.L[0]); r /= g.L[0];
        c[1] = (int)(r % g.L[1]); r /= g.L[1];
        c[2] = (int)(r % g.L[2]); c[3] = (int)(r / g.L[2]);
    }
    const int parity = (c[0] + c[1] + c[2] + c[3]) & 1;
    const long long cb = lex >> 1;
    double2 *C = parity ? Co : Ce;

    // G[blk][l] for l = 1,2,3 (0-based 0..2)
    M3 G[2][3];
#pragma unroll
    for (int b = 0; b < 2; b++)
#pragma unroll
        for (int l = 0; l < 3; l++)
#pragma unroll
            for (int k = 0; k < 9; k++) G[b][l].a[k] = {0.0, 0.0};

    // planes: (mu,nu), the G it feeds and the sign of the space-space term;
    // time-plane terms enter block 0 with + and block 1 with -.
    // G1 = -F_yz +- F_xt ; G2 = F_xz +- F_yt ; G3 = -F_xy +- F_zt
    const int pmu[6] = {0, 0, 1, 0, 1, 2};
    const int pnu[6] = {1, 2, 2, 3, 3, 3};
    const int gl[6] = {2, 1, 0, 0, 1, 2};
    const double sgn[6] = {-1.0, 1.0, -1.0, 1.0, 1.0, 1.0};
    for (int p = 0; p < 6; p++) {
        M3 F;
        field_strength(g, U, c, pmu[p], pnu[p], F);
        const bool time_plane = pnu[p] == 3;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            G[0][gl[p]].a[k] = G[0][gl[p]].a[k] + sgn[p] * F.a[k];
            const double s1 = time_plane ? -sgn[p] : sgn[p];
            G[1][gl[p]].a[k] = G[1][gl[p]].a[k] + s1 * F.a[k];
        }
    }

    const double diag = 4.0 + m0;
    const double h = 0.5 * csw;   // (i c_sw / 2) * ...
    for (int b = 0; b < 2; b++) {
        // M = i h [[G3, G1 - i G2], [G1 + i G2, -G3]]
        double r[36];
        for (int i = 0; i < 6; i++) {
            const int si = i / 3, ai = i % 3;
            cx<double> gd = G[b][2].a[ai * 3 + ai];
            double v = -h * gd.im;      // Re(i h G3_aa) = -h Im(G3_aa)
            r[i] = diag + (si == 0 ? v : -v);
        }
        for (int i = 1; i < 6; i++)
            for (int j = 0; j < i; j++) {
                const int si = i / 3, ai = i % 3, sj = j / 3, aj = j % 3;
                cx<double> m;
                if (si == sj) {
                    cx<double> g3 = G[b][2].a[ai * 3 + aj];
                    m = ti(h * g3);
                    if (si == 1) m = -m;
                } else {   // si = 1, sj = 0: i h (G1 + i G2)
                    cx<double> g1 = G[b][0].a[ai * 3 + aj], g2 = G[b][1].a[ai * 3 + aj];
                    m = ti(h * (g1 + ti(g2)));
                }
                const int k = 6 + 2 * tri(i, j);
                r[k] = m.re;
                r[k + 1] = m.im;
            }
        for (int k = 0; k < 18; k++) C[(b * 18 + k) * g.stride + cb] = make_double2(r[2 * k], r[2 * k + 1]);
    }
}

// LDL^+ factorisation and inverse of one packed Hermitian 6x6 block.
// A = L D L^+ (L unit lower, D real); A^{-1} = L^{-+} D^{-1} L^{-1}.
__global__ void __launch_bounds__(128) clover_invert_kernel(Geom g, const double2 *__restrict__ C,
                                                            double2 *Ci, int *flag)
{
    long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= 2 * g.Vh) return;
    const int b = (int)(id / g.Vh);
    const long long s = id - b * g.Vh;
    double r[36];
    for (int k = 0; k < 18; k++) {
        double2 t = C[(b * 18 + k) * g.stride + s];
        r[2 * k] = t.x;
        r[2 * k + 1] = t.y;
    }
    cx<double> Lm[6][6];
    double D[6];
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) Lm[i][j] = {i == j ? 1.0 : 0.0, 0.0};
    bool bad = false;
    for (int j = 0; j < 6; j++) {
        double d = r[j];
        for (int k = 0; k < j; k++) d -= (Lm[j][k].re * Lm[j][k].re + Lm[j][k].im * Lm[j][k].im) * D[k];
        if (!(d > 0.0)) bad = true;   // Hermitian positive definite expected; NaN fails too
        D[j] = d;
        const double dinv = 1.0 / d;
        for (int i = j + 1; i < 6; i++) {
            const int kk = 6 + 2 * tri(i, j);
            cx<double> a = {r[kk], r[kk + 1]};
            for (int k = 0; k < j; k++) a = a - D[k] * cmul(Lm[i][k], cconj(Lm[j][k]));
            Lm[i][j] = dinv * a;
        }
    }
    // X = L^{-1} (unit lower) by forward substitution
    cx<double> X[6][6];
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) X[i][j] = {i == j ? 1.0 : 0.0, 0.0};
    for (int i = 1; i < 6; i++)
        for (int j = 0; j < i; j++) {
            cx<double> acc = {0.0, 0.0};
            for (int k = j; k < i; k++) acc = cfma(Lm[i][k], X[k][j], acc);
            X[i][j] = -acc;
        }
    // A^{-1}_{ij} = sum_{k >= max(i,j)} conj(X_ki) X_kj / D_k  (lower part, i >= j)
    double out[36];
    for (int i = 0; i < 6; i++) {
        double acc = 0.0;
        for (int k = i; k < 6; k++) acc += (X[k][i].re * X[k][i].re + X[k][i].im * X[k][i].im) / D[k];
        out[i] = acc;
    }
    for (int i = 1; i < 6; i++)
        for (int j = 0; j < i; j++) {
            cx<double> acc = {0.0, 0.0};
            for (int k = i; k < 6; k++) acc = acc + (1.0 / D[k]) * cmulc(X[k][i], X[k][j]);
            const int kk = 6 + 2 * tri(i, j);
            out[kk] = acc.re;
            out[kk + 1] = acc.im;
        }
    for (int k = 0; k < 18; k++) Ci[(b * 18 + k) * g.stride + s] = make_double2(out[2 * k], out[2 * k + 1]);
    if (bad) atomicAdd(flag, 1);
}

__global__ void clover_f32_kernel(Geom g, const double2 *__restrict__ C, float4 *C32)
{
    long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= 2 * g.Vh) return;
    const int b = (int)(id / g.Vh);
    const long long s = id - b * g.Vh;
    for (int k = 0; k < 9; k++) {
        double2 u = C[(b * 18 + 2 * k) * g.stride + s];
        double2 v = C[(b * 18 + 2 * k + 1) * g.stride + s];
        C32[(b * 9 + k) * g.stride + s] = make_float4((float)u.x, (float)u.y, (float)v.x, (float)v.y);
    }
}

__global__ void clover_export_kernel(Geom g, const double2 *__restrict__ Ce, const double2 *__restrict__ Co,
                                     double2 *out)
{
    long long lex = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (lex >= g.V) return;
    long long r = lex;
    int c0 = (int)(r % g.L[0]); r /= g.L[0];
    int c1 = (int)(r % g.L[1]); r /= g.L[1];
    int c2 = (int)(r % g.L[2]); int c3 = (int)(r / g.L[2]);
    const int parity = (c0 + c1 + c2 + c3) & 1;
    const long long cb = lex >> 1;
    const double2 *C = parity ? Co : Ce;
    double2 *o = out + lex * 72;
    for (int b = 0; b < 2; b++) {
        double rr[36];
        for (int k = 0; k < 18; k++) {
            double2 t = C ? C[(b * 18 + k) * g.stride + cb] : make_double2(0.0, 0.0);
            rr[2 * k] = t.x;
            rr[2 * k + 1] = t.y;
        }
        for (int i = 0; i < 6; i++)
            for (int j = 0; j < 6; j++) {
                double2 v;
                if (i == j) v = make_double2(rr[i], 0.0);
                else if (i > j) v = make_double2(rr[6 + 2 * tri(i, j)], rr[6 + 2 * tri(i, j) + 1]);
                else v = make_double2(rr[6 + 2 * tri(j, i)], -rr[6 + 2 * tri(j, i) + 1]);
                o[b * 36 + i * 6 + j] = v;
            }
    }
}

static inline unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

void clover_build(const Exec &e, const void *U_nat, double csw, double m0, void *C64[2])
{
    Launch L_(e, K_CLOVER, (double)e.g.V * (4 * 9 * 16 + 72 * 8));
    clover_build_kernel<<<blocks_for(e.g.V, 128), 128, 0, e.st>>>(
        e.g, (const double2 *)U_nat, csw, m0, (double2 *)C64[0], (double2 *)C64[1]);
}

void clover_invert(const Exec &e, const void *C64, void *Cinv64, int *flag)
{
    Launch L_(e, K_CLOVER, (double)e.g.Vh * 2 * 72 * 8);
    clover_invert_kernel<<<blocks_for(2 * e.g.Vh, 128), 128, 0, e.st>>>(e.g, (const double2 *)C64,
                                                                        (double2 *)Cinv64, flag);
}

void clover_to_f32(const Exec &e, const void *C64, void *C32)
{
    Launch L_(e, K_CLOVER, (double)e.g.Vh * 72 * (8 + 4));
    clover_f32_kernel<<<blocks_for(2 * e.g.Vh, 256), 256, 0, e.st>>>(e.g, (const double2 *)C64, (float4 *)C32);
}

void clover_export(const Exec &e, const void *Ce, const void *Co, void *out)
{
    Launch L_(e, K_CLOVER, (double)e.g.V * (72 * 8 + 72 * 16));
    clover_export_kernel<<<blocks_for(e.g.V, 128), 128, 0, e.st>>>(e.g, (const double2 *)Ce,
                                                                  (const double2 *)Co, (double2 *)out);
}

}  // namespace lq
