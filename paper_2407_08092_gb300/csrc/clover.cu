// Clover term on the device: build from the gauge field, LDL^+ inverse of the
// 6x6 Hermitian blocks, copies in the other precisions and natural export.
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
//
// The library builds and inverts in df64 (FP64-accurate, on the FP32 units,
// which GB300 runs at 64 times its FP64 rate); the assembly and inverse kernels
// also write the FP64 and FP32 copies, rounded from df64.  The build is split in two launches: one thread per
// (site, plane) computes the four leaves and F of that plane into a scratch
// array, then one thread per site assembles the two 6x6 blocks.
#include "leaves.cuh"
#include "lq_kernels.h"

namespace lq {

__device__ __forceinline__ void store_pair(double2 *p, double a, double b) { *p = make_double2(a, b); }

// one packed 6x6 block (36 df64 reals) of the site with checkerboard index s:
// the df64 copy and its rounding to FP64 and FP32 (FP32: two complex slots per
// float4)
__device__ __forceinline__ void store_block_all(const Geom &g, int b, long long s, const df64 r[36], df2 *Cdf,
                                                double2 *C64, float4 *C32)
{
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const df64 a0 = r[4 * k], a1 = r[4 * k + 1], a2 = r[4 * k + 2], a3 = r[4 * k + 3];
        Cdf[(b * 18 + 2 * k) * g.stride + s] = df2{a0.hi, a0.lo, a1.hi, a1.lo};
        Cdf[(b * 18 + 2 * k + 1) * g.stride + s] = df2{a2.hi, a2.lo, a3.hi, a3.lo};
        const double d0 = df_to_double(a0), d1 = df_to_double(a1), d2 = df_to_double(a2), d3 = df_to_double(a3);
        C64[(b * 18 + 2 * k) * g.stride + s] = make_double2(d0, d1);
        C64[(b * 18 + 2 * k + 1) * g.stride + s] = make_double2(d2, d3);
        C32[(b * 9 + k) * g.stride + s] = make_float4((float)d0, (float)d1, (float)d2, (float)d3);
    }
}
__device__ __forceinline__ void store_pair(df2 *p, df64 a, df64 b) { *p = df2{a.hi, a.lo, b.hi, b.lo}; }
__device__ __forceinline__ bool positive(double d) { return d > 0.0; }
__device__ __forceinline__ bool positive(df64 d) { return df_positive(d); }

// Field strength of one plane at one site per thread: F = (Q - Q^+)/8 is
// anti-Hermitian, so 9 reals describe it: Im F_aa (a = 0,1,2), then F_01, F_02,
// F_12 (re, im).  Stored as df64 pairs in F[plane][9][V].  The leaf factors
// come from the tables of leaves.cuh.
__global__ void __launch_bounds__(128) clover_field_kernel(Geom g, const df2 *__restrict__ Ue,
                                                           const df2 *__restrict__ Uo, float2 *Fb)
{
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= 6 * g.V) return;
    const int p = (int)(id / g.V);
    const long long lex = id - p * g.V;
    int c[4];
    {
        long long r = lex;
        c[0] = (int)(r % g.L[0]); r /= g.L[0];
        c[1] = (int)(r % g.L[1]); r /= g.L[1];
        c[2] = (int)(r % g.L[2]); c[3] = (int)(r / g.L[2]);
    }
    const int mu = c_pmu[p], nu = c_pnu[p];
    M3<df64> Q;
#pragma unroll
    for (int k = 0; k < 9; k++) Q.a[k] = {df64(0.0f, 0.0f), df64(0.0f, 0.0f)};
#pragma unroll 1
    for (int leaf = 0; leaf < 4; leaf++) {
        M3<df64> T;
#pragma unroll 1
        for (int i = 0; i < 4; i++) {
            const int f = 4 * leaf + i;
            int cc[4] = {c[0], c[1], c[2], c[3]};
            cc[mu] = (cc[mu] + c_ldmu[f] + g.L[mu]) % g.L[mu];
            cc[nu] = (cc[nu] + c_ldnu[f] + g.L[nu]) % g.L[nu];
            M3<df64> Lk = link_at<df64>(g, Ue, Uo, cc, c_lnu[f] ? nu : mu);
            if (c_ldag[f]) {
                M3<df64> d;
#pragma unroll
                for (int a = 0; a < 3; a++)
#pragma unroll
                    for (int b = 0; b < 3; b++) d.a[a * 3 + b] = cconj(Lk.a[b * 3 + a]);
                Lk = d;
            }
            T = i == 0 ? Lk : mat_mul(T, Lk);
        }
#pragma unroll
        for (int k = 0; k < 9; k++) dl_cadd(Q.a[k], T.a[k]);   // renormalised after the four leaves
    }
#pragma unroll
    for (int k = 0; k < 9; k++) Q.a[k] = dl_cnorm(Q.a[k]);
    // F = (Q - Q^+)/8: Im F_aa, then F_01, F_02, F_12
    const df64 eighth(0.125f, 0.0f);
    auto fa = [&](int a, int b) { return eighth * (Q.a[a * 3 + b] - cconj(Q.a[b * 3 + a])); };
    const cx<df64> f01 = fa(0, 1), f02 = fa(0, 2), f12 = fa(1, 2);
    const df64 v[9] = {fa(0, 0).im, fa(1, 1).im, fa(2, 2).im, f01.re, f01.im, f02.re, f02.im, f12.re, f12.im};
#pragma unroll
    for (int k = 0; k < 9; k++) Fb[((long long)p * 9 + k) * g.V + lex] = make_float2(v[k].hi, v[k].lo);
}

// entry (a, b) of the anti-Hermitian F of plane p at site lex
__device__ __forceinline__ cx<df64> f_entry(const float2 *__restrict__ Fb, long long V, long long lex, int p, int a,
                                            int b)
{
    auto ld = [&](int k) {
        const float2 t = __ldg(Fb + ((long long)p * 9 + k) * V + lex);
        return df64(t.x, t.y);
    };
    if (a == b) return {df64(0.0f, 0.0f), ld(a)};
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    const int k = 3 + 2 * (lo == 0 ? hi - 1 : 2);   // (0,1) -> 3, (0,2) -> 5, (1,2) -> 7
    const cx<df64> u = {ld(k), ld(k + 1)};
    return a < b ? u : cx<df64>{-u.re, u.im};       // F_ba = -conj(F_ab)
}

// Assemble the two packed 6x6 blocks of C(x) from the six field strengths:
// block b: G1 = -F_yz +- F_xt, G2 = F_xz +- F_yt, G3 = -F_xy +- F_zt (+ for b = 0),
// M = i h [[G3, G1 - i G2], [G1 + i G2, -G3]], h = c_sw / 2, C = (4 + m0) + M.
__global__ void __launch_bounds__(128) clover_assemble_kernel(Geom g, const float2 *__restrict__ Fb, double csw,
                                                              double m0, df2 *Ce, df2 *Co, double2 *C64e,
                                                              double2 *C64o, float4 *C32e, float4 *C32o)
{
    const long long lex = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (lex >= g.V) return;
    long long r = lex;
    const int c0 = (int)(r % g.L[0]); r /= g.L[0];
    const int c1 = (int)(r % g.L[1]); r /= g.L[1];
    const int c2 = (int)(r % g.L[2]); const int c3 = (int)(r / g.L[2]);
    const int parity = (c0 + c1 + c2 + c3) & 1;
    const long long cb = lex >> 1;
    df2 *C = parity ? Co : Ce;
    const df64 diag(4.0 + m0), h(0.5 * csw);
#pragma unroll 1
    for (int b = 0; b < 2; b++) {
        const bool plus = b == 0;
        // G_l entries (a, c) for this block
        auto G = [&](int l, int a, int cc) {
            const int ps = l == 0 ? 2 : l == 1 ? 1 : 0;   // space plane: yz, xz, xy
            const int pt = l == 0 ? 3 : l == 1 ? 4 : 5;   // time plane: xt, yt, zt
            const cx<df64> fs = f_entry(Fb, g.V, lex, ps, a, cc), ft = f_entry(Fb, g.V, lex, pt, a, cc);
            const cx<df64> s = l == 1 ? fs : -fs;
            return plus ? s + ft : s - ft;
        };
        df64 out[36];
#pragma unroll 1
        for (int i = 0; i < 6; i++) {
            const int si = i / 3, ai = i % 3;
            const df64 v = -(h * G(2, ai, ai).im);          // Re(i h G3_aa) = -h Im(G3_aa)
            out[i] = si == 0 ? diag + v : diag - v;
        }
#pragma unroll 1
        for (int i = 1; i < 6; i++)
            for (int j = 0; j < i; j++) {
                const int si = i / 3, ai = i % 3, sj = j / 3, aj = j % 3;
                cx<df64> m;
                if (si == sj) {
                    m = ti(h * G(2, ai, aj));
                    if (si == 1) m = -m;
                } else {   // si = 1, sj = 0: i h (G1 + i G2)
                    m = ti(h * (G(0, ai, aj) + ti(G(1, ai, aj))));
                }
                const int k = 6 + 2 * tri(i, j);
                out[k] = m.re;
                out[k + 1] = m.im;
            }
        store_block_all(g, b, cb, out, C, parity ? C64o : C64e, parity ? C32o : C32e);
    }
}

// LDL^+ factorisation and inverse of one packed Hermitian 6x6 block.
// A = L D L^+ (L unit lower, D real); A^{-1} = L^{-+} D^{-1} L^{-1}.
template <typename R>
__global__ void __launch_bounds__(128) clover_invert_kernel(Geom g, const typename St<R>::vec *__restrict__ C,
                                                            typename St<R>::vec *Ci, double2 *Ci64, float4 *Ci32,
                                                            int *flag)
{
    long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= 2 * g.Vh) return;
    const int b = (int)(id / g.Vh);
    const long long s = id - b * g.Vh;
    R r[36];
    load_block(C, g.stride, b, s, r);
    cx<R> Lm[6][6];
    R D[6];
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) Lm[i][j] = {R(i == j ? 1.0 : 0.0), R(0.0)};
    bool bad = false;
    for (int j = 0; j < 6; j++) {
        R d = r[j];
        for (int k = 0; k < j; k++) d = d - (Lm[j][k].re * Lm[j][k].re + Lm[j][k].im * Lm[j][k].im) * D[k];
        if (!positive(d)) bad = true;   // Hermitian positive definite expected; NaN fails too
        D[j] = d;
        const R dinv = R(1.0) / d;
        for (int i = j + 1; i < 6; i++) {
            const int kk = 6 + 2 * tri(i, j);
            cx<R> a = {r[kk], r[kk + 1]};
            for (int k = 0; k < j; k++) a = a - D[k] * cmul(Lm[i][k], cconj(Lm[j][k]));
            Lm[i][j] = dinv * a;
        }
    }
    // X = L^{-1} (unit lower) by forward substitution
    cx<R> X[6][6];
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) X[i][j] = {R(i == j ? 1.0 : 0.0), R(0.0)};
    for (int i = 1; i < 6; i++)
        for (int j = 0; j < i; j++) {
            cx<R> acc = {R(0.0), R(0.0)};
            for (int k = j; k < i; k++) acc = cfma(Lm[i][k], X[k][j], acc);
            X[i][j] = -acc;
        }
    R Dinv[6];
    for (int k = 0; k < 6; k++) Dinv[k] = R(1.0) / D[k];
    // A^{-1}_{ij} = sum_{k >= max(i,j)} conj(X_ki) X_kj / D_k  (lower part, i >= j)
    R out[36];
    for (int i = 0; i < 6; i++) {
        R acc = R(0.0);
        for (int k = i; k < 6; k++) acc = acc + (X[k][i].re * X[k][i].re + X[k][i].im * X[k][i].im) * Dinv[k];
        out[i] = acc;
    }
    for (int i = 1; i < 6; i++)
        for (int j = 0; j < i; j++) {
            cx<R> acc = {R(0.0), R(0.0)};
            for (int k = i; k < 6; k++) acc = acc + Dinv[k] * cmulc(X[k][i], X[k][j]);
            const int kk = 6 + 2 * tri(i, j);
            out[kk] = acc.re;
            out[kk + 1] = acc.im;
        }
    store_block_all(g, b, s, out, Ci, Ci64, Ci32);
    if (bad) atomicAdd(flag, 1);
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

void clover_build(const Exec &e, const void *Udf[2], double csw, double m0, void *Cdf[2], void *C64[2],
                  void *C32[2], void *Fscratch)
{
    {
        // unique bytes per site: its four df64 links (4 x 144) and the six F
        // (6 x 72); per (site, plane): 12 complex 3x3 products of 198 flops,
        // the leaf sum and (Q - Q^+)/8
        Launch L_(e, K_CLOVER_FIELD, (double)e.g.V * (4 * 144 + 6 * 72), (double)e.g.V * 6 * (12 * 198 + 54 + 36));
        clover_field_kernel<<<blocks_for(6 * e.g.V, 128), 128, 0, e.st>>>(e.g, (const df2 *)Udf[0],
                                                                                (const df2 *)Udf[1],
                                                                                (float2 *)Fscratch);
    }
    // reads the six F, writes the blocks in df64, FP64 and FP32
    Launch L_(e, K_CLOVER, (double)e.g.V * (6 * 72 + 72 * (8 + 8 + 4)));
    clover_assemble_kernel<<<blocks_for(e.g.V, 128), 128, 0, e.st>>>(
        e.g, (const float2 *)Fscratch, csw, m0, (df2 *)Cdf[0], (df2 *)Cdf[1], (double2 *)C64[0],
        (double2 *)C64[1], (float4 *)C32[0], (float4 *)C32[1]);
}

void clover_invert(const Exec &e, const void *Cdf, void *Cidf, void *Ci64, void *Ci32, int *flag)
{
    Launch L_(e, K_CLOVER, (double)e.g.Vh * 72 * (8 + 8 + 8 + 4), (double)e.g.Vh * 2 * 1500);
    clover_invert_kernel<df64><<<blocks_for(2 * e.g.Vh, 128), 128, 0, e.st>>>(
        e.g, (const df2 *)Cdf, (df2 *)Cidf, (double2 *)Ci64, (float4 *)Ci32, flag);
}

void clover_export(const Exec &e, const void *Ce, const void *Co, void *out)
{
    Launch L_(e, K_CLOVER, (double)e.g.V * (72 * 8 + 72 * 16));
    clover_export_kernel<<<blocks_for(e.g.V, 128), 128, 0, e.st>>>(e.g, (const double2 *)Ce,
                                                                  (const double2 *)Co, (double2 *)out);
}

}  // namespace lq
