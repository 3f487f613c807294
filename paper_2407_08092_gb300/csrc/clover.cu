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
// also write the FP32 copies, rounded from df64.  The FP64 copies are rounded
// from df64 by clover_to_f64 when an FP64 operator first needs them.  The
// field strengths F of the six planes come from three passes over plaquettes
// (one thread per (site, plane) each, into scratch arrays), then one thread
// per site assembles the two 6x6 blocks.
#include "leaves.cuh"
#include "lq_kernels.h"

namespace lq {

__device__ __forceinline__ void store_pair(double2 *p, double a, double b) { *p = make_double2(a, b); }

// one packed 6x6 block (36 df64 reals) of the site with checkerboard index s:
// the df64 copy and its rounding to FP32 (two complex slots per float4)
__device__ __forceinline__ void store_block_df32(const Geom &g, int b, long long s, const df64 r[36], df2 *Cdf,
                                                 float4 *C32)
{
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const df64 a0 = r[4 * k], a1 = r[4 * k + 1], a2 = r[4 * k + 2], a3 = r[4 * k + 3];
        Cdf[(b * 18 + 2 * k) * g.stride + s] = df2{a0.hi, a0.lo, a1.hi, a1.lo};
        Cdf[(b * 18 + 2 * k + 1) * g.stride + s] = df2{a2.hi, a2.lo, a3.hi, a3.lo};
        C32[(b * 9 + k) * g.stride + s] =
            make_float4(df_to_float(a0), df_to_float(a1), df_to_float(a2), df_to_float(a3));
    }
}
__device__ __forceinline__ void store_pair(df2 *p, df64 a, df64 b) { *p = df2{a.hi, a.lo, b.hi, b.lo}; }
__device__ __forceinline__ bool positive(double d) { return d > 0.0; }
__device__ __forceinline__ bool positive(df64 d) { return df_positive(d); }

// ---------------------------------------------------------------------------
// The field strengths in three passes over plaquettes.  Each of the four
// leaves at x is the plaquette of a neighbouring corner rotated to start at x,
// and the anti-Hermitian part AH(M) = M - M^+ commutes with that unitary
// rotation, so with P(y) = U_mu(y) U_nu(y+mu) U_mu(y+nu)^+ U_nu(y)^+:
//   pass 1  H(y) = AH(P(y))
//   pass 2  R(y) = H(y) + U_mu(y-mu)^+ H(y-mu) U_mu(y-mu)       (leaves 1, 2)
//   pass 3  F(x) = [R(x) + U_nu(x-nu)^+ R(x-nu) U_nu(x-nu)] / 8 (leaves 1..4)
// which is F = (Q - Q^+)/8 with Q the sum of the four leaves.  Per (site,
// plane) this takes two full 3x3 products and one anti-Hermitian-only product
// in pass 1 and one product plus one anti-Hermitian-only product in each of
// passes 2 and 3, against twelve full products for the four leaves formed one
// by one.  H, R and F are anti-Hermitian and stored as 9 reals (df64 pairs in
// [plane][9][V] float2: Im A_aa, then A_01, A_02, A_12).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void site_coords(const Geom &g, long long lex, int c[4])
{
    long long r = lex;
    c[0] = (int)(r % g.L[0]);
    r /= g.L[0];
    c[1] = (int)(r % g.L[1]);
    r /= g.L[1];
    c[2] = (int)(r % g.L[2]);
    c[3] = (int)(r / g.L[2]);
}

// coordinates c shifted by s (-1, 0, +1) along mu
__device__ __forceinline__ void shifted(const Geom &g, const int c[4], int mu, int s, int out[4])
{
#pragma unroll
    for (int k = 0; k < 4; k++) out[k] = c[k];
    const int L = mu == 0 ? g.L[0] : mu == 1 ? g.L[1] : mu == 2 ? g.L[2] : g.L[3];
    int v = (mu == 0 ? c[0] : mu == 1 ? c[1] : mu == 2 ? c[2] : c[3]) + s;
    v = v < 0 ? v + L : (v >= L ? v - L : v);
    if (mu == 0) out[0] = v;
    else if (mu == 1) out[1] = v;
    else if (mu == 2) out[2] = v;
    else out[3] = v;
}

// A B^+ (full product), each entry a lazily normalised compensated sum
__device__ __forceinline__ M3<df64> mat_mul_nd(const M3<df64> &A, const M3<df64> &B)
{
    M3<df64> P;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            // sum_k A_ak conj(B_bk) = sum_k conj(B_bk) A_ak
            cx<df64> acc = dl_cmul(cconj(B.a[b * 3]), A.a[a * 3]);
            dl_cfmac(acc, B.a[b * 3 + 1], A.a[a * 3 + 1]);
            dl_cfmac(acc, B.a[b * 3 + 2], A.a[a * 3 + 2]);
            P.a[a * 3 + b] = dl_cnorm(acc);
        }
    return P;
}

// the 9 reals of AH(A B^+): Im 2 (A B^+)_aa, then (A B^+)_ab - conj((A B^+)_ba) for a < b
__device__ __forceinline__ void ah_of_mul_nd(const M3<df64> &A, const M3<df64> &B, df64 v[9])
{
#pragma unroll
    for (int a = 0; a < 3; a++) {   // Im sum_k A_ak conj(B_ak) = sum_k (A.im B.re - A.re B.im)
        df64 s = dl_prod(A.a[a * 3].im, B.a[a * 3].re);
        dl_fma(s, dl_neg(A.a[a * 3].re), B.a[a * 3].im);
#pragma unroll
        for (int k = 1; k < 3; k++) {
            dl_fma(s, A.a[a * 3 + k].im, B.a[a * 3 + k].re);
            dl_fma(s, dl_neg(A.a[a * 3 + k].re), B.a[a * 3 + k].im);
        }
        v[a] = dl_scale2(dl_norm(s), 2.0f);
    }
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const int a = pa[q], b = pb[q];
        // X = sum_k A_ak conj(B_bk), Y = sum_k A_bk conj(B_ak); AH_ab = X - conj(Y)
        cx<df64> x = dl_cmul(cconj(B.a[b * 3]), A.a[a * 3]), y = dl_cmul(cconj(B.a[a * 3]), A.a[b * 3]);
#pragma unroll
        for (int k = 1; k < 3; k++) {
            dl_cfmac(x, B.a[b * 3 + k], A.a[a * 3 + k]);
            dl_cfmac(y, B.a[a * 3 + k], A.a[b * 3 + k]);
        }
        dl_add(x.re, dl_neg(y.re));
        dl_add(x.im, y.im);
        v[3 + 2 * q] = dl_norm(x.re);
        v[4 + 2 * q] = dl_norm(x.im);
    }
}

// the 9 reals of W^+ H W for an anti-Hermitian H (itself anti-Hermitian)
__device__ __forceinline__ void ah_conj(const M3<df64> &H, const M3<df64> &W, df64 v[9])
{
    const M3<df64> Y = mat_mul<df64>(H, W);
#pragma unroll
    for (int a = 0; a < 3; a++) {   // Im sum_k conj(W_ka) Y_ka = sum_k (W.re Y.im - W.im Y.re)
        df64 s = dl_prod(W.a[a].re, Y.a[a].im);
        dl_fma(s, dl_neg(W.a[a].im), Y.a[a].re);
#pragma unroll
        for (int k = 1; k < 3; k++) {
            dl_fma(s, W.a[k * 3 + a].re, Y.a[k * 3 + a].im);
            dl_fma(s, dl_neg(W.a[k * 3 + a].im), Y.a[k * 3 + a].re);
        }
        v[a] = dl_norm(s);
    }
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const int a = pa[q], b = pb[q];
        cx<df64> z = dl_cmul(cconj(W.a[a]), Y.a[b]);   // sum_k conj(W_ka) Y_kb
#pragma unroll
        for (int k = 1; k < 3; k++) dl_cfmac(z, W.a[k * 3 + a], Y.a[k * 3 + b]);
        v[3 + 2 * q] = dl_norm(z.re);
        v[4 + 2 * q] = dl_norm(z.im);
    }
}

// pass 1: H(y) = AH(P(y)), one thread per (site, plane)
#ifndef LQ_PLAQ_MINB
#define LQ_PLAQ_MINB 4
#endif
__global__ void __launch_bounds__(128, LQ_PLAQ_MINB) clover_plaq_kernel(Geom g, const df2 *__restrict__ Ue,
                                                          const df2 *__restrict__ Uo, float2 *H)
{
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= 6 * g.V) return;
    const int p = (int)(id / g.V);
    const long long lex = id - p * g.V;
    int c[4], cm[4], cn[4];
    site_coords(g, lex, c);
    const int mu = c_pmu[p], nu = c_pnu[p];
    shifted(g, c, mu, +1, cm);
    shifted(g, c, nu, +1, cn);
    const M3<df64> T1 = mat_mul<df64>(link_at<df64>(g, Ue, Uo, c, mu), link_at<df64>(g, Ue, Uo, cm, nu));
    const M3<df64> T2 = mat_mul_nd(T1, link_at<df64>(g, Ue, Uo, cn, mu));
    df64 v[9];
    ah_of_mul_nd(T2, link_at<df64>(g, Ue, Uo, c, nu), v);
    store_antiherm(H, g.V, lex, p, v);
}

// passes 2 and 3: Out(x) = scale [In(x) + W^+ In(x - e) W], W = U_e(x - e) with
// e = mu (pass 2) or nu (pass 3) of the thread's plane
template <bool NU>
__global__ void __launch_bounds__(128) clover_rot_kernel(Geom g, const df2 *__restrict__ Ue,
                                                         const df2 *__restrict__ Uo, const float2 *__restrict__ In,
                                                         float2 *Out, float scale)
{
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= 6 * g.V) return;
    const int p = (int)(id / g.V);
    const long long lex = id - p * g.V;
    int c[4], cs[4];
    site_coords(g, lex, c);
    const int e = NU ? c_pnu[p] : c_pmu[p];
    shifted(g, c, e, -1, cs);
    df64 v[9];
    ah_conj(load_antiherm(In, g.V, lex_of(g, cs), p), link_at<df64>(g, Ue, Uo, cs, e), v);
    df64 w[9];
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const float2 t = __ldg(In + ((long long)p * 9 + k) * g.V + lex);
        df64 sum = df64(t.x, t.y) + v[k];
        w[k] = dl_scale2(sum, scale);   // scale 1 or 1/8: exact
    }
    store_antiherm(Out, g.V, lex, p, w);
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
// The entries are formed in their packed order and stored four at a time (two
// df2 and one FP32 float4), so only four of a block's 36 entries are held in
// registers at once.  diag = 4 + m0 and h come as df64 pairs split on the host.
// Four resident blocks per SM (128 registers, a few bytes of spills) against
// two unbounded: 0.60 against 0.74 ms per launch of assembly and inverse on
// 32^3 x 64, on average.
#ifndef LQ_CLA_MINB
#define LQ_CLA_MINB 4
#endif
__global__ void __launch_bounds__(128, LQ_CLA_MINB) clover_assemble_kernel(Geom g, const float2 *__restrict__ Fb, df64 diag,
                                                              df64 h, df2 *Ce, df2 *Co, float4 *C32e, float4 *C32o)
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
    float4 *C32 = parity ? C32o : C32e;
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
        // packed entry k (every k below is a constant): kept until its group of
        // four is complete, then stored
        df64 buf[4];
        auto emit = [&](int k, df64 v) {
            buf[k & 3] = v;
            if ((k & 3) == 3) {
                const int q = k >> 2;
                C[(b * 18 + 2 * q) * g.stride + cb] = df2{buf[0].hi, buf[0].lo, buf[1].hi, buf[1].lo};
                C[(b * 18 + 2 * q + 1) * g.stride + cb] = df2{buf[2].hi, buf[2].lo, buf[3].hi, buf[3].lo};
                C32[(b * 9 + q) * g.stride + cb] =
                    make_float4(df_to_float(buf[0]), df_to_float(buf[1]), df_to_float(buf[2]), df_to_float(buf[3]));
            }
        };
#pragma unroll
        for (int i = 0; i < 6; i++) {
            const int si = i / 3, ai = i % 3;
            const df64 v = -(h * G(2, ai, ai).im);          // Re(i h G3_aa) = -h Im(G3_aa)
            emit(i, si == 0 ? diag + v : diag - v);
        }
#pragma unroll
        for (int i = 1; i < 6; i++)
#pragma unroll
            for (int j = 0; j < i; j++) {
                const int si = i / 3, ai = i % 3, sj = j / 3, aj = j % 3;
                cx<df64> m;
                if (si == sj) {
                    m = ti(h * G(2, ai, aj));
                    if (si == 1) m = -m;
                } else {   // si = 1, sj = 0: i h (G1 + i G2)
                    m = ti(h * (G(0, ai, aj) + ti(G(1, ai, aj))));
                }
                const int k = 6 + 2 * tri(i, j);   // increasing with (i, j) in this order
                emit(k, m.re);
                emit(k + 1, m.im);
            }
    }
}

// LDL^+ factorisation and inverse of one packed Hermitian 6x6 block in df64:
// A = L D L^+ (L unit lower, D real), X = L^{-1}, A^{-1} = X^+ D^{-1} X.
// Every loop is unrolled, so the factors live in registers, and the sums are
// lazily normalised compensated sums (dl_*).
__global__ void __launch_bounds__(128) clover_invert_kernel(Geom g, const df2 *__restrict__ C, df2 *Ci,
                                                            float4 *Ci32, int *flag)
{
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= 2 * g.Vh) return;
    const int b = (int)(id / g.Vh);
    const long long s = id - b * g.Vh;
    df64 r[36];
    load_block(C, g.stride, b, s, r);
    cx<df64> L[15];   // strictly lower entries, packed by tri(i, j)
    df64 D[6], Dinv[6];
    bool bad = false;
#pragma unroll
    for (int j = 0; j < 6; j++) {
        // c_k = D_k conj(L_jk), k < j
        cx<df64> cj[5];
#pragma unroll
        for (int k = 0; k < j; k++) {
            const cx<df64> l = L[tri(j, k)];
            cj[k] = {D[k] * l.re, dl_neg(D[k] * l.im)};
        }
        // D_j = A_jj - sum_k Re(L_jk c_k)
        df64 d = r[j];
#pragma unroll
        for (int k = 0; k < j; k++) {
            dl_fma(d, dl_neg(L[tri(j, k)].re), cj[k].re);
            dl_fma(d, L[tri(j, k)].im, cj[k].im);
        }
        d = dl_norm(d);
        if (!df_positive(d)) bad = true;   // Hermitian positive definite expected; NaN fails too
        D[j] = d;
        Dinv[j] = df64(1.0f, 0.0f) / d;
        // L_ij = (A_ij - sum_k L_ik c_k) / D_j, i > j
#pragma unroll
        for (int i = j + 1; i < 6; i++) {
            const int kk = 6 + 2 * tri(i, j);
            cx<df64> a = {r[kk], r[kk + 1]};
#pragma unroll
            for (int k = 0; k < j; k++) dl_cfma(a, {dl_neg(L[tri(i, k)].re), dl_neg(L[tri(i, k)].im)}, cj[k]);
            a = dl_cnorm(a);
            L[tri(i, j)] = {a.re * Dinv[j], a.im * Dinv[j]};
        }
    }
    // X = L^{-1}: X_ij = -(L_ij + sum_{j<k<i} L_ik X_kj), i > j
    cx<df64> X[15];
#pragma unroll
    for (int i = 1; i < 6; i++)
#pragma unroll
        for (int j = 0; j < i; j++) {
            cx<df64> acc = L[tri(i, j)];
#pragma unroll
            for (int k = j + 1; k < i; k++) dl_cfma(acc, L[tri(i, k)], X[tri(k, j)]);
            acc = dl_cnorm(acc);
            X[tri(i, j)] = {dl_neg(acc.re), dl_neg(acc.im)};
        }
    // A^{-1}_ij = sum_{k >= i} conj(X_ki) X_kj / D_k (i >= j, X_kk = 1)
    df64 out[36];
#pragma unroll
    for (int i = 0; i < 6; i++) {
        df64 acc = Dinv[i];
#pragma unroll
        for (int k = i + 1; k < 6; k++) {
            const cx<df64> x = X[tri(k, i)];
            const df64 m2 = dl_norm([&] { df64 t = dl_prod(x.re, x.re); dl_fma(t, x.im, x.im); return t; }());
            dl_fma(acc, m2, Dinv[k]);
        }
        out[i] = dl_norm(acc);
    }
#pragma unroll
    for (int i = 1; i < 6; i++)
#pragma unroll
        for (int j = 0; j < i; j++) {
            const cx<df64> xij = X[tri(i, j)];
            cx<df64> acc = {dl_prod(Dinv[i], xij.re), dl_prod(Dinv[i], xij.im)};
#pragma unroll
            for (int k = i + 1; k < 6; k++) {
                const cx<df64> y = {Dinv[k] * X[tri(k, j)].re, Dinv[k] * X[tri(k, j)].im};
                dl_cfmac(acc, X[tri(k, i)], y);
            }
            acc = dl_cnorm(acc);
            const int kk = 6 + 2 * tri(i, j);
            out[kk] = acc.re;
            out[kk + 1] = acc.im;
        }
    store_block_df32(g, b, s, out, Ci, Ci32);
    if (bad) atomicAdd(flag, 1);
}

// df64 clover blocks (both 6x6 blocks of n sites' fields) rounded to FP64
__global__ void clover_f64_kernel(long long n, const df2 *__restrict__ in, double2 *out)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const df2 t = in[i];
    out[i] = make_double2((double)t.rh + (double)t.rl, (double)t.ih + (double)t.il);
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

void clover_build(const Exec &e, const void *Udf[2], double csw, double m0, void *Cdf[2], void *C32[2],
                  void *Fscratch, void *Rscratch)
{
    {
        // the field strengths in three passes (H into Fscratch, R into Rscratch,
        // F into Fscratch).  Unique bytes per site and pass: its four df64 links
        // (4 x 144), the six anti-Hermitian matrices read (6 x 72, passes 2, 3)
        // and written (6 x 72).  Flops per (site, plane): pass 1 two 3x3
        // products (2 x 198) and AH(A B^+) (3 x 12 + 3 x 48); passes 2 and 3
        // one product (198), the anti-Hermitian part of W^+ Y (3 x 12 + 3 x 24)
        // and the sum (9)
        const unsigned nb = blocks_for(6 * e.g.V, 128);
        const df2 *U0 = (const df2 *)Udf[0], *U1 = (const df2 *)Udf[1];
        {
            Launch L_(e, K_CLOVER_FIELD, (double)e.g.V * (4 * 144 + 6 * 72), (double)e.g.V * 6 * (2 * 198 + 180));
            clover_plaq_kernel<<<nb, 128, 0, e.st>>>(e.g, U0, U1, (float2 *)Fscratch);
        }
        {
            Launch L_(e, K_CLOVER_FIELD, (double)e.g.V * (4 * 144 + 2 * 6 * 72), (double)e.g.V * 6 * (198 + 117));
            clover_rot_kernel<false><<<nb, 128, 0, e.st>>>(e.g, U0, U1, (const float2 *)Fscratch, (float2 *)Rscratch,
                                                           1.0f);
        }
        {
            Launch L_(e, K_CLOVER_FIELD, (double)e.g.V * (4 * 144 + 2 * 6 * 72), (double)e.g.V * 6 * (198 + 117));
            clover_rot_kernel<true><<<nb, 128, 0, e.st>>>(e.g, U0, U1, (const float2 *)Rscratch, (float2 *)Fscratch,
                                                          0.125f);
        }
    }
    // reads the six F, writes the blocks in df64 and FP32
    Launch L_(e, K_CLOVER, (double)e.g.V * (6 * 72 + 72 * (8 + 4)));
    const double dg = 4.0 + m0, hh = 0.5 * csw;
    const float dg_hi = (float)dg, hh_hi = (float)hh;
    clover_assemble_kernel<<<blocks_for(e.g.V, 128), 128, 0, e.st>>>(
        e.g, (const float2 *)Fscratch, df64(dg_hi, (float)(dg - (double)dg_hi)), df64(hh_hi, (float)(hh - (double)hh_hi)),
        (df2 *)Cdf[0], (df2 *)Cdf[1], (float4 *)C32[0], (float4 *)C32[1]);
}

void clover_invert(const Exec &e, const void *Cdf, void *Cidf, void *Ci32, int *flag)
{
    Launch L_(e, K_CLOVER, (double)e.g.Vh * 72 * (8 + 8 + 4), (double)e.g.Vh * 2 * 1500);
    clover_invert_kernel<<<blocks_for(2 * e.g.Vh, 128), 128, 0, e.st>>>(e.g, (const df2 *)Cdf, (df2 *)Cidf,
                                                                          (float4 *)Ci32, flag);
}

void clover_to_f64(const Exec &e, const void *Cdf, void *C64)
{
    const long long n = 36LL * e.g.stride;   // two blocks of 18 complex slots
    Launch L_(e, K_LAYOUT, (double)n * 32);
    clover_f64_kernel<<<blocks_for(n, 256), 256, 0, e.st>>>(n, (const df2 *)Cdf, (double2 *)C64);
}

void df64_to_f64(const Exec &e, const void *in, void *out, long long n)
{
    Launch L_(e, K_LAYOUT, (double)n * 32);
    clover_f64_kernel<<<blocks_for(n, 256), 256, 0, e.st>>>(n, (const df2 *)in, (double2 *)out);
}

void clover_export(const Exec &e, const void *Ce, const void *Co, void *out)
{
    Launch L_(e, K_CLOVER, (double)e.g.V * (72 * 8 + 72 * 16));
    clover_export_kernel<<<blocks_for(e.g.V, 128), 128, 0, e.st>>>(e.g, (const double2 *)Ce,
                                                                  (const double2 *)Co, (double2 *)out);
}

}  // namespace lq
