// Fermion force on the device: the gradient of the bilinear form
//   b(U) = Re( Y^+ D(U) X )
// with respect to every link, for full-lattice fields X and Y.  For the
// pseudofermion action S = phi^+ (D^+ D)^{-1} phi with X = (D^+ D)^{-1} phi and
// Y = D X, varying U gives dS = -2 Re(Y^+ dD X), so dS/dU = -2 grad b.  The
// paper has no force; the operator is the Wilson-clover D of Sec. 2.3.
//
// Convention: G = db/dRe U + i db/dIm U, so that db = Re sum conj(G) dU.
// For b = Re tr(U M) the gradient is M^+; for b = Re tr(U^+ M) it is M.
//
// Hopping term.  U_mu(x) enters row x as -1/2 s (1 - g_mu) U psi(x+mu) and row
// x+mu as -1/2 s (1 + g_mu) U^+ psi(x), s the fermion time-boundary sign:
//   G_hop(x, mu) = -1/2 s sum_spin [ Y(x) (P- X(x+mu))^+ + (P+ X(x)) Y(x+mu)^+ ]
// with colour outer products and P-+ = 1 -+ g_mu.
//
// Clover term.  C = (4 + m0) + c_sw (i/2) sum_{mu<nu} sigma_mu_nu F_mu_nu with
// F = (Q - Q^+)/8, so
//   Re(Y^+ C X) = const + sum_y sum_{mu<nu} Re tr( Q_mu_nu(y) Gam_mu_nu(y) ),
//   Gam = (i c_sw / 16)(Lam + Lam^+),  Lam_mu_nu = sum_{s,s'} sigma_mu_nu[s][s'] X_s' Y_s^+
// (colour matrices).  In the chiral basis sigma_jk = -eps_jkl diag(s_l, s_l)
// and sigma_j4 = diag(s_j, -s_j), so with, per chirality block (spins 0,1 and
// 2,3), u_1 = X_1 Y_0^+ + X_0 Y_1^+, u_2 = i (X_0 Y_1^+ - X_1 Y_0^+),
// u_3 = X_0 Y_0^+ - X_1 Y_1^+ (upper block u, lower block l):
//   Lam_xy = -(u_3 + l_3), Lam_xz = u_2 + l_2, Lam_yz = -(u_1 + l_1),
//   Lam_xt = u_1 - l_1,    Lam_yt = u_2 - l_2, Lam_zt = u_3 - l_3.
// A link U_mu(x) is a factor f_k of eight leaves of each of the three planes
// that contain mu; for each such leaf of Q(y), with M = f_{k+1}..f_3 Gam(y)
// f_0..f_{k-1} the rest of the loop, G += M^+ (U enters as U) or M (as U^+).
//
// Arithmetic is df64 (FP64-accurate on the FP32 units) throughout.
#include "leaves.cuh"
#include "lq_kernels.h"

namespace lq {

// gamma_mu psi: component s is i^k[mu][s] psi_perm[mu][s] (chiral basis)
__constant__ unsigned char c_gperm[4][4] = {{3, 2, 1, 0}, {3, 2, 1, 0}, {2, 3, 0, 1}, {2, 3, 0, 1}};
__constant__ unsigned char c_gipow[4][4] = {{3, 3, 1, 1}, {2, 0, 0, 2}, {3, 1, 1, 3}, {0, 0, 0, 0}};
// plane number of (mu, nu), mu < nu, in the numbering of leaves.cuh
__constant__ signed char c_plane[16] = {-1, 0, 1, 3, -1, -1, 2, 4, -1, -1, -1, 5, -1, -1, -1, -1};

__device__ __forceinline__ cx<df64> times_ipow(cx<df64> v, int k)
{
    switch (k & 3) {
    case 0: return v;
    case 1: return ti(v);
    case 2: return -v;
    default: return tmi(v);
    }
}

__device__ __forceinline__ cx<df64> ld_comp(const df2 *__restrict__ f, long long stride, int comp, long long cb)
{
    return df2_cx(ldg(f + (long long)comp * stride + cb));
}

// Gam of the six planes at one site per thread, from X(x) and Y(x)
__global__ void __launch_bounds__(128) force_insertion_kernel(Geom g, const df2 *__restrict__ Xe,
                                                              const df2 *__restrict__ Xo,
                                                              const df2 *__restrict__ Ye,
                                                              const df2 *__restrict__ Yo, double csw, float2 *Gam)
{
    const long long lex = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (lex >= g.V) return;
    int c[4];
    lex_coords(g, lex, c);
    const int parity = (c[0] + c[1] + c[2] + c[3]) & 1;
    const long long cb = lex >> 1;
    const df2 *X = parity ? Xo : Xe, *Y = parity ? Yo : Ye;
    const df64 k16(csw / 16.0);
#pragma unroll 1
    for (int l = 1; l <= 3; l++) {
        // H_block = u_l + u_l^+ for the upper (blk 0) and lower (blk 1) chirality
        M3<df64> H[2];
#pragma unroll 1
        for (int blk = 0; blk < 2; blk++) {
            cx<df64> x0[3], x1[3], y0[3], y1[3];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                x0[a] = ld_comp(X, g.stride, (2 * blk) * 3 + a, cb);
                x1[a] = ld_comp(X, g.stride, (2 * blk + 1) * 3 + a, cb);
                y0[a] = ld_comp(Y, g.stride, (2 * blk) * 3 + a, cb);
                y1[a] = ld_comp(Y, g.stride, (2 * blk + 1) * 3 + a, cb);
            }
            M3<df64> u;
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = 0; b < 3; b++) {
                    // entry (a, b) of X_s' Y_s^+ is X_s'[a] conj(Y_s[b])
                    const cx<df64> p10 = cmulc(y0[b], x1[a]), p01 = cmulc(y1[b], x0[a]);
                    cx<df64> v;
                    if (l == 1) v = p10 + p01;
                    else if (l == 2) v = ti(p01 - p10);
                    else v = cmulc(y0[b], x0[a]) - cmulc(y1[b], x1[a]);
                    u.a[a * 3 + b] = v;
                }
            H[blk] = u;
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = 0; b < 3; b++) H[blk].a[a * 3 + b] = u.a[a * 3 + b] + cconj(u.a[b * 3 + a]);
        }
        // the two planes built from l: (space plane, time plane) with the space
        // sign: l = 1 -> (yz, -; xt), l = 2 -> (xz, +; yt), l = 3 -> (xy, -; zt)
        const int ps = l == 1 ? 2 : l == 2 ? 1 : 0, pt = l == 1 ? 3 : l == 2 ? 4 : 5;
#pragma unroll 1
        for (int q = 0; q < 2; q++) {
            const int p = q == 0 ? ps : pt;
            const bool neg = q == 0 && l != 2;
            df64 v[9];
            auto h = [&](int a, int b) {
                cx<df64> t = q == 0 ? H[0].a[a * 3 + b] + H[1].a[a * 3 + b] : H[0].a[a * 3 + b] - H[1].a[a * 3 + b];
                return neg ? -t : t;
            };
            // Gam = i (c_sw/16) Hm: Im Gam_aa = (c_sw/16) Re Hm_aa; Gam_ab = i (c_sw/16) Hm_ab
#pragma unroll
            for (int a = 0; a < 3; a++) v[a] = k16 * h(a, a).re;
            const cx<df64> g01 = ti(h(0, 1)), g02 = ti(h(0, 2)), g12 = ti(h(1, 2));
            v[3] = k16 * g01.re;
            v[4] = k16 * g01.im;
            v[5] = k16 * g02.re;
            v[6] = k16 * g02.im;
            v[7] = k16 * g12.re;
            v[8] = k16 * g12.im;
            store_antiherm(Gam, g.V, lex, p, v);
        }
    }
}

// G(x, mu) for one (site, direction) per thread; mu is uniform across a warp
// except at the seams of the four direction ranges.
__global__ void __launch_bounds__(128) force_link_kernel(Geom g, const df2 *__restrict__ Ue,
                                                         const df2 *__restrict__ Uo, const df2 *__restrict__ Xe,
                                                         const df2 *__restrict__ Xo, const df2 *__restrict__ Ye,
                                                         const df2 *__restrict__ Yo, const float2 *__restrict__ Gam,
                                                         double coef, double2 *G)
{
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= 4 * g.V) return;
    const int mu = (int)(id / g.V);
    const long long lex = id - mu * g.V;
    int c[4];
    lex_coords(g, lex, c);
    const int parity = (c[0] + c[1] + c[2] + c[3]) & 1;
    int cn[4] = {c[0], c[1], c[2], c[3]};
    cn[mu] = cn[mu] + 1 == g.L[mu] ? 0 : cn[mu] + 1;
    const long long cb = lex >> 1, cbn = lex_of(g, cn) >> 1;
    const df2 *Xx = parity ? Xo : Xe, *Yx = parity ? Yo : Ye;      // at x
    const df2 *Xn = parity ? Xe : Xo, *Yn = parity ? Ye : Yo;      // at x + mu
    const df64 z(0.0f, 0.0f);

    M3<df64> acc;
#pragma unroll
    for (int k = 0; k < 9; k++) acc.a[k] = {z, z};

    // ---- hopping term: sum_s Y_s(x) (P- X(x+mu))_s^+ + (P+ X(x))_s Y_s(x+mu)^+ ----
    {
        M3<df64> hop;
#pragma unroll
        for (int k = 0; k < 9; k++) hop.a[k] = {z, z};
#pragma unroll 1
        for (int s = 0; s < 4; s++) {
            const int sp = c_gperm[mu][s], ip = c_gipow[mu][s];
            cx<df64> ya[3], w[3];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                ya[a] = ld_comp(Yx, g.stride, s * 3 + a, cb);
                w[a] = ld_comp(Xn, g.stride, s * 3 + a, cbn) -
                       times_ipow(ld_comp(Xn, g.stride, sp * 3 + a, cbn), ip);   // (1 - g_mu) X(x+mu)
            }
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = 0; b < 3; b++) hop.a[a * 3 + b] = hop.a[a * 3 + b] + cmulc(w[b], ya[a]);
#pragma unroll
            for (int a = 0; a < 3; a++) {
                ya[a] = ld_comp(Yn, g.stride, s * 3 + a, cbn);
                w[a] = ld_comp(Xx, g.stride, s * 3 + a, cb) +
                       times_ipow(ld_comp(Xx, g.stride, sp * 3 + a, cb), ip);    // (1 + g_mu) X(x)
            }
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int b = 0; b < 3; b++) hop.a[a * 3 + b] = hop.a[a * 3 + b] + cmulc(ya[b], w[a]);
        }
        const bool wrap = mu == 3 && c[3] == g.L[3] - 1;
        const df64 f = df64((wrap && g.tbc < 0) ? 0.5f : -0.5f, 0.0f);
#pragma unroll
        for (int k = 0; k < 9; k++) acc.a[k] = f * hop.a[k];
    }

    // ---- clover term: the 24 leaves that contain U_mu(x) ----
#pragma unroll 1
    for (int q = 0; q < 3; q++) {
        const int nu = q < mu ? q : q + 1;
        const int pmu = mu < nu ? mu : nu, pnu = mu < nu ? nu : mu;
        const int p = c_plane[pmu * 4 + pnu];
        const unsigned char along_nu = mu == pnu;
#pragma unroll 1
        for (int f = 0; f < 16; f++) {
            if (c_lnu[f] != along_nu) continue;
            const int leaf = f >> 2, kf = f & 3;
            // the leaf starts at y = x - offset(f)
            int y[4] = {c[0], c[1], c[2], c[3]};
            y[pmu] = (y[pmu] - c_ldmu[f] + 2 * g.L[pmu]) % g.L[pmu];
            y[pnu] = (y[pnu] - c_ldnu[f] + 2 * g.L[pnu]) % g.L[pnu];
            M3<df64> T;
#pragma unroll 1
            for (int j = 1; j <= 4; j++) {
                const int slot = kf + j;   // 0..3: factors of the leaf, 4: Gam(y), 5..: wrap to factor 0
                M3<df64> Fj;
                if (slot == 4) {
                    Fj = load_antiherm(Gam, g.V, lex_of(g, y), p);
                } else {
                    const int ff = 4 * leaf + (slot < 4 ? slot : slot - 5);
                    int cc[4] = {y[0], y[1], y[2], y[3]};
                    cc[pmu] = (cc[pmu] + c_ldmu[ff] + g.L[pmu]) % g.L[pmu];
                    cc[pnu] = (cc[pnu] + c_ldnu[ff] + g.L[pnu]) % g.L[pnu];
                    Fj = link_at<df64>(g, Ue, Uo, cc, c_lnu[ff] ? pnu : pmu);
                    if (c_ldag[ff]) Fj = dagger(Fj);
                }
                T = j == 1 ? Fj : mat_mul(T, Fj);
            }
            if (c_ldag[f]) {
#pragma unroll
                for (int k = 0; k < 9; k++) acc.a[k] = acc.a[k] + T.a[k];
            } else {
#pragma unroll
                for (int a = 0; a < 3; a++)
#pragma unroll
                    for (int b = 0; b < 3; b++) acc.a[a * 3 + b] = acc.a[a * 3 + b] + cconj(T.a[b * 3 + a]);
            }
        }
    }

    double2 *o = G + (lex * 4 + mu) * 9;
#pragma unroll
    for (int k = 0; k < 9; k++)
        o[k] = make_double2(coef * df_to_double(acc.a[k].re), coef * df_to_double(acc.a[k].im));
}

// out = g5 in on natural full spinors [V][4][3] complex double (spins 2, 3 negated)
__global__ void gamma5_nat_kernel(long long V, const double2 *in, double2 *out)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= V * 12) return;
    const double2 v = in[i];
    out[i] = ((i % 12) >= 6) ? make_double2(-v.x, -v.y) : v;
}

static inline unsigned blocks_of(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

void force_insertion(const Exec &e, const void *X[2], const void *Y[2], double csw, void *Gam)
{
    // reads X, Y (2 x 192 B df64), writes six anti-Hermitian 3x3 (6 x 72 B);
    // per site 6 blocks x (2 x 9 products + 9 additions) and the Hermitian parts
    Launch L_(e, K_FORCE, (double)e.g.V * (2 * 192 + 6 * 72), (double)e.g.V * 3 * 2 * (18 * 6 + 18 * 2 + 18 * 2));
    force_insertion_kernel<<<blocks_of(e.g.V, 128), 128, 0, e.st>>>(
        e.g, (const df2 *)X[0], (const df2 *)X[1], (const df2 *)Y[0], (const df2 *)Y[1], csw, (float2 *)Gam);
}

void force_links(const Exec &e, const void *Udf[2], const void *X[2], const void *Y[2], const void *Gam,
                 double coef, void *G)
{
    // unique bytes per site: 4 df64 links, X and Y, six Gam, the 4 gradients
    // (c128); per (site, mu): 24 leaves x 3 complex 3x3 products of 198 flops
    // and their sum, plus the hopping term's 2 x 4 x 9 outer-product entries
    Launch L_(e, K_FORCE, (double)e.g.V * (4 * 144 + 2 * 192 + 6 * 72 + 4 * 144),
              (double)e.g.V * 4 * (24 * (3 * 198 + 18) + 2 * 4 * (9 * 8 + 12)));
    force_link_kernel<<<blocks_of(4 * e.g.V, 128), 128, 0, e.st>>>(
        e.g, (const df2 *)Udf[0], (const df2 *)Udf[1], (const df2 *)X[0], (const df2 *)X[1], (const df2 *)Y[0],
        (const df2 *)Y[1], (const float2 *)Gam, coef, (double2 *)G);
}

void gamma5_nat(const Exec &e, const void *in, void *out)
{
    Launch L_(e, K_LAYOUT, (double)e.g.V * 2 * 192);
    gamma5_nat_kernel<<<blocks_of(e.g.V * 12, 256), 256, 0, e.st>>>(e.g.V, (const double2 *)in, (double2 *)out);
}

}  // namespace lq
