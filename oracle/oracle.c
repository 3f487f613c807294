/*
 * FP64 CPU oracle for the odd-even Wilson-clover path -- TEST INFRASTRUCTURE.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg may load this library.  The product path (the CUDA library) never links,
 * loads or calls it, and the two share no code.
 *
 * Everything here is the plain definition, written out site by site in
 * complex double precision, with full 4x4 gamma matrices and full 12x12
 * clover matrices (no spin projection, no packed storage, no fusion):
 *
 *   (D psi)(x) = C(x) psi(x) - 1/2 (H psi)(x)
 *   (H psi)(x) = sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu) ]
 *   C(x)       = (4 + m0) 1 + c_sw (i/4) sum_{mu != nu} sigma_mu_nu (x) F_mu_nu(x)
 *   sigma_mu_nu = (i/2) [g_mu, g_nu]
 *   F_mu_nu(x)  = (Q_mu_nu(x) - Q_mu_nu(x)^+) / 8,  Q = sum of the four plaquette
 *                 leaves in the (mu,nu) plane that start and end at x.
 *
 * The paper (Sec. 2.3) names the operator "Wilson-Dirac with clover
 * improvement" and fixes its block structure (nine 12x12 blocks per block
 * row, Sec. 2.3; 6x6 diagonal blocks after odd-even reordering, Sec. 2.4.5)
 * but prints no formula; the textbook Sheikholeslami-Wohlert form above is the
 * reading used.  Hops that cross the time boundary are multiplied by t_bc
 * (-1: antiperiodic), space is periodic.  The gamma matrices are in the
 * chiral basis, g_k = [[0, -i s_k], [i s_k, 0]], g_4 = [[0, 1], [1, 0]],
 * so that g_5 = g_1 g_2 g_3 g_4 is diagonal and the clover term splits into
 * two 6x6 blocks (spins {0,1} and {2,3}) as the paper states.
 *
 * Layouts (natural order): site lex = x + Lx*(y + Ly*(z + Lz*t));
 * U[V][4][3][3], spinor[V][4][3], clover[V][12][12] with row/column index
 * spin*3 + colour.  All lattice extents must be even.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

/* ------------------------------------------------------------------ */
/* geometry                                                            */
/* ------------------------------------------------------------------ */

static void site_coords(const int *L, long s, int c[4])
{
    c[0] = (int)(s % L[0]); s /= L[0];
    c[1] = (int)(s % L[1]); s /= L[1];
    c[2] = (int)(s % L[2]); s /= L[2];
    c[3] = (int)s;
}

static long site_index(const int *L, const int c[4])
{
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

/* One step from site s along direction mu (0..3), dir = +1 or -1, periodic.
 * *crossed_t is set to 1 when the step wraps around the time extent. */
static long site_step(const int *L, long s, int mu, int dir, int *crossed_t)
{
    int c[4];
    site_coords(L, s, c);
    int v = c[mu] + dir;
    int wrapped = 0;
    if (v < 0) { v += L[mu]; wrapped = 1; }
    if (v >= L[mu]) { v -= L[mu]; wrapped = 1; }
    c[mu] = v;
    if (crossed_t) *crossed_t = (mu == 3) && wrapped;
    return site_index(L, c);
}

/* Paper Sec. 2.4.5: a site is even iff x1 + x2 + x3 + x4 is even. */
int orc_parity(const int *L, long s)
{
    int c[4];
    site_coords(L, s, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* ------------------------------------------------------------------ */
/* gamma matrices (chiral basis)                                       */
/* ------------------------------------------------------------------ */

static void pauli(int k, cplx p[2][2])
{
    memset(p, 0, 4 * sizeof(cplx));
    if (k == 0) { p[0][1] = 1; p[1][0] = 1; }
    if (k == 1) { p[0][1] = -I; p[1][0] = I; }
    if (k == 2) { p[0][0] = 1; p[1][1] = -1; }
}

static void mat4_mul(const cplx *A, const cplx *B, cplx *C)
{
    cplx T[16];
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            cplx acc = 0;
            for (int k = 0; k < 4; k++) acc += A[i * 4 + k] * B[k * 4 + j];
            T[i * 4 + j] = acc;
        }
    memcpy(C, T, sizeof T);
}

/* g[4][4] for mu = 0,1,2 (gamma_1..3), 3 (gamma_4) and 4 (gamma_5). */
void orc_gamma(int mu, cplx *g)
{
    memset(g, 0, 16 * sizeof(cplx));
    if (mu < 3) {
        cplx p[2][2];
        pauli(mu, p);
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) {
                g[a * 4 + (2 + b)] = -I * p[a][b];
                g[(2 + a) * 4 + b] = I * p[a][b];
            }
    } else if (mu == 3) {
        for (int a = 0; a < 2; a++) { g[a * 4 + 2 + a] = 1; g[(2 + a) * 4 + a] = 1; }
    } else {
        cplx g1[16], g2[16], g3[16], g4[16];
        orc_gamma(0, g1); orc_gamma(1, g2); orc_gamma(2, g3); orc_gamma(3, g4);
        mat4_mul(g1, g2, g);
        mat4_mul(g, g3, g);
        mat4_mul(g, g4, g);
    }
}

/* ------------------------------------------------------------------ */
/* colour algebra                                                      */
/* ------------------------------------------------------------------ */

static const cplx *link(const cplx *U, long s, int mu) { return U + (s * 4 + mu) * 9; }

static void m3_mul(const cplx *A, const cplx *B, cplx *C)
{
    cplx T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx acc = 0;
            for (int k = 0; k < 3; k++) acc += A[i * 3 + k] * B[k * 3 + j];
            T[i * 3 + j] = acc;
        }
    memcpy(C, T, sizeof T);
}

static void m3_dag(const cplx *A, cplx *B)
{
    cplx T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) T[i * 3 + j] = conj(A[j * 3 + i]);
    memcpy(B, T, sizeof T);
}

/* ------------------------------------------------------------------ */
/* hopping term                                                        */
/* ------------------------------------------------------------------ */

/* out[12] = (H psi)(x), the sum of the eight nearest-neighbour hops into x. */
static void hop_site(const int *L, int tbc, const cplx *U, const cplx *psi, long x,
                     const cplx G[4][16], cplx *out)
{
    for (int i = 0; i < 12; i++) out[i] = 0;
    for (int mu = 0; mu < 4; mu++) {
        for (int dir = +1; dir >= -1; dir -= 2) {
            int crossed = 0;
            long y = site_step(L, x, mu, dir, &crossed);
            double sign = crossed ? (double)tbc : 1.0;
            /* colour: W = U_mu(x) psi(y) forward, U_mu(y)^+ psi(y) backward */
            cplx Um[9];
            if (dir > 0) memcpy(Um, link(U, x, mu), sizeof Um);
            else m3_dag(link(U, y, mu), Um);
            const cplx *p = psi + y * 12;
            cplx W[12];
            for (int s = 0; s < 4; s++)
                for (int a = 0; a < 3; a++) {
                    cplx acc = 0;
                    for (int b = 0; b < 3; b++) acc += Um[a * 3 + b] * p[s * 3 + b];
                    W[s * 3 + a] = acc;
                }
            /* spin: (1 - g_mu) forward, (1 + g_mu) backward */
            for (int s = 0; s < 4; s++)
                for (int a = 0; a < 3; a++) {
                    cplx acc = W[s * 3 + a];
                    for (int t = 0; t < 4; t++) acc -= (double)dir * G[mu][s * 4 + t] * W[t * 3 + a];
                    out[s * 3 + a] += sign * acc;
                }
        }
    }
}

static void load_gammas(cplx G[4][16])
{
    for (int mu = 0; mu < 4; mu++) orc_gamma(mu, G[mu]);
}

/* out(x) = (H in)(x) at every site of the given parity (0 even, 1 odd, -1 all);
 * out is zero at the other sites.  in and out are [V][12]. */
void orc_hop(const int *L, int tbc, const cplx *U, const cplx *in, cplx *out, int parity)
{
    long V = (long)L[0] * L[1] * L[2] * L[3];
    cplx G[4][16];
    load_gammas(G);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; x++) {
        if (parity >= 0 && orc_parity(L, x) != parity) {
            for (int i = 0; i < 12; i++) out[x * 12 + i] = 0;
            continue;
        }
        hop_site(L, tbc, U, in, x, G, out + x * 12);
    }
}

/* ------------------------------------------------------------------ */
/* clover term                                                         */
/* ------------------------------------------------------------------ */

/* Q_mu_nu(x): the four same-orientation plaquette leaves that start and end
 * at x (steps +mu,+nu,-mu,-nu and the three rotations into the other
 * quadrants), summed. */
static void clover_leaves(const int *L, const cplx *U, long x, int mu, int nu, cplx *Q)
{
    long xpm = site_step(L, x, mu, +1, 0), xpn = site_step(L, x, nu, +1, 0);
    long xmm = site_step(L, x, mu, -1, 0), xmn = site_step(L, x, nu, -1, 0);
    long xmm_pn = site_step(L, xmm, nu, +1, 0);
    long xmm_mn = site_step(L, xmm, nu, -1, 0);
    long xmn_pm = site_step(L, xmn, mu, +1, 0);
    cplx A[9], B[9], T[9];
    for (int i = 0; i < 9; i++) Q[i] = 0;

    /* leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ */
    m3_mul(link(U, x, mu), link(U, xpm, nu), T);
    m3_dag(link(U, xpn, mu), A); m3_mul(T, A, T);
    m3_dag(link(U, x, nu), A);   m3_mul(T, A, T);
    for (int i = 0; i < 9; i++) Q[i] += T[i];

    /* leaf 2: U_nu(x) U_mu(x-mu+nu)^+ U_nu(x-mu)^+ U_mu(x-mu) */
    m3_dag(link(U, xmm_pn, mu), A); m3_mul(link(U, x, nu), A, T);
    m3_dag(link(U, xmm, nu), A);    m3_mul(T, A, T);
    m3_mul(T, link(U, xmm, mu), T);
    for (int i = 0; i < 9; i++) Q[i] += T[i];

    /* leaf 3: U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu) */
    m3_dag(link(U, xmm, mu), A); m3_dag(link(U, xmm_mn, nu), B); m3_mul(A, B, T);
    m3_mul(T, link(U, xmm_mn, mu), T);
    m3_mul(T, link(U, xmn, nu), T);
    for (int i = 0; i < 9; i++) Q[i] += T[i];

    /* leaf 4: U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+ */
    m3_dag(link(U, xmn, nu), A); m3_mul(A, link(U, xmn, mu), T);
    m3_mul(T, link(U, xmn_pm, nu), T);
    m3_dag(link(U, x, mu), A);   m3_mul(T, A, T);
    for (int i = 0; i < 9; i++) Q[i] += T[i];
}

/* The full 12x12 clover matrix C(x) (row/column index spin*3 + colour). */
static void clover_site(const int *L, const cplx *U, double csw, double m0, long x,
                        const cplx G[4][16], cplx *C)
{
    for (int i = 0; i < 144; i++) C[i] = 0;
    for (int i = 0; i < 12; i++) C[i * 12 + i] = 4.0 + m0;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = 0; nu < 4; nu++) {
            if (mu == nu) continue;
            /* F_mu_nu = (Q - Q^+)/8 (Q_nu_mu = Q_mu_nu^+ gives F_nu_mu = -F_mu_nu) */
            cplx Q[9], Qd[9], F[9];
            clover_leaves(L, U, x, mu, nu, Q);
            m3_dag(Q, Qd);
            for (int i = 0; i < 9; i++) F[i] = (Q[i] - Qd[i]) / 8.0;
            /* sigma_mu_nu = (i/2)(g_mu g_nu - g_nu g_mu) */
            cplx gg[16], hh[16], sig[16];
            mat4_mul(G[mu], G[nu], gg);
            mat4_mul(G[nu], G[mu], hh);
            for (int i = 0; i < 16; i++) sig[i] = 0.5 * I * (gg[i] - hh[i]);
            cplx coef = csw * 0.25 * I;
            for (int s = 0; s < 4; s++)
                for (int t = 0; t < 4; t++)
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++)
                            C[(s * 3 + a) * 12 + (t * 3 + b)] += coef * sig[s * 4 + t] * F[a * 3 + b];
        }
}

/* C[V][144] at every site. */
void orc_clover(const int *L, const cplx *U, double csw, double m0, cplx *C)
{
    long V = (long)L[0] * L[1] * L[2] * L[3];
    cplx G[4][16];
    load_gammas(G);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; x++) clover_site(L, U, csw, m0, x, G, C + x * 144);
}

/* C[n][144] at the listed sites. */
void orc_clover_sites(const int *L, const cplx *U, double csw, double m0, long n,
                      const long *sites, cplx *C)
{
    cplx G[4][16];
    load_gammas(G);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) clover_site(L, U, csw, m0, sites[i], G, C + i * 144);
}

/* ------------------------------------------------------------------ */
/* dense inverse: Gauss-Jordan elimination with partial pivoting       */
/* ------------------------------------------------------------------ */

/* Ainv = A^{-1} for one n x n row-major matrix (n <= 12).  Returns 0, or 1
 * when a pivot vanishes. */
static int invert_one(int n, const cplx *A, cplx *Ainv)
{
    cplx M[12 * 24];
    int w = 2 * n;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            M[i * w + j] = A[i * n + j];
            M[i * w + n + j] = (i == j) ? 1.0 : 0.0;
        }
    for (int col = 0; col < n; col++) {
        int piv = col;
        for (int r = col + 1; r < n; r++)
            if (cabs(M[r * w + col]) > cabs(M[piv * w + col])) piv = r;
        if (cabs(M[piv * w + col]) == 0.0) return 1;
        if (piv != col)
            for (int j = 0; j < w; j++) {
                cplx t = M[col * w + j]; M[col * w + j] = M[piv * w + j]; M[piv * w + j] = t;
            }
        cplx inv = 1.0 / M[col * w + col];
        for (int j = 0; j < w; j++) M[col * w + j] *= inv;
        for (int r = 0; r < n; r++) {
            if (r == col) continue;
            cplx f = M[r * w + col];
            if (f == 0) continue;
            for (int j = 0; j < w; j++) M[r * w + j] -= f * M[col * w + j];
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) Ainv[i * n + j] = M[i * w + n + j];
    return 0;
}

/* Invert `count` consecutive n x n matrices; returns the number that failed. */
long orc_invert(long count, int n, const cplx *A, cplx *Ainv)
{
    long bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (long i = 0; i < count; i++) bad += invert_one(n, A + i * n * n, Ainv + i * n * n);
    return bad;
}

/* ------------------------------------------------------------------ */
/* site-diagonal (clover) apply                                        */
/* ------------------------------------------------------------------ */

/* out(x) = M(x) in(x) for the 12x12 matrices M[V][144], at sites of the given
 * parity (-1: all); out is zero elsewhere. */
void orc_block(const int *L, const cplx *M, const cplx *in, cplx *out, int parity)
{
    long V = (long)L[0] * L[1] * L[2] * L[3];
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; x++) {
        if (parity >= 0 && orc_parity(L, x) != parity) {
            for (int i = 0; i < 12; i++) out[x * 12 + i] = 0;
            continue;
        }
        for (int i = 0; i < 12; i++) {
            cplx acc = 0;
            for (int j = 0; j < 12; j++) acc += M[x * 144 + i * 12 + j] * in[x * 12 + j];
            out[x * 12 + i] = acc;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Schur complement at sampled even sites (for large-lattice checks)   */
/* ------------------------------------------------------------------ */

/* (D_S x_e)(x) at n listed even sites, Eq. 3:  D_ee x_e - D_eo D_oo^{-1} D_oe x_e,
 * with every ingredient evaluated only where the listed outputs need it.
 * xfull[V][12] holds x_e at even sites (odd entries ignored); tscratch[V][12]
 * is caller-provided scratch, zero on entry and returned zero. */
long orc_schur_sites(const int *L, int tbc, const cplx *U, double csw, double m0,
                     const cplx *xfull, long n, const long *sites, cplx *out,
                     cplx *tscratch)
{
    cplx G[4][16];
    load_gammas(G);
    long bad = 0;
    long V = (long)L[0] * L[1] * L[2] * L[3];
    cplx *xe = (cplx *)calloc((size_t)V * 12, sizeof(cplx));
    for (long s = 0; s < V; s++)
        if (orc_parity(L, s) == 0) memcpy(xe + s * 12, xfull + s * 12, 12 * sizeof(cplx));
    for (long i = 0; i < n; i++) {
        long x = sites[i];
        long nb[8];
        int k = 0;
        for (int mu = 0; mu < 4; mu++) {
            nb[k++] = site_step(L, x, mu, +1, 0);
            nb[k++] = site_step(L, x, mu, -1, 0);
        }
        /* t_o = D_oo^{-1} D_oe x_e at the odd neighbours */
        for (int j = 0; j < 8; j++) {
            long y = nb[j];
            cplx h[12], Cy[144], Ci[144];
            hop_site(L, tbc, U, xe, y, G, h);
            clover_site(L, U, csw, m0, y, G, Cy);
            bad += invert_one(12, Cy, Ci);
            for (int r = 0; r < 12; r++) {
                cplx acc = 0;
                for (int c = 0; c < 12; c++) acc += Ci[r * 12 + c] * (-0.5 * h[c]);
                tscratch[y * 12 + r] = acc;
            }
        }
        cplx h[12], Cx[144];
        hop_site(L, tbc, U, tscratch, x, G, h);
        clover_site(L, U, csw, m0, x, G, Cx);
        for (int r = 0; r < 12; r++) {
            cplx acc = 0;
            for (int c = 0; c < 12; c++) acc += Cx[r * 12 + c] * xe[x * 12 + c];
            out[i * 12 + r] = acc - (-0.5 * h[r]);
        }
        for (int j = 0; j < 8; j++) memset(tscratch + nb[j] * 12, 0, 12 * sizeof(cplx));
    }
    free(xe);
    return bad;
}

/* number of OpenMP threads the oracle runs with */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
