// Batched (multi right-hand side, multi lattice) BLAS-1 and the device-side
// Arnoldi/Givens bookkeeping of the batched GMRES cycle.
//
// A batch holds N systems (right-hand sides, possibly of lattices of
// different sizes).  System r's field occupies vectors [off_r, off_r + len_r)
// of a "multi-field" (Segs; the uniform layout off_r = r * n, len_r = n when
// no table is given).  The Krylov basis of the batched GMRES is stored
// vector-major: basis vector j is one multi-field, the next one vjs vectors
// further, so that one batched operator launch maps V_j to V_{j+1} for every
// system.
//
// Every kernel here runs a grid (blocks, N): blockIdx.y selects the system and
// the blocks stride over its field.  Reductions keep the deterministic
// two-stage scheme of the single-right-hand-side kernels, per system.
//
// The Givens bookkeeping (Algorithm 2's least-squares problem) runs on the
// device, one thread per system, so that a whole GMRES cycle is a fixed
// sequence of launches with no host synchronisation.
#include <cmath>

#include "lq_kernels.h"

namespace lq {

static constexpr int BT = 256;

// offset and length (vectors) of system r
__device__ __forceinline__ void seg_of(const longlong2 *seg, long long n, int r, long long &off, long long &len)
{
    if (seg) {
        const longlong2 t = seg[r];
        off = t.x;
        len = t.y;
    } else {
        off = (long long)r * n;
        len = n;
    }
}

__device__ __forceinline__ float2 cdot4(float4 v, float4 w, float2 a)
{
    a.x = fmaf(v.x, w.x, fmaf(v.y, w.y, fmaf(v.z, w.z, fmaf(v.w, w.w, a.x))));
    a.y = fmaf(v.x, w.y, fmaf(-v.y, w.x, fmaf(v.z, w.w, fmaf(-v.w, w.z, a.y))));
    return a;
}

template <int N>
__device__ __forceinline__ void bsum(float v[N], float *sh)
{
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < N; i++) sh[warp * N + i] = v[i];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < N; i++) v[i] = lane < BT / 32 ? sh[lane * N + i] : 0.0f;
#pragma unroll
        for (int i = 0; i < N; i++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    }
    __syncthreads();
}

// partial[(r * gridDim.x + block) * pitch + 2 * (slot0 + j) + re/im] = block share of (v_jr, w_r)
template <int NJ>
__global__ void __launch_bounds__(BT, 4) bdot_kernel(const float4 *__restrict__ V, long long vjs,
                                                     const longlong2 *seg, long long n,
                                                     const float4 *__restrict__ w, double *partial, int pitch,
                                                     int slot0)
{
    __shared__ float sh[(BT / 32) * 2 * NJ];
    const int r = blockIdx.y;
    long long off, len;
    seg_of(seg, n, r, off, len);
    const float4 *Vr = V + off, *wr = w + off;
    float acc[2 * NJ];
#pragma unroll
    for (int i = 0; i < 2 * NJ; i++) acc[i] = 0.0f;
    for (long long i = blockIdx.x * (long long)BT + threadIdx.x; i < len; i += (long long)gridDim.x * BT) {
        const float4 wv = __ldg(wr + i);
#pragma unroll
        for (int j = 0; j < NJ; j++) {
            float2 a = make_float2(acc[2 * j], acc[2 * j + 1]);
            a = cdot4(__ldg(Vr + j * vjs + i), wv, a);
            acc[2 * j] = a.x;
            acc[2 * j + 1] = a.y;
        }
    }
    bsum<2 * NJ>(acc, sh);
    if (threadIdx.x == 0) {
        double *p = partial + ((long long)r * gridDim.x + blockIdx.x) * pitch + 2 * slot0;
#pragma unroll
        for (int j = 0; j < 2 * NJ; j++) p[j] = (double)acc[j];
    }
}

// y_r += sign * sum_j c_{r,j} v_{j,r}; with NORM also the partials of ||y_r||^2.
// Coefficients (complex doubles) for right-hand side r start at c + r * cstride.
template <bool NORM>
__global__ void __launch_bounds__(BT, 4) baxpy_kernel(const float4 *__restrict__ V, long long vjs,
                                                      const longlong2 *seg, long long n, int nv,
                                                      const double2 *__restrict__ c, int cstride, float sign,
                                                      float4 *y, double *partial, int pitch, int slot)
{
    __shared__ float csr[256], csi[256];
    __shared__ float sh[BT / 32];
    const int r = blockIdx.y;
    for (int j = threadIdx.x; j < nv; j += BT) {
        const double2 cj = c[(long long)r * cstride + j];
        csr[j] = sign * (float)cj.x;
        csi[j] = sign * (float)cj.y;
    }
    __syncthreads();
    long long off, len;
    seg_of(seg, n, r, off, len);
    const float4 *Vr = V + off;
    float4 *yr = y + off;
    float nrm[1] = {0.0f};
    for (long long i = blockIdx.x * (long long)BT + threadIdx.x; i < len; i += (long long)gridDim.x * BT) {
        float4 yv = yr[i];
        auto acc = [&](int j, const float4 v) {
            const float cr = csr[j], ci = csi[j];
            yv.x = fmaf(cr, v.x, fmaf(-ci, v.y, yv.x));
            yv.y = fmaf(cr, v.y, fmaf(ci, v.x, yv.y));
            yv.z = fmaf(cr, v.z, fmaf(-ci, v.w, yv.z));
            yv.w = fmaf(cr, v.w, fmaf(ci, v.z, yv.w));
        };
        // four basis loads in flight before their sums (the same order of sums)
        int j = 0;
        for (; j + 4 <= nv; j += 4) {
            float4 vv[4];
#pragma unroll
            for (int q = 0; q < 4; q++) vv[q] = __ldg(Vr + (j + q) * vjs + i);
#pragma unroll
            for (int q = 0; q < 4; q++) acc(j + q, vv[q]);
        }
        for (; j < nv; j++) acc(j, __ldg(Vr + j * vjs + i));
        yr[i] = yv;
        if (NORM) nrm[0] = fmaf(yv.x, yv.x, fmaf(yv.y, yv.y, fmaf(yv.z, yv.z, fmaf(yv.w, yv.w, nrm[0]))));
    }
    if (NORM) {
        bsum<1>(nrm, sh);
        if (threadIdx.x == 0) {
            double *p = partial + ((long long)r * gridDim.x + blockIdx.x) * pitch + 2 * slot;
            p[0] = (double)nrm[0];
            p[1] = 0.0;
        }
    }
}

__global__ void __launch_bounds__(BT) bnorm_kernel(const float4 *__restrict__ w, const longlong2 *seg, long long n,
                                                   double *partial, int pitch, int slot)
{
    __shared__ float sh[BT / 32];
    const int r = blockIdx.y;
    long long off, len;
    seg_of(seg, n, r, off, len);
    const float4 *wr = w + off;
    float nrm[1] = {0.0f};
    for (long long i = blockIdx.x * (long long)BT + threadIdx.x; i < len; i += (long long)gridDim.x * BT) {
        const float4 v = __ldg(wr + i);
        nrm[0] = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, nrm[0]))));
    }
    bsum<1>(nrm, sh);
    if (threadIdx.x == 0) {
        double *p = partial + ((long long)r * gridDim.x + blockIdx.x) * pitch + 2 * slot;
        p[0] = (double)nrm[0];
        p[1] = 0.0;
    }
}

// df64 norms (the outer residuals): per right-hand side, df64 accumulation
__device__ __forceinline__ df64 bshfl_df(df64 v, int o)
{
    return df64(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o));
}
__global__ void __launch_bounds__(BT) bnorm_df_kernel(const df2 *__restrict__ w, const longlong2 *seg, long long n,
                                                      double *partial, int pitch, int slot)
{
    __shared__ df64 sh[BT / 32];
    const int r = blockIdx.y;
    long long off, len;
    seg_of(seg, n, r, off, len);
    const df2 *wr = w + off;
    df64 acc = df64(0.0f, 0.0f);
    for (long long i = blockIdx.x * (long long)BT + threadIdx.x; i < len; i += (long long)gridDim.x * BT) {
        const cx<df64> v = df2_cx(ldg(wr + i));
        acc = fma(v.re, v.re, fma(v.im, v.im, acc));
    }
    for (int o = 16; o > 0; o >>= 1) acc = acc + bshfl_df(acc, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        acc = lane < BT / 32 ? sh[lane] : df64(0.0f, 0.0f);
        for (int o = 16; o > 0; o >>= 1) acc = acc + bshfl_df(acc, o);
        if (lane == 0) {
            double *p = partial + ((long long)r * gridDim.x + blockIdx.x) * pitch + 2 * slot;
            p[0] = df_to_double(acc);
            p[1] = 0.0;
        }
    }
}

// out[r * opitch + v] = sum_b partial[(r * blocks + b) * pitch + v], fixed order
__global__ void __launch_bounds__(BT) bfinish_kernel(const double *__restrict__ partial, int blocks, int pitch,
                                                     int first, double *out, int opitch)
{
    __shared__ double sh[BT / 32];
    const int r = blockIdx.y, v = first + blockIdx.x;
    double acc = 0.0;
    for (int b = threadIdx.x; b < blocks; b += BT) acc += partial[((long long)r * blocks + b) * pitch + v];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < BT / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) out[(long long)r * opitch + v] = acc;
    }
}

// y_r = s_r x_r (FP32 fields, device scale per system)
__global__ void __launch_bounds__(BT) bscale_kernel(const float4 *x, const longlong2 *seg, long long n,
                                                    const double *s, float4 *y)
{
    const int r = blockIdx.y;
    long long off, len;
    seg_of(seg, n, r, off, len);
    const float f = (float)s[r];
    for (long long i = blockIdx.x * (long long)BT + threadIdx.x; i < len; i += (long long)gridDim.x * BT) {
        float4 v = x[off + i];
        v.x *= f;
        v.y *= f;
        v.z *= f;
        v.w *= f;
        y[off + i] = v;
    }
}

// y_r = x_r - y_r (FP32 fields)
__global__ void __launch_bounds__(BT) bxmy_kernel(const float4 *__restrict__ x, const longlong2 *seg, long long n,
                                                  float4 *y)
{
    const int r = blockIdx.y;
    long long off, len;
    seg_of(seg, n, r, off, len);
    for (long long i = blockIdx.x * (long long)BT + threadIdx.x; i < len; i += (long long)gridDim.x * BT) {
        const float4 a = __ldg(x + off + i);
        float4 b = y[off + i];
        b.x = a.x - b.x;
        b.y = a.y - b.y;
        b.z = a.z - b.z;
        b.w = a.w - b.w;
        y[off + i] = b;
    }
}

// ---------------------------------------------------------------------------
// device-side Givens least squares, one thread per right-hand side
// ---------------------------------------------------------------------------
struct cdbl {
    double re, im;
};
__device__ __forceinline__ cdbl cd_mul(cdbl a, cdbl b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cdbl cd_conj(cdbl a) { return {a.re, -a.im}; }
__device__ __forceinline__ double cd_abs(cdbl a) { return hypot(a.re, a.im); }

// Start of a cycle: beta_r = sqrt(nrm2_r); g_r = beta e_1; the cycle of a
// right-hand side whose residual already meets its target (or is 0) stays
// inactive.  scale_r = 1/beta (0 when inactive).
__global__ void ks_init_kernel(int N, int m, const double *nrm2, int nstride, const double *target, double2 *g,
                               int *active, int *kused, double *scale, double *est)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const double beta = sqrt(nrm2[(long long)r * nstride]);
    for (int j = 0; j <= m; j++) g[(long long)r * (m + 1) + j] = make_double2(j == 0 ? beta : 0.0, 0.0);
    const bool on = beta > target[r] && beta > 0.0 && isfinite(beta);
    active[r] = on ? 1 : 0;
    kused[r] = 0;
    scale[r] = on ? 1.0 / beta : 0.0;
    est[r] = beta;
}

// After Arnoldi step k.  Two orthogonalisation passes (CGS2): h_jk = h1_j + h2_j
// (j <= k) from slots [0, k] and [k+1, 2k+1], ||w||^2 in slot 2k+2 of each
// right-hand side's row of `dots`; one pass (CGS): h_jk from slots [0, k] and
// ||w||^2 in slot k+1.
// Rotates the new Hessenberg column, updates g, and decides whether the cycle
// continues for this right-hand side (residual estimate above target, no
// breakdown).  scale_r = 1/h_{k+1,k} normalises the next basis vector.
__global__ void ks_step_kernel(int N, int m, int k, int passes, const double *dots, int dstride, const double *target,
                               double2 *H, double *cs, double2 *sn, double2 *g, int *active, int *kused,
                               double *scale, double *est, int *nanflag)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    if (!active[r]) {
        scale[r] = 0.0;
        return;
    }
    const double *d = dots + (long long)r * dstride;
    double2 *Hr = H + (long long)r * (m + 1) * m;   // column-major (m+1) x m
    double *csr = cs + (long long)r * m;
    double2 *snr = sn + (long long)r * m;
    double2 *gr = g + (long long)r * (m + 1);
    const double hk1 = sqrt(d[2 * (passes == 2 ? 2 * k + 2 : k + 1)]);
    double colnorm2 = hk1 * hk1;
    for (int j = 0; j <= k; j++) {
        const double re = d[2 * j] + (passes == 2 ? d[2 * (k + 1 + j)] : 0.0);
        const double im = d[2 * j + 1] + (passes == 2 ? d[2 * (k + 1 + j) + 1] : 0.0);
        Hr[(long long)k * (m + 1) + j] = make_double2(re, im);
        colnorm2 += re * re + im * im;
    }
    if (!isfinite(colnorm2)) {
        atomicAdd(nanflag, 1);
        active[r] = 0;
        scale[r] = 0.0;
        return;
    }
    // previous rotations on the new column
    for (int i = 0; i < k; i++) {
        const double2 a2 = Hr[(long long)k * (m + 1) + i], b2 = Hr[(long long)k * (m + 1) + i + 1];
        const cdbl a = {a2.x, a2.y}, b = {b2.x, b2.y}, s = {snr[i].x, snr[i].y};
        const cdbl sb = cd_mul(s, b), sca = cd_mul(cd_conj(s), a);
        Hr[(long long)k * (m + 1) + i] = make_double2(csr[i] * a.re + sb.re, csr[i] * a.im + sb.im);
        Hr[(long long)k * (m + 1) + i + 1] = make_double2(-sca.re + csr[i] * b.re, -sca.im + csr[i] * b.im);
    }
    const double2 a2 = Hr[(long long)k * (m + 1) + k];
    const cdbl a = {a2.x, a2.y}, b = {hk1, 0.0};
    const double t = sqrt(a.re * a.re + a.im * a.im + hk1 * hk1);
    double c;
    cdbl s;
    if (cd_abs(a) == 0.0) {
        c = 0.0;
        s = {1.0, 0.0};
    } else {
        const double aa = cd_abs(a);
        c = aa / t;
        s = cd_mul({a.re / aa, a.im / aa}, cd_conj(b));
        s = {s.re / t, s.im / t};
    }
    csr[k] = c;
    snr[k] = make_double2(s.re, s.im);
    const cdbl sbk = cd_mul(s, b);
    Hr[(long long)k * (m + 1) + k] = make_double2(c * a.re + sbk.re, c * a.im + sbk.im);
    Hr[(long long)k * (m + 1) + k + 1] = make_double2(0.0, 0.0);
    const cdbl gk = {gr[k].x, gr[k].y};
    const cdbl ng = cd_mul(cd_conj(s), gk);
    gr[k] = make_double2(c * gk.re, c * gk.im);
    gr[k + 1] = make_double2(-ng.re, -ng.im);
    const double e = hypot(ng.re, ng.im);
    est[r] = e;
    kused[r] = k + 1;
    const bool breakdown = hk1 <= 1e-14 * sqrt(colnorm2);
    const bool go = !breakdown && e > target[r] && k + 1 < m;
    active[r] = go ? 1 : 0;
    scale[r] = go ? 1.0 / hk1 : 0.0;
}

// y_r = R^{-1} g over the kused_r columns; zeros beyond (coefficients of x += V y)
__global__ void ks_solve_kernel(int N, int m, const double2 *H, const double2 *g, const int *kused, double2 *y,
                                int ystride)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const double2 *Hr = H + (long long)r * (m + 1) * m;
    const double2 *gr = g + (long long)r * (m + 1);
    double2 *yr = y + (long long)r * ystride;
    const int n = kused[r];
    for (int j = n; j < m; j++) yr[j] = make_double2(0.0, 0.0);
    for (int i = n - 1; i >= 0; i--) {
        cdbl acc = {gr[i].x, gr[i].y};
        for (int j = i + 1; j < n; j++) {
            const cdbl hij = {Hr[(long long)j * (m + 1) + i].x, Hr[(long long)j * (m + 1) + i].y};
            const cdbl p = cd_mul(hij, {yr[j].x, yr[j].y});
            acc.re -= p.re;
            acc.im -= p.im;
        }
        const cdbl hii = {Hr[(long long)i * (m + 1) + i].x, Hr[(long long)i * (m + 1) + i].y};
        const double den = hii.re * hii.re + hii.im * hii.im;
        const cdbl q = cd_mul(acc, cd_conj(hii));
        yr[i] = make_double2(q.re / den, q.im / den);
    }
}

// ---- launchers --------------------------------------------------------------------
static inline int bblocks(long long maxlen, int N)
{
    // about 4 blocks per SM over the whole batch, at least 16 per system, and no
    // more than the longest field needs
    long long b = (4LL * 152 + N - 1) / N;
    if (b < 16) b = 16;
    const long long need = (maxlen + BT - 1) / BT;
    return (int)(b < need ? b : need < 1 ? 1 : need);
}

void bdot(const Exec &e, const Segs &S, const void *V, long long vjs, int nv, const void *w, int N, BatchRed &br,
          int slot0)
{
    for (int j0 = 0; j0 < nv; j0 += 8) {
        const int nj = nv - j0 < 8 ? nv - j0 : 8;
        Launch L_(e, K_DOT_F32, S.sites * 96.0 * (nj + 1), S.sites * 96 * nj);
        const float4 *Vj = (const float4 *)V + j0 * vjs;
        const dim3 grid(br.blocks, N);
#define LQ_BDOT(NJ)                                                                                     \
    case NJ:                                                                                            \
        bdot_kernel<NJ><<<grid, BT, 0, e.st>>>(Vj, vjs, S.seg, S.n, (const float4 *)w, br.partial, br.pitch, \
                                               slot0 + j0);                                             \
        break;
        switch (nj) {
            LQ_BDOT(1)
            LQ_BDOT(2)
            LQ_BDOT(3)
            LQ_BDOT(4)
            LQ_BDOT(5)
            LQ_BDOT(6)
            LQ_BDOT(7)
            LQ_BDOT(8)
        }
#undef LQ_BDOT
    }
}

void baxpy(const Exec &e, const Segs &S, const void *V, long long vjs, int nv, const double *c, int cstride,
           int sign, void *y, int N, BatchRed *br, int slot)
{
    Launch L_(e, K_AXPY_F32, S.sites * 96.0 * (nv + 2), S.sites * 96 * nv);
    const int blocks = br ? br->blocks : S.blocks;
    const dim3 grid(blocks, N);
    if (br)
        baxpy_kernel<true><<<grid, BT, 0, e.st>>>((const float4 *)V, vjs, S.seg, S.n, nv, (const double2 *)c,
                                                  cstride, (float)sign, (float4 *)y, br->partial, br->pitch, slot);
    else
        baxpy_kernel<false><<<grid, BT, 0, e.st>>>((const float4 *)V, vjs, S.seg, S.n, nv, (const double2 *)c,
                                                   cstride, (float)sign, (float4 *)y, nullptr, 0, slot);
}

void bnorm(const Exec &e, int prec, const Segs &S, const void *w, int N, BatchRed &br, int slot)
{
    Launch L_(e, K_NORM, S.sites * (prec == P32 ? 96.0 : 192.0));
    const dim3 grid(br.blocks, N);
    if (prec == P32)
        bnorm_kernel<<<grid, BT, 0, e.st>>>((const float4 *)w, S.seg, S.n, br.partial, br.pitch, slot);
    else
        bnorm_df_kernel<<<grid, BT, 0, e.st>>>((const df2 *)w, S.seg, S.n, br.partial, br.pitch, slot);
}

void bfinish(const Exec &e, BatchRed &br, int N, int first, int count)
{
    if (count <= 0) return;
    Launch L_(e, K_FINISH, (double)N * br.blocks * 2 * count * 8.0);
    bfinish_kernel<<<dim3(2 * count, N), BT, 0, e.st>>>(br.partial, br.blocks, br.pitch, 2 * first, br.out,
                                                        br.pitch);
}

void bscale(const Exec &e, const Segs &S, const void *x, const double *s, void *y, int N)
{
    Launch L_(e, K_AXPY_F32, S.sites * 192.0);
    bscale_kernel<<<dim3(S.blocks, N), BT, 0, e.st>>>((const float4 *)x, S.seg, S.n, s, (float4 *)y);
}

void bxmy(const Exec &e, const Segs &S, const void *x, void *y, int N)
{
    Launch L_(e, K_AXPY_F32, S.sites * 288.0, S.sites * 24.0);
    bxmy_kernel<<<dim3(S.blocks, N), BT, 0, e.st>>>((const float4 *)x, S.seg, S.n, (float4 *)y);
}

void ks_init(const Exec &e, const KState &k, const double *nrm2, int nstride)
{
    Launch L_(e, K_FINISH, 0.0);
    ks_init_kernel<<<(k.N + 31) / 32, 32, 0, e.st>>>(k.N, k.m, nrm2, nstride, k.target, k.g, k.active, k.kused,
                                                     k.scale, k.est);
}

void ks_step(const Exec &e, const KState &k, int step, int passes, const double *dots, int dstride)
{
    Launch L_(e, K_FINISH, 0.0);
    ks_step_kernel<<<(k.N + 31) / 32, 32, 0, e.st>>>(k.N, k.m, step, passes, dots, dstride, k.target, k.H, k.cs, k.sn, k.g,
                                                     k.active, k.kused, k.scale, k.est, k.nanflag);
}

void ks_solve(const Exec &e, const KState &k)
{
    Launch L_(e, K_FINISH, 0.0);
    ks_solve_kernel<<<(k.N + 31) / 32, 32, 0, e.st>>>(k.N, k.m, k.H, k.g, k.kused, k.y, k.m);
}

int batch_blocks(long long maxlen, int N) { return bblocks(maxlen, N); }

}  // namespace lq
