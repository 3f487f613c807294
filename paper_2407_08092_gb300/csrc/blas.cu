// BLAS-1 steps and deterministic reductions on internal spinor fields.
//
// A field of one parity is, in memory, one linear array of 16-byte vectors
// (6 * stride float4 in FP32, 12 * stride double2 / df2 in FP64 / df64).  The
// context zero-fills every field when it allocates it and no kernel writes the
// padding sites (cb >= V/2), so these kernels simply sweep the whole array:
// fully coalesced, no per-site index arithmetic, the padding contributing 0.
//
// Reductions are two-stage and deterministic: a fixed grid (set by the
// lattice size alone) writes one partial per block and value, then one block
// per value sums the partials in a fixed tree order in FP64.  Dot products are
// (v, w) = sum conj(v) w, the inner product of Algorithm 2.
#include "lq_kernels.h"

namespace lq {

static constexpr int RT = 256;   // threads of reduction / BLAS blocks
static constexpr int MAXJ = 8;   // vectors per multi-dot launch

int reduction_blocks(const Geom &g)
{
    long long b = (g.Vh + RT - 1) / RT;
    return (int)(b < 608 ? b : 608);
}

template <typename R>
struct Vec;
template <>
struct Vec<double> {
    typedef double2 V;
    static constexpr int N = 12;   // vectors per site
};
template <>
struct Vec<float> {
    typedef float4 V;
    static constexpr int N = 6;
};

// dot / axpy / norm on one 16-byte vector (1 complex in FP64, 2 in FP32)
__device__ __forceinline__ void cdot_acc(const double2 v, const double2 w, double &re, double &im)
{
    re = fma(v.x, w.x, fma(v.y, w.y, re));
    im = fma(v.x, w.y, fma(-v.y, w.x, im));
}
__device__ __forceinline__ void cdot_acc(const float4 v, const float4 w, float &re, float &im)
{
    re = fmaf(v.x, w.x, fmaf(v.y, w.y, fmaf(v.z, w.z, fmaf(v.w, w.w, re))));
    im = fmaf(v.x, w.y, fmaf(-v.y, w.x, fmaf(v.z, w.w, fmaf(-v.w, w.z, im))));
}
__device__ __forceinline__ void caxpy(double cr, double ci, const double2 v, double2 &y)
{
    y.x = fma(cr, v.x, fma(-ci, v.y, y.x));
    y.y = fma(cr, v.y, fma(ci, v.x, y.y));
}
__device__ __forceinline__ void caxpy(float cr, float ci, const float4 v, float4 &y)
{
    y.x = fmaf(cr, v.x, fmaf(-ci, v.y, y.x));
    y.y = fmaf(cr, v.y, fmaf(ci, v.x, y.y));
    y.z = fmaf(cr, v.z, fmaf(-ci, v.w, y.z));
    y.w = fmaf(cr, v.w, fmaf(ci, v.z, y.w));
}
__device__ __forceinline__ double nrm_acc(const double2 v, double a) { return fma(v.x, v.x, fma(v.y, v.y, a)); }
__device__ __forceinline__ float nrm_acc(const float4 v, float a)
{
    return fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, a))));
}

// sum over a block of N values held per thread; the result is valid in thread 0
template <typename A, int N>
__device__ __forceinline__ void block_sum(A v[N], A *sh /* [RT/32][N] */)
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
        for (int i = 0; i < N; i++) v[i] = lane < RT / 32 ? sh[lane * N + i] : A(0);
#pragma unroll
        for (int i = 0; i < N; i++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    }
    __syncthreads();
}

// The last block of a launch to finish (counted on `ticket`, which it resets to
// zero) sums the blocks' partials of `nval` values from value index v0 in a
// fixed order (warp w takes values w, w + 8, ..., each lane the blocks lane,
// lane + 32, ...), scales value v by scale[v / 2] when a scale is given, and
// writes them to out[v]: a deterministic second stage without a second launch.
__device__ __forceinline__ void last_block_finish(double *partial, int pitch, int v0, int nval,
                                                  const double *scale, double *out, unsigned *ticket)
{
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = v0 + warp; v < v0 + nval; v += RT / 32) {
        double a = 0.0;
        for (int b = lane; b < gridDim.x; b += 32) a += __ldcg(partial + (long long)b * pitch + v);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) out[v] = scale ? a * scale[v >> 1] : a;
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

// ---- multi-dot: partial[blk][2*(slot0+j) + re/im] = block share of (v_j, w) ------
// (FIN: the last block also finishes the launch's values into out)
template <typename R, int NJ, bool FIN = false>
__global__ void __launch_bounds__(RT, 4) multi_dot_kernel(const typename Vec<R>::V *__restrict__ Vb, long long n,
                                                          const typename Vec<R>::V *__restrict__ w, double *partial,
                                                          int pitch, int slot0, const double *scale = nullptr,
                                                          double *out = nullptr, unsigned *ticket = nullptr)
{
    __shared__ R sh[(RT / 32) * 2 * NJ];
    R acc[2 * NJ];
#pragma unroll
    for (int i = 0; i < 2 * NJ; i++) acc[i] = R(0);
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        const auto wv = __ldg(w + i);
#pragma unroll
        for (int j = 0; j < NJ; j++) cdot_acc(__ldg(Vb + j * n + i), wv, acc[2 * j], acc[2 * j + 1]);
    }
    block_sum<R, 2 * NJ>(acc, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int j = 0; j < 2 * NJ; j++) partial[(long long)blockIdx.x * pitch + 2 * slot0 + j] = (double)acc[j];
    if (FIN) last_block_finish(partial, pitch, 2 * slot0, 2 * NJ, scale, out, ticket);
}

// ---- y = y + sign * sum_j c_j v_j, optionally the partials of ||y_new||^2 ------------
template <typename R, bool NORM>
__global__ void __launch_bounds__(RT, 4) multi_axpy_kernel(const typename Vec<R>::V *__restrict__ Vb, long long n,
                                                           int nv, const double2 *__restrict__ c, R sign,
                                                           typename Vec<R>::V *y, double *partial, int pitch, int slot)
{
    typedef typename Vec<R>::V V;
    __shared__ R sh[RT / 32];
    // the coefficients, converted once per block (a double -> float conversion
    // per use would keep the FP64 pipe busy)
    __shared__ R csr[256], csi[256];
    for (int j = threadIdx.x; j < nv; j += RT) {
        const double2 cj = c[j];
        csr[j] = sign * (R)cj.x;
        csi[j] = sign * (R)cj.y;
    }
    __syncthreads();
    R nrm[1] = {R(0)};
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        V yv = y[i];
        int j = 0;
        for (; j + 4 <= nv; j += 4) {
            V vv[4];
#pragma unroll
            for (int q = 0; q < 4; q++) vv[q] = __ldg(Vb + (j + q) * n + i);
#pragma unroll
            for (int q = 0; q < 4; q++) caxpy(csr[j + q], csi[j + q], vv[q], yv);
        }
        for (; j < nv; j++) caxpy(csr[j], csi[j], __ldg(Vb + j * n + i), yv);
        y[i] = yv;
        if (NORM) nrm[0] = nrm_acc(yv, nrm[0]);
    }
    if (NORM) {
        block_sum<R, 1>(nrm, sh);
        if (threadIdx.x == 0) {
            partial[(long long)blockIdx.x * pitch + 2 * slot] = (double)nrm[0];
            partial[(long long)blockIdx.x * pitch + 2 * slot + 1] = 0.0;
        }
    }
}

// multi_axpy_finish (FP32): see lq_kernels.h
__global__ void __launch_bounds__(RT, 4) multi_axpy_fin_kernel(const float4 *__restrict__ Vb, long long n, int nv,
                                                               const double *c, float sign, float4 *y,
                                                               double *partial, int pitch, int nrm_slot, double *out,
                                                               unsigned *ticket)
{
    __shared__ float sh[RT / 32];
    __shared__ float csr[256], csi[256];
    for (int j = threadIdx.x; j < nv; j += RT) {
        const double2 cj = reinterpret_cast<const double2 *>(c)[j];
        csr[j] = sign * (float)cj.x;
        csi[j] = sign * (float)cj.y;
    }
    __syncthreads();
    float nrm[1] = {0.0f};
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        float4 yv = y[i];
        int j = 0;
        for (; j + 4 <= nv; j += 4) {
            float4 vv[4];
#pragma unroll
            for (int q = 0; q < 4; q++) vv[q] = __ldg(Vb + (j + q) * n + i);
#pragma unroll
            for (int q = 0; q < 4; q++) caxpy(csr[j + q], csi[j + q], vv[q], yv);
        }
        for (; j < nv; j++) caxpy(csr[j], csi[j], __ldg(Vb + j * n + i), yv);
        y[i] = yv;
        nrm[0] = nrm_acc(yv, nrm[0]);
    }
    block_sum<float, 1>(nrm, sh);
    if (threadIdx.x == 0) {
        partial[(long long)blockIdx.x * pitch + 2 * nrm_slot] = (double)nrm[0];
        partial[(long long)blockIdx.x * pitch + 2 * nrm_slot + 1] = 0.0;
    }
    last_block_finish(partial, pitch, 2 * nrm_slot, 2, nullptr, out, ticket);
}

template <typename R>
__global__ void __launch_bounds__(RT) norm2_kernel(const typename Vec<R>::V *__restrict__ w, long long n,
                                                   double *partial, int pitch, int slot)
{
    __shared__ R sh[RT / 32];
    R nrm[1] = {R(0)};
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT)
        nrm[0] = nrm_acc(__ldg(w + i), nrm[0]);
    block_sum<R, 1>(nrm, sh);
    if (threadIdx.x == 0) {
        partial[(long long)blockIdx.x * pitch + 2 * slot] = (double)nrm[0];
        partial[(long long)blockIdx.x * pitch + 2 * slot + 1] = 0.0;
    }
}

// natural complex-double field of n complexes
__global__ void __launch_bounds__(RT) nat_norm2_kernel(const double2 *__restrict__ v, long long n, double *partial,
                                                       int pitch, int slot)
{
    __shared__ double sh[RT / 32];
    double acc[1] = {0.0};
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT)
        acc[0] = nrm_acc(__ldg(v + i), acc[0]);
    block_sum<double, 1>(acc, sh);
    if (threadIdx.x == 0) {
        partial[(long long)blockIdx.x * pitch + 2 * slot] = acc[0];
        partial[(long long)blockIdx.x * pitch + 2 * slot + 1] = 0.0;
    }
}

// one block per value: out[v] = sum_b partial[b][v] in a fixed tree order,
// times scale[v / 2] when a scale (one real per complex value) is given
__global__ void __launch_bounds__(RT) reduce_finish_kernel(const double *__restrict__ partial, int blocks, int pitch,
                                                           const double *__restrict__ scale, double *out)
{
    __shared__ double sh[RT / 32];
    const int v = blockIdx.x;
    double acc[1] = {0.0};
    for (int b = threadIdx.x; b < blocks; b += RT) acc[0] += partial[(long long)b * pitch + v];
    block_sum<double, 1>(acc, sh);
    if (threadIdx.x == 0) out[v] = scale ? acc[0] * scale[v >> 1] : acc[0];
}

// y = a x + b y
template <typename R>
__global__ void __launch_bounds__(RT) axpby_kernel(R ar, R ai, const typename Vec<R>::V *x, R br, R bi,
                                                   typename Vec<R>::V *y, long long n)
{
    const long long i = blockIdx.x * (long long)RT + threadIdx.x;
    if (i >= n) return;
    typename Vec<R>::V o = {}, xv = x[i], yv = y[i];
    caxpy(ar, ai, xv, o);
    caxpy(br, bi, yv, o);
    y[i] = o;
}

// ---- df64 variants (FP64-accurate arithmetic on the FP32 units) ---------------------
__device__ __forceinline__ df64 shfl_down_df(df64 v, int o)
{
    return df64(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o));
}

template <int N>
__device__ __forceinline__ void block_sum_df(df64 v[N], df64 *sh /* [RT/32][N] */)
{
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] = v[i] + shfl_down_df(v[i], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < N; i++) sh[warp * N + i] = v[i];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < N; i++) v[i] = lane < RT / 32 ? sh[lane * N + i] : df64(0.0f, 0.0f);
#pragma unroll
        for (int i = 0; i < N; i++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[i] = v[i] + shfl_down_df(v[i], o);
    }
    __syncthreads();
}

template <int NJ>
__global__ void __launch_bounds__(RT) multi_dot_df_kernel(const df2 *__restrict__ Vb, long long n,
                                                          const df2 *__restrict__ w, double *partial, int pitch,
                                                          int slot0)
{
    __shared__ df64 sh[(RT / 32) * 2 * NJ];
    df64 acc[2 * NJ];
#pragma unroll
    for (int i = 0; i < 2 * NJ; i++) acc[i] = df64(0.0f, 0.0f);
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        const cx<df64> wv = df2_cx(ldg(w + i));
#pragma unroll
        for (int j = 0; j < NJ; j++) {
            const cx<df64> vv = df2_cx(ldg(Vb + j * n + i));
            acc[2 * j] = fma(vv.re, wv.re, fma(vv.im, wv.im, acc[2 * j]));
            acc[2 * j + 1] = fma(vv.re, wv.im, fma(-vv.im, wv.re, acc[2 * j + 1]));
        }
    }
    block_sum_df<2 * NJ>(acc, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int j = 0; j < 2 * NJ; j++) partial[(long long)blockIdx.x * pitch + 2 * slot0 + j] = df_to_double(acc[j]);
}

template <bool NORM>
__global__ void __launch_bounds__(RT) multi_axpy_df_kernel(const df2 *__restrict__ Vb, long long n, int nv,
                                                           const double2 *__restrict__ c, int sign, df2 *y,
                                                           double *partial, int pitch, int slot)
{
    __shared__ df64 cs[2 * 256];
    __shared__ df64 sh[RT / 32];
    for (int j = threadIdx.x; j < nv; j += RT) {
        const double2 cj = c[j];
        cs[2 * j] = df64(sign * cj.x);
        cs[2 * j + 1] = df64(sign * cj.y);
    }
    __syncthreads();
    df64 nrm[1] = {df64(0.0f, 0.0f)};
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        cx<df64> yv = df2_cx(y[i]);
        for (int j = 0; j < nv; j++)
            yv = cfma(cx<df64>{cs[2 * j], cs[2 * j + 1]}, df2_cx(ldg(Vb + j * n + i)), yv);
        y[i] = cx_df2(yv);
        if (NORM) nrm[0] = fma(yv.re, yv.re, fma(yv.im, yv.im, nrm[0]));
    }
    if (NORM) {
        block_sum_df<1>(nrm, sh);
        if (threadIdx.x == 0) {
            partial[(long long)blockIdx.x * pitch + 2 * slot] = df_to_double(nrm[0]);
            partial[(long long)blockIdx.x * pitch + 2 * slot + 1] = 0.0;
        }
    }
}

__global__ void __launch_bounds__(RT) norm2_df_kernel(const df2 *__restrict__ w, long long n, double *partial,
                                                      int pitch, int slot)
{
    __shared__ df64 sh[RT / 32];
    df64 nrm[1] = {df64(0.0f, 0.0f)};
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        const cx<df64> v = df2_cx(ldg(w + i));
        nrm[0] = fma(v.re, v.re, fma(v.im, v.im, nrm[0]));
    }
    block_sum_df<1>(nrm, sh);
    if (threadIdx.x == 0) {
        partial[(long long)blockIdx.x * pitch + 2 * slot] = df_to_double(nrm[0]);
        partial[(long long)blockIdx.x * pitch + 2 * slot + 1] = 0.0;
    }
}

__global__ void __launch_bounds__(RT) axpby_df_kernel(df64 ar, df64 ai, const df2 *x, df64 br, df64 bi, df2 *y,
                                                      long long n)
{
    const long long i = blockIdx.x * (long long)RT + threadIdx.x;
    if (i >= n) return;
    const cx<df64> a = {ar, ai}, b = {br, bi};
    y[i] = cx_df2(cfma(a, df2_cx(x[i]), cmul(b, df2_cx(y[i]))));
}

// ---- launchers -------------------------------------------------------------------------
static inline unsigned nblk(long long n) { return (unsigned)((n + RT - 1) / RT); }
static inline double sp_bytes(int prec) { return prec == P32 ? 96.0 : prec == P16 ? 48.0 : 192.0; }
static inline long long nvec(const Geom &g, int prec) { return (prec == P32 ? 6 : 12) * g.stride; }
static inline int axpy_class(int prec) { return prec == P64 ? K_AXPY_F64 : prec == P32 ? K_AXPY_F32 : K_AXPY_DF; }
static inline int dot_class(int prec) { return prec == P64 ? K_DOT_F64 : prec == P32 ? K_DOT_F32 : K_DOT_DF; }

void zero(const Exec &e, int prec, void *x)
{
    Launch L_(e, K_COPY, (double)e.g.Vh * sp_bytes(prec));
    cudaMemsetAsync(x, 0, spinor_bytes(e.g, prec), e.st);
}

__global__ void __launch_bounds__(RT) copy_kernel(const float4 *__restrict__ x, float4 *__restrict__ y, long long n)
{
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) y[i] = __ldg(x + i);
}

void copy_bytes(const Exec &e, const void *x, void *y, size_t bytes)
{
    const long long n = (long long)(bytes / sizeof(float4));
    if (n == 0) return;
    const long long b = (n + RT - 1) / RT;
    copy_kernel<<<(unsigned)(b < 4 * 608 ? b : 4 * 608), RT, 0, e.st>>>((const float4 *)x, (float4 *)y, n);
}

// a field copy by a kernel rather than cudaMemcpyAsync, which a copy engine
// would serve behind any large transfer the caller has queued on another stream
void copy(const Exec &e, int prec, const void *x, void *y)
{
    Launch L_(e, K_COPY, 2.0 * e.g.Vh * sp_bytes(prec), 0.0, true);
    copy_bytes(e, x, y, spinor_bytes(e.g, prec));
}

// ---- small host <-> device transfers ------------------------------------------------
// The solvers exchange a few scalars with the host at every Arnoldi step.  They
// move through kernels: values to the device as a kernel argument, values to
// the host written by a kernel into pinned host memory through its device
// mapping.  A cudaMemcpyAsync would be served by a copy engine in order, behind
// whatever large transfer the caller has queued on another stream.
struct SmallVals {
    double v[kSmallVals];
};
__global__ void put_values_kernel(SmallVals s, int n, double *d)
{
    if ((int)threadIdx.x < n) d[threadIdx.x] = s.v[threadIdx.x];
}
__global__ void get_values_kernel(const double *__restrict__ d, int n, double *h)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) h[i] = d[i];
}
__global__ void get_ints_kernel(const int *__restrict__ d, int n, int *h)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) h[i] = d[i];
}

void put_values(const Exec &e, const double *h, int n, double *d)
{
    for (int k = 0; k < n; k += kSmallVals) {
        const int m = n - k < kSmallVals ? n - k : kSmallVals;
        SmallVals s;
        for (int i = 0; i < m; i++) s.v[i] = h[k + i];
        Launch L_(e, K_FINISH, 0.0);
        put_values_kernel<<<1, kSmallVals, 0, e.st>>>(s, m, d + k);
    }
}
void get_values(const Exec &e, const double *d, int n, double *h_mapped)
{
    if (n <= 0) return;
    Launch L_(e, K_FINISH, 0.0);
    get_values_kernel<<<1, 128, 0, e.st>>>(d, n, h_mapped);
}
void get_ints(const Exec &e, const int *d, int n, int *h_mapped)
{
    if (n <= 0) return;
    Launch L_(e, K_FINISH, 0.0);
    get_ints_kernel<<<1, 128, 0, e.st>>>(d, n, h_mapped);
}

void axpby(const Exec &e, int prec, double ar, double ai, const void *x, double br, double bi, void *y, int nfields)
{
    if (prec == P16) {
        bf16_axpby(e, ar, ai, x, br, bi, y, nfields);
        return;
    }
    // nfields consecutive fields are one linear array
    Launch L_(e, axpy_class(prec), 3.0 * nfields * e.g.Vh * sp_bytes(prec), (double)nfields * e.g.Vh * 12 * 14);
    const long long n = nvec(e.g, prec) * nfields;
    if (prec == PDF)
        axpby_df_kernel<<<nblk(n), RT, 0, e.st>>>(df64(ar), df64(ai), (const df2 *)x, df64(br), df64(bi), (df2 *)y, n);
    else if (prec == P64)
        axpby_kernel<double><<<nblk(n), RT, 0, e.st>>>(ar, ai, (const double2 *)x, br, bi, (double2 *)y, n);
    else
        axpby_kernel<float><<<nblk(n), RT, 0, e.st>>>((float)ar, (float)ai, (const float4 *)x, (float)br, (float)bi,
                                                     (float4 *)y, n);
}

void multi_axpy(const Exec &e, int prec, const void *V, int nv, const double *c_dev, int sign, void *y,
                const RedScratch *r, int slot)
{
    if (nv <= 0 && !r) return;
    Launch L_(e, axpy_class(prec), (double)e.g.Vh * sp_bytes(prec) * (nv + 2), (double)e.g.Vh * 96 * nv);
    const int blocks = reduction_blocks(e.g);
    const int pitch = r ? 2 * r->maxv : 0;
    double *part = r ? r->partial : nullptr;
    const long long n = nvec(e.g, prec);
    const double2 *c = (const double2 *)c_dev;
    if (prec == PDF) {
        if (r)
            multi_axpy_df_kernel<true><<<blocks, RT, 0, e.st>>>((const df2 *)V, n, nv, c, sign, (df2 *)y, part, pitch, slot);
        else
            multi_axpy_df_kernel<false><<<blocks, RT, 0, e.st>>>((const df2 *)V, n, nv, c, sign, (df2 *)y, part, pitch, slot);
    } else if (prec == P64) {
        if (r)
            multi_axpy_kernel<double, true><<<blocks, RT, 0, e.st>>>((const double2 *)V, n, nv, c, (double)sign,
                                                                     (double2 *)y, part, pitch, slot);
        else
            multi_axpy_kernel<double, false><<<blocks, RT, 0, e.st>>>((const double2 *)V, n, nv, c, (double)sign,
                                                                      (double2 *)y, part, pitch, slot);
    } else {
        if (r)
            multi_axpy_kernel<float, true><<<blocks, RT, 0, e.st>>>((const float4 *)V, n, nv, c, (float)sign,
                                                                    (float4 *)y, part, pitch, slot);
        else
            multi_axpy_kernel<float, false><<<blocks, RT, 0, e.st>>>((const float4 *)V, n, nv, c, (float)sign,
                                                                     (float4 *)y, part, pitch, slot);
    }
}

void multi_axpy_finish(const Exec &e, const void *V, int nv, const RedScratch &r, int sign, void *y, int nrm_slot)
{
    Launch L_(e, K_AXPY_F32, (double)e.g.Vh * sp_bytes(P32) * (nv + 2), (double)e.g.Vh * 96 * nv);
    const int blocks = reduction_blocks(e.g);
    multi_axpy_fin_kernel<<<blocks, RT, 0, e.st>>>((const float4 *)V, nvec(e.g, P32), nv, r.out, (float)sign,
                                                   (float4 *)y, r.partial, 2 * r.maxv, nrm_slot, r.out, r.ticket);
}

template <int NJ>
static void dot_fin_launch(const Exec &e, const RedScratch &r, const void *V, long long n, const void *w, int slot0,
                           const double *scale)
{
    multi_dot_kernel<float, NJ, true><<<r.blocks, RT, 0, e.st>>>((const float4 *)V, n, (const float4 *)w, r.partial,
                                                                 2 * r.maxv, slot0, scale, r.out, r.ticket);
}

void multi_dot_finish(const Exec &e, const void *V, int nv, const void *w, const RedScratch &r, const double *scale)
{
    const long long n = nvec(e.g, P32);
    const size_t vb = spinor_bytes(e.g, P32);
    for (int j0 = 0; j0 < nv; j0 += MAXJ) {
        const int nj = nv - j0 < MAXJ ? nv - j0 : MAXJ;
        Launch L_(e, K_DOT_F32, (double)e.g.Vh * sp_bytes(P32) * (nj + 1), (double)e.g.Vh * 96 * nj);
        const void *Vj = (const char *)V + (size_t)j0 * vb;
        switch (nj) {
        case 1: dot_fin_launch<1>(e, r, Vj, n, w, j0, scale); break;
        case 2: dot_fin_launch<2>(e, r, Vj, n, w, j0, scale); break;
        case 3: dot_fin_launch<3>(e, r, Vj, n, w, j0, scale); break;
        case 4: dot_fin_launch<4>(e, r, Vj, n, w, j0, scale); break;
        case 5: dot_fin_launch<5>(e, r, Vj, n, w, j0, scale); break;
        case 6: dot_fin_launch<6>(e, r, Vj, n, w, j0, scale); break;
        case 7: dot_fin_launch<7>(e, r, Vj, n, w, j0, scale); break;
        default: dot_fin_launch<8>(e, r, Vj, n, w, j0, scale); break;
        }
    }
}

template <typename R, int NJ>
static void dot_launch(const Exec &e, int blocks, const void *V, long long n, const void *w, double *part, int pitch,
                       int slot0)
{
    typedef typename Vec<R>::V VV;
    multi_dot_kernel<R, NJ><<<blocks, RT, 0, e.st>>>((const VV *)V, n, (const VV *)w, part, pitch, slot0);
}
template <int NJ>
static void dot_launch_df(const Exec &e, int blocks, const void *V, long long n, const void *w, double *part,
                          int pitch, int slot0)
{
    multi_dot_df_kernel<NJ><<<blocks, RT, 0, e.st>>>((const df2 *)V, n, (const df2 *)w, part, pitch, slot0);
}

template <int NJ>
static void dot_dispatch(const Exec &e, int prec, int blocks, const void *V, long long n, const void *w,
                         double *part, int pitch, int slot0)
{
    if (prec == PDF) dot_launch_df<NJ>(e, blocks, V, n, w, part, pitch, slot0);
    else if (prec == P64) dot_launch<double, NJ>(e, blocks, V, n, w, part, pitch, slot0);
    else dot_launch<float, NJ>(e, blocks, V, n, w, part, pitch, slot0);
}

void multi_dot(const Exec &e, int prec, const void *V, int nv, const void *w, const RedScratch &r, int slot0)
{
    if (nv <= 0) return;
    const int pitch = 2 * r.maxv;
    const long long n = nvec(e.g, prec);
    const size_t vb = spinor_bytes(e.g, prec);
    for (int j0 = 0; j0 < nv; j0 += MAXJ) {
        const int nj = nv - j0 < MAXJ ? nv - j0 : MAXJ;
        Launch L_(e, dot_class(prec), (double)e.g.Vh * sp_bytes(prec) * (nj + 1), (double)e.g.Vh * 96 * nj);
        const void *Vj = (const char *)V + (size_t)j0 * vb;
        switch (nj) {
        case 1: dot_dispatch<1>(e, prec, r.blocks, Vj, n, w, r.partial, pitch, slot0 + j0); break;
        case 2: dot_dispatch<2>(e, prec, r.blocks, Vj, n, w, r.partial, pitch, slot0 + j0); break;
        case 3: dot_dispatch<3>(e, prec, r.blocks, Vj, n, w, r.partial, pitch, slot0 + j0); break;
        case 4: dot_dispatch<4>(e, prec, r.blocks, Vj, n, w, r.partial, pitch, slot0 + j0); break;
        case 5: dot_dispatch<5>(e, prec, r.blocks, Vj, n, w, r.partial, pitch, slot0 + j0); break;
        case 6: dot_dispatch<6>(e, prec, r.blocks, Vj, n, w, r.partial, pitch, slot0 + j0); break;
        case 7: dot_dispatch<7>(e, prec, r.blocks, Vj, n, w, r.partial, pitch, slot0 + j0); break;
        default: dot_dispatch<8>(e, prec, r.blocks, Vj, n, w, r.partial, pitch, slot0 + j0); break;
        }
    }
}

void norm2(const Exec &e, int prec, const void *w, const RedScratch &r, int slot)
{
    Launch L_(e, K_NORM, (double)e.g.Vh * sp_bytes(prec));
    const int pitch = 2 * r.maxv;
    const long long n = nvec(e.g, prec);
    if (prec == PDF)
        norm2_df_kernel<<<r.blocks, RT, 0, e.st>>>((const df2 *)w, n, r.partial, pitch, slot);
    else if (prec == P64)
        norm2_kernel<double><<<r.blocks, RT, 0, e.st>>>((const double2 *)w, n, r.partial, pitch, slot);
    else
        norm2_kernel<float><<<r.blocks, RT, 0, e.st>>>((const float4 *)w, n, r.partial, pitch, slot);
}

void nat_norm2(const Exec &e, const void *v, long long n_sites, const RedScratch &r, int slot)
{
    Launch L_(e, K_NORM, (double)n_sites * 192.0);
    const int pitch = 2 * r.maxv;
    nat_norm2_kernel<<<r.blocks, RT, 0, e.st>>>((const double2 *)v, n_sites * 12, r.partial, pitch, slot);
}

void reduce_finish(const Exec &e, const RedScratch &r, int first, int count, const double *scale)
{
    if (count <= 0) return;
    Launch L_(e, K_FINISH, (double)r.blocks * 2 * count * 8.0);
    reduce_finish_kernel<<<2 * count, RT, 0, e.st>>>(r.partial + 2 * first, r.blocks, 2 * r.maxv, scale,
                                                     r.out + 2 * first);
}

}  // namespace lq
