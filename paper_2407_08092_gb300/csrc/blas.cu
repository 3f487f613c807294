// BLAS-1 steps and deterministic reductions on internal spinor fields.
//
// Reductions are two-stage and deterministic: a fixed grid (set by the
// lattice size alone) writes one partial per block and slot, then one block
// per value sums the partials in a fixed tree order in FP64.  Dot products
// are (v, w) = sum conj(v) w, the inner product of Algorithm 2.
#include "lq_kernels.h"

namespace lq {

static constexpr int RT = 256;   // threads of reduction / BLAS blocks
static constexpr int MAXJ = 8;   // vectors per pass of the multi-dot

int reduction_blocks(const Geom &g)
{
    long long b = (g.Vh + RT - 1) / RT;
    return (int)(b < 608 ? b : 608);
}

// ---- element access: a site as 12 complexes in precision R ------------------
template <typename R>
struct Vec;
template <>
struct Vec<double> {
    typedef double2 V;
    static constexpr int N = 12;
};
template <>
struct Vec<float> {
    typedef float4 V;
    static constexpr int N = 6;
};

// sum over a block of `n` values held per thread in `v`; result valid in thread 0
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

// ---- multi-dot: partial[blk][2*(slot0+j) + re/im] = block share of (v_j, w) --
template <typename R>
__global__ void __launch_bounds__(RT) multi_dot_kernel(Geom g, const typename Vec<R>::V *__restrict__ Vb,
                                                       long long vstride, int nv,
                                                       const typename Vec<R>::V *__restrict__ w, double *partial,
                                                       int pitch, int slot0)
{
    typedef typename Vec<R>::V V;
    __shared__ R sh[(RT / 32) * 2 * MAXJ];
    for (int j0 = 0; j0 < nv; j0 += MAXJ) {
        R acc[2 * MAXJ];
#pragma unroll
        for (int i = 0; i < 2 * MAXJ; i++) acc[i] = R(0);
        const int nj = nv - j0 < MAXJ ? nv - j0 : MAXJ;
        for (long long s = blockIdx.x * (long long)RT + threadIdx.x; s < g.Vh; s += (long long)gridDim.x * RT) {
#pragma unroll 2
            for (int k = 0; k < Vec<R>::N; k++) {
                const V wv = __ldg(w + k * g.stride + s);
#pragma unroll
                for (int j = 0; j < MAXJ; j++) {
                    if (j < nj) {
                        const V vv = __ldg(Vb + (j0 + j) * vstride + k * g.stride + s);
                        if constexpr (sizeof(R) == 8) {
                            acc[2 * j] += vv.x * wv.x + vv.y * wv.y;
                            acc[2 * j + 1] += vv.x * wv.y - vv.y * wv.x;
                        } else {
                            acc[2 * j] += vv.x * wv.x + vv.y * wv.y + vv.z * wv.z + vv.w * wv.w;
                            acc[2 * j + 1] += vv.x * wv.y - vv.y * wv.x + vv.z * wv.w - vv.w * wv.z;
                        }
                    }
                }
            }
        }
        block_sum<R, 2 * MAXJ>(acc, sh);
        if (threadIdx.x == 0)
            for (int j = 0; j < nj; j++) {
                partial[(long long)blockIdx.x * pitch + 2 * (slot0 + j0 + j)] = (double)acc[2 * j];
                partial[(long long)blockIdx.x * pitch + 2 * (slot0 + j0 + j) + 1] = (double)acc[2 * j + 1];
            }
    }
}

// ---- y = y + sign * sum_j c_j v_j, optionally ||y_new||^2 partials -----------
template <typename R, bool NORM>
__global__ void __launch_bounds__(RT) multi_axpy_kernel(Geom g, const typename Vec<R>::V *__restrict__ Vb,
                                                        long long vstride, int nv, const double2 *__restrict__ c,
                                                        R sign, typename Vec<R>::V *y, double *partial, int pitch,
                                                        int slot)
{
    typedef typename Vec<R>::V V;
    __shared__ R sh[(RT / 32) * 1];
    R nrm[1] = {R(0)};
    for (long long s = blockIdx.x * (long long)RT + threadIdx.x; s < g.Vh; s += (long long)gridDim.x * RT) {
#pragma unroll
        for (int k = 0; k < Vec<R>::N; k++) {
            V yv = y[k * g.stride + s];
            int j = 0;
            for (; j + 4 <= nv; j += 4) {
                V vv[4];
#pragma unroll
                for (int q = 0; q < 4; q++) vv[q] = __ldg(Vb + (j + q) * vstride + k * g.stride + s);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const double2 cj = __ldg(c + j + q);
                    const R cr = sign * (R)cj.x, ci = sign * (R)cj.y;
                    yv.x += cr * vv[q].x - ci * vv[q].y;
                    yv.y += cr * vv[q].y + ci * vv[q].x;
                    if constexpr (sizeof(R) == 4) {
                        yv.z += cr * vv[q].z - ci * vv[q].w;
                        yv.w += cr * vv[q].w + ci * vv[q].z;
                    }
                }
            }
            for (; j < nv; j++) {
                const V vv = __ldg(Vb + j * vstride + k * g.stride + s);
                const double2 cj = __ldg(c + j);
                const R cr = sign * (R)cj.x, ci = sign * (R)cj.y;
                yv.x += cr * vv.x - ci * vv.y;
                yv.y += cr * vv.y + ci * vv.x;
                if constexpr (sizeof(R) == 4) {
                    yv.z += cr * vv.z - ci * vv.w;
                    yv.w += cr * vv.w + ci * vv.z;
                }
            }
            y[k * g.stride + s] = yv;
            if (NORM) {
                nrm[0] += yv.x * yv.x + yv.y * yv.y;
                if constexpr (sizeof(R) == 4) nrm[0] += yv.z * yv.z + yv.w * yv.w;
            }
        }
    }
    if (NORM) {
        block_sum<R, 1>(nrm, sh);
        if (threadIdx.x == 0) {
            partial[(long long)blockIdx.x * pitch + 2 * slot] = (double)nrm[0];
            partial[(long long)blockIdx.x * pitch + 2 * slot + 1] = 0.0;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(RT) norm2_kernel(Geom g, const typename Vec<R>::V *__restrict__ w, double *partial,
                                                   int pitch, int slot)
{
    typedef typename Vec<R>::V V;
    __shared__ R sh[(RT / 32) * 1];
    R nrm[1] = {R(0)};
    for (long long s = blockIdx.x * (long long)RT + threadIdx.x; s < g.Vh; s += (long long)gridDim.x * RT) {
#pragma unroll
        for (int k = 0; k < Vec<R>::N; k++) {
            const V v = __ldg(w + k * g.stride + s);
            nrm[0] += v.x * v.x + v.y * v.y;
            if constexpr (sizeof(R) == 4) nrm[0] += v.z * v.z + v.w * v.w;
        }
    }
    block_sum<R, 1>(nrm, sh);
    if (threadIdx.x == 0) {
        partial[(long long)blockIdx.x * pitch + 2 * slot] = (double)nrm[0];
        partial[(long long)blockIdx.x * pitch + 2 * slot + 1] = 0.0;
    }
}

// natural complex-double field of n sites x 12 complexes
__global__ void __launch_bounds__(RT) nat_norm2_kernel(const double2 *__restrict__ v, long long n, double *partial,
                                                       int pitch, int slot)
{
    __shared__ double sh[RT / 32];
    double acc[1] = {0.0};
    for (long long i = blockIdx.x * (long long)RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        const double2 t = __ldg(v + i);
        acc[0] += t.x * t.x + t.y * t.y;
    }
    block_sum<double, 1>(acc, sh);
    if (threadIdx.x == 0) {
        partial[(long long)blockIdx.x * pitch + 2 * slot] = acc[0];
        partial[(long long)blockIdx.x * pitch + 2 * slot + 1] = 0.0;
    }
}

// one block per value: out[v] = sum_b partial[b][v] in a fixed tree order
__global__ void __launch_bounds__(RT) reduce_finish_kernel(const double *__restrict__ partial, int blocks, int pitch,
                                                           double *out)
{
    __shared__ double sh[RT / 32];
    const int v = blockIdx.x;
    double acc[1] = {0.0};
    for (int b = threadIdx.x; b < blocks; b += RT) acc[0] += partial[(long long)b * pitch + v];
    block_sum<double, 1>(acc, sh);
    if (threadIdx.x == 0) out[v] = acc[0];
}

template <typename R>
__global__ void __launch_bounds__(RT) scale_kernel(Geom g, const typename Vec<R>::V *x, const double *nrm2,
                                                   typename Vec<R>::V *y)
{
    typedef typename Vec<R>::V V;
    const long long s = blockIdx.x * (long long)RT + threadIdx.x;
    if (s >= g.Vh) return;
    const R f = (R)(1.0 / sqrt(*nrm2));
#pragma unroll
    for (int k = 0; k < Vec<R>::N; k++) {
        V v = x[k * g.stride + s];
        v.x *= f;
        v.y *= f;
        if constexpr (sizeof(R) == 4) {
            v.z *= f;
            v.w *= f;
        }
        y[k * g.stride + s] = v;
    }
}

template <typename R>
__global__ void __launch_bounds__(RT) axpby_kernel(Geom g, R ar, R ai, const typename Vec<R>::V *x, R br, R bi,
                                                   typename Vec<R>::V *y)
{
    typedef typename Vec<R>::V V;
    const long long s = blockIdx.x * (long long)RT + threadIdx.x;
    if (s >= g.Vh) return;
#pragma unroll
    for (int k = 0; k < Vec<R>::N; k++) {
        const V a = x[k * g.stride + s];
        V b = y[k * g.stride + s];
        V o;
        o.x = ar * a.x - ai * a.y + br * b.x - bi * b.y;
        o.y = ar * a.y + ai * a.x + br * b.y + bi * b.x;
        if constexpr (sizeof(R) == 4) {
            o.z = ar * a.z - ai * a.w + br * b.z - bi * b.w;
            o.w = ar * a.w + ai * a.z + br * b.w + bi * b.z;
        }
        y[k * g.stride + s] = o;
    }
}

// ---- launchers -----------------------------------------------------------------
static inline unsigned nblk(long long n) { return (unsigned)((n + RT - 1) / RT); }
static inline double sp_bytes(int prec) { return prec == P64 ? 192.0 : 96.0; }

void zero(const Exec &e, int prec, void *x)
{
    Launch L_(e, K_COPY, (double)e.g.Vh * sp_bytes(prec));
    cudaMemsetAsync(x, 0, spinor_bytes(e.g, prec), e.st);
}

void copy(const Exec &e, int prec, const void *x, void *y)
{
    Launch L_(e, K_COPY, 2.0 * e.g.Vh * sp_bytes(prec));
    cudaMemcpyAsync(y, x, spinor_bytes(e.g, prec), cudaMemcpyDeviceToDevice, e.st);
}

void axpby(const Exec &e, int prec, double ar, double ai, const void *x, double br, double bi, void *y)
{
    Launch L_(e, (prec == P64 ? K_AXPY_F64 : K_AXPY_F32), 3.0 * e.g.Vh * sp_bytes(prec));
    if (prec == P64)
        axpby_kernel<double><<<nblk(e.g.Vh), RT, 0, e.st>>>(e.g, ar, ai, (const double2 *)x, br, bi, (double2 *)y);
    else
        axpby_kernel<float><<<nblk(e.g.Vh), RT, 0, e.st>>>(e.g, (float)ar, (float)ai, (const float4 *)x, (float)br,
                                                          (float)bi, (float4 *)y);
}

void multi_axpy(const Exec &e, int prec, const void *V, int nv, const double *c_dev, int sign, void *y,
                const RedScratch *r, int slot)
{
    if (nv <= 0 && !r) return;
    Launch L_(e, (prec == P64 ? K_AXPY_F64 : K_AXPY_F32), (double)e.g.Vh * sp_bytes(prec) * (nv + 2));
    const int blocks = reduction_blocks(e.g);
    const int pitch = r ? 2 * r->maxv : 0;
    double *part = r ? r->partial : nullptr;
    if (prec == P64) {
        const long long vstride = 12 * e.g.stride;
        if (r)
            multi_axpy_kernel<double, true><<<blocks, RT, 0, e.st>>>(e.g, (const double2 *)V, vstride, nv,
                                                                     (const double2 *)c_dev, (double)sign,
                                                                     (double2 *)y, part, pitch, slot);
        else
            multi_axpy_kernel<double, false><<<blocks, RT, 0, e.st>>>(e.g, (const double2 *)V, vstride, nv,
                                                                      (const double2 *)c_dev, (double)sign,
                                                                      (double2 *)y, part, pitch, slot);
    } else {
        const long long vstride = 6 * e.g.stride;
        if (r)
            multi_axpy_kernel<float, true><<<blocks, RT, 0, e.st>>>(e.g, (const float4 *)V, vstride, nv,
                                                                    (const double2 *)c_dev, (float)sign,
                                                                    (float4 *)y, part, pitch, slot);
        else
            multi_axpy_kernel<float, false><<<blocks, RT, 0, e.st>>>(e.g, (const float4 *)V, vstride, nv,
                                                                     (const double2 *)c_dev, (float)sign,
                                                                     (float4 *)y, part, pitch, slot);
    }
}

void multi_dot(const Exec &e, int prec, const void *V, int nv, const void *w, const RedScratch &r, int slot0)
{
    if (nv <= 0) return;
    Launch L_(e, (prec == P64 ? K_DOT_F64 : K_DOT_F32), (double)e.g.Vh * sp_bytes(prec) * (nv + (nv + MAXJ - 1) / MAXJ));
    const int pitch = 2 * r.maxv;
    if (prec == P64)
        multi_dot_kernel<double><<<r.blocks, RT, 0, e.st>>>(e.g, (const double2 *)V, 12 * e.g.stride, nv,
                                                            (const double2 *)w, r.partial, pitch, slot0);
    else
        multi_dot_kernel<float><<<r.blocks, RT, 0, e.st>>>(e.g, (const float4 *)V, 6 * e.g.stride, nv,
                                                           (const float4 *)w, r.partial, pitch, slot0);
}

void norm2(const Exec &e, int prec, const void *w, const RedScratch &r, int slot)
{
    Launch L_(e, K_NORM, (double)e.g.Vh * sp_bytes(prec));
    const int pitch = 2 * r.maxv;
    if (prec == P64)
        norm2_kernel<double><<<r.blocks, RT, 0, e.st>>>(e.g, (const double2 *)w, r.partial, pitch, slot);
    else
        norm2_kernel<float><<<r.blocks, RT, 0, e.st>>>(e.g, (const float4 *)w, r.partial, pitch, slot);
}

void nat_norm2(const Exec &e, const void *v, long long n_sites, const RedScratch &r, int slot)
{
    Launch L_(e, K_NORM, (double)n_sites * 192.0);
    const int pitch = 2 * r.maxv;
    nat_norm2_kernel<<<r.blocks, RT, 0, e.st>>>((const double2 *)v, n_sites * 12, r.partial, pitch, slot);
}

void reduce_finish(const Exec &e, const RedScratch &r, int first, int count)
{
    if (count <= 0) return;
    Launch L_(e, K_FINISH, (double)r.blocks * 2 * count * 8.0);
    reduce_finish_kernel<<<2 * count, RT, 0, e.st>>>(r.partial + 2 * first, r.blocks, 2 * r.maxv, r.out + 2 * first);
}

void scale_by_inv_norm(const Exec &e, int prec, const void *x, const RedScratch &r, int slot, void *y)
{
    Launch L_(e, (prec == P64 ? K_AXPY_F64 : K_AXPY_F32), 2.0 * e.g.Vh * sp_bytes(prec));
    if (prec == P64)
        scale_kernel<double><<<nblk(e.g.Vh), RT, 0, e.st>>>(e.g, (const double2 *)x, r.out + 2 * slot, (double2 *)y);
    else
        scale_kernel<float><<<nblk(e.g.Vh), RT, 0, e.st>>>(e.g, (const float4 *)x, r.out + 2 * slot, (float4 *)y);
}

}  // namespace lq
