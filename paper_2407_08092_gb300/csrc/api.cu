// C-ABI entry points, the library context and the host-side solver drivers.
//
// Solvers (host control flow, device arithmetic):
//  * GMRES(m) on D_S (Algorithm 2).  The Arnoldi step orthogonalises with
//    classical Gram-Schmidt applied twice (CGS2: one fused multi-dot and one
//    multi-axpy per pass, both over the whole basis) instead of the listing's
//    modified Gram-Schmidt, so that each pass is one sweep over memory; the
//    Hessenberg least-squares problem is solved by Givens rotations on the host.
//  * Flexible GMRES(m) in FP64 or df64 (the outer solver of every level,
//    Sec. 2.3), right-preconditioned by a Richardson or GMRES smoother in
//    FP64, df64 or FP32.
// Precisions: native FP64, FP32, and df64 (FP64-accurate double-float
// arithmetic on the FP32 units, several times faster than native FP64 on
// GB300).
//  * Richardson(n) on D_S (Algorithm 4) with the update fused into the second
//    hopping kernel; the first sweep from x = 0 is x = omega b.
//  * The odd-even smoother M_n (Sec. 2.4.5): prepare, smoother on D_S,
//    reconstruct (Eq. 2).
//  * Power iteration on D_S^+ D_S for ||D_S||_2 (Sec. 2.4.4).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/lqdd.h"
#include <nvtx3/nvToolsExt.h>
#include "lq_kernels.h"

using namespace lq;
typedef std::complex<double> cd;

static constexpr int MAX_RESTART = 256;
static constexpr int RED_SLOTS = 2 * MAX_RESTART + 8;

struct lq_ctx {
    Geom g;
    lq_lattice lat;
    cudaStream_t st;
    Counters ctr;
    int device;
    bool have_gauge = false;
    bool clover64 = false;            // C64 / Ci64 rounded from the current df64 blocks
    bool links16 = false;             // U16 rounded from the current FP32 links
    bool links64 = false;             // U64 rounded from the current df64 links
    void *U64[2] = {nullptr, nullptr};
    void *U32[2] = {nullptr, nullptr};
    void *C64[2] = {nullptr, nullptr};
    void *C32[2] = {nullptr, nullptr};
    void *Ci64 = nullptr;
    void *Ci32 = nullptr;
    void *Udf[2] = {nullptr, nullptr};
    void *U16[2] = {nullptr, nullptr};   // BF16 12-real links
    void *Cdf[2] = {nullptr, nullptr};
    void *Cidf = nullptr;
    int *dflag = nullptr;
    RedScratch red{};
    double *h_pin = nullptr;   // pinned host mirror of red.out / coefficients
    double *h_pin_dev = nullptr;   // h_pin's device mapping (written by get_values)
    int *h_int = nullptr, *h_int_dev = nullptr;   // pinned host ints and their device mapping
    double *d_coef = nullptr;  // device coefficients [2 * RED_SLOTS]
    double *d_s2 = nullptr;    // device: squared scales s_j^2 of the FP32 GMRES basis [RED_SLOTS]
    std::map<std::string, std::pair<void *, size_t>> ws;
    std::vector<void *> owned;
    std::string err;
    Prof prof;
    lq_group *self_group = nullptr;   // the one-member group behind lq_solve_batch
    int sap_b[4] = {0, 0, 0, 0};      // block extents of the SAP origin tables below
    int sapbm_b[4] = {0, 0, 0, 0};    // block extents of the block-major SAP copies (0: none for this gauge)
    int4 *sap_origin[2] = {nullptr, nullptr};
    int sap_count[2] = {0, 0};
    Exec ex() { return Exec{g, st, &ctr, &prof}; }
};

namespace lq {
cudaEvent_t Prof::get()
{
    if (next == pool.size()) {
        cudaEvent_t ev = nullptr;
        if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
        pool.push_back(ev);
    }
    return pool[next++];
}
}  // namespace lq

// An NVTX range around one C-ABI call, so that profiler timelines show which
// call each kernel belongs to (header-only NVTX: a no-op without a profiler).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

namespace {

struct Fail {
    lq_status s;
};

void fail(lq_ctx *c, lq_status s, const std::string &msg)
{
    if (c) c->err = msg;
    throw Fail{s};
}

void ck(lq_ctx *c, cudaError_t e, const char *what)
{
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(c, e == cudaErrorMemoryAllocation ? LQ_ERR_OOM : LQ_ERR_CUDA,
             std::string(what) + ": " + cudaGetErrorString(e));
    }
}

void ck_launch(lq_ctx *c, const char *what) { ck(c, cudaGetLastError(), what); }

void *dev_alloc(lq_ctx *c, size_t bytes)
{
    void *p = nullptr;
    ck(c, cudaMalloc(&p, bytes), "cudaMalloc");
    // zero-fill: the BLAS kernels sweep whole fields and rely on the padding
    // sites (cb >= V/2), which no kernel writes, staying zero
    ck(c, cudaMemsetAsync(p, 0, bytes, c->st), "cudaMemsetAsync");
    c->owned.push_back(p);
    return p;
}

// named, grow-only workspace buffer
void *ws(lq_ctx *c, const std::string &name, size_t bytes)
{
    auto it = c->ws.find(name);
    if (it != c->ws.end() && it->second.second >= bytes) return it->second.first;
    if (it != c->ws.end()) {
        cudaFree(it->second.first);
        for (auto &p : c->owned)
            if (p == it->second.first) p = nullptr;
        c->ws.erase(it);
    }
    void *p = dev_alloc(c, bytes);
    c->ws[name] = {p, bytes};
    return p;
}

const char *suffix(int prec) { return prec == P64 ? "/64" : prec == P32 ? "/32" : prec == P16 ? "/16" : "/df"; }

void *field(lq_ctx *c, int prec, const char *name)
{
    return ws(c, std::string(name) + suffix(prec), spinor_bytes(c->g, prec));
}

void *basis(lq_ctx *c, int prec, const char *name, int n)
{
    return ws(c, std::string(name) + suffix(prec), (size_t)n * spinor_bytes(c->g, prec));
}

inline void *vec_at(lq_ctx *c, int prec, void *base, int j)
{
    return (char *)base + (size_t)j * spinor_bytes(c->g, prec);
}

void sync(lq_ctx *c) { ck(c, cudaStreamSynchronize(c->st), "cudaStreamSynchronize"); }

// copy r.out[first .. first+count) (complex slots) to the pinned mirror and wait
const double *fetch(lq_ctx *c, int first, int count)
{
    get_values(c->ex(), c->red.out + 2 * first, 2 * count, c->h_pin_dev + 2 * first);
    ck_launch(c, "fetch");
    sync(c);
    return c->h_pin + 2 * first;
}

double norm2_of(lq_ctx *c, int prec, const void *v)
{
    Exec e = c->ex();
    norm2(e, prec, v, c->red, 0);
    reduce_finish(e, c->red, 0, 1);
    ck_launch(c, "norm2");
    return fetch(c, 0, 1)[0];
}

void need_gauge(lq_ctx *c)
{
    if (!c->have_gauge) fail(c, LQ_ERR_STATE, "no gauge field: call lq_set_gauge first");
}

// The FP64 clover blocks and links and the BF16 links are rounded copies that
// only the FP64 operator and the BF16 hops read: they are made on first use
// after each lq_set_gauge, on the context's stream.  The FP64 copies are
// hi + lo of the df64 ones (about 48 significand bits of the caller's field).
void need_clover64(lq_ctx *c)
{
    if (c->clover64) return;
    Exec e = c->ex();
    for (int p = 0; p < 2; p++) clover_to_f64(e, c->Cdf[p], c->C64[p]);
    clover_to_f64(e, c->Cidf, c->Ci64);
    c->clover64 = true;
}
void need_links64(lq_ctx *c)
{
    if (c->links64) return;
    Exec e = c->ex();
    for (int p = 0; p < 2; p++) df64_to_f64(e, c->Udf[p], c->U64[p], 36LL * c->g.stride);
    c->links64 = true;
}
void need_links16(lq_ctx *c)
{
    if (c->links16) return;
    Exec e = c->ex();
    for (int p = 0; p < 2; p++) links_to_bf16(e, c->U32[p], c->U16[p]);
    c->links16 = true;
}

// clover blocks of a precision (BF16 fields use the FP32 blocks)
const void *Cp(lq_ctx *c, int prec, int parity)
{
    if (prec == P64) need_clover64(c);
    return prec == P64 ? c->C64[parity] : (prec == P32 || prec == P16) ? c->C32[parity] : c->Cdf[parity];
}
const void *Cip(lq_ctx *c, int prec)
{
    if (prec == P64) need_clover64(c);
    return prec == P64 ? c->Ci64 : (prec == P32 || prec == P16) ? c->Ci32 : c->Cidf;
}
bool valid_prec(int p) { return p == LQ_F64 || p == LQ_F32 || p == LQ_DF64; }

HopCall hopcall(lq_ctx *c, int mode, int prec, int pout)
{
    HopCall h{};
    h.mode = mode;
    h.prec = prec;
    h.pout = pout;
    if (prec == P16) need_links16(c);
    if (prec == P64) need_links64(c);
    for (int p = 0; p < 2; p++)
        h.U[p] = prec == P64 ? c->U64[p] : prec == P32 ? c->U32[p] : prec == P16 ? c->U16[p] : c->Udf[p];
    return h;
}

// ---- operators on internal fields ---------------------------------------------

// out_e = D_S in_e (Eq. 3) via K1 (odd sites) and K2 (even sites); t: odd temporary
void op_schur(lq_ctx *c, int prec, const void *in, void *out, void *t)
{
    Exec e = c->ex();
    HopCall k1 = hopcall(c, HOP_K1, prec, 1);
    k1.in = in;
    k1.out = t;
    k1.clov = Cip(c, prec);
    hop(e, k1);
    HopCall k2 = hopcall(c, HOP_K2, prec, 0);
    k2.in = t;
    k2.in2 = in;
    k2.out = out;
    k2.clov = Cp(c, prec, 0);
    hop(e, k2);
}

// x_e += omega (b_e - D_S x_e), fused into K2
void op_rich_sweep(lq_ctx *c, int prec, void *x, const void *b, double omega, void *t)
{
    Exec e = c->ex();
    HopCall k1 = hopcall(c, HOP_K1, prec, 1);
    k1.in = x;
    k1.out = t;
    k1.clov = Cip(c, prec);
    hop(e, k1);
    HopCall k2 = hopcall(c, HOP_RICH, prec, 0);
    k2.in = t;
    k2.in2 = x;
    k2.b = b;
    k2.out = x;
    k2.clov = Cp(c, prec, 0);
    k2.omega = omega;
    hop(e, k2);
}

void op_full(lq_ctx *c, int prec, const void *ie, const void *io, void *oe, void *oo)
{
    Exec e = c->ex();
    HopCall a = hopcall(c, HOP_FULL, prec, 0);
    a.in = io;
    a.in2 = ie;
    a.out = oe;
    a.clov = Cp(c, prec, 0);
    hop(e, a);
    HopCall b = hopcall(c, HOP_FULL, prec, 1);
    b.in = ie;
    b.in2 = io;
    b.out = oo;
    b.clov = Cp(c, prec, 1);
    hop(e, b);
}

// bhat_e = b_e - D_eo D_oo^{-1} b_o
void op_prepare(lq_ctx *c, int prec, const void *be, const void *bo, void *bhat, void *t)
{
    Exec e = c->ex();
    clover_mul(e, prec, Cip(c, prec), bo, t);
    HopCall p = hopcall(c, HOP_PREP, prec, 0);
    p.in = t;
    p.in2 = be;
    p.out = bhat;
    hop(e, p);
}

// x_o = D_oo^{-1} (b_o - D_oe x_e)
void op_reconstruct(lq_ctx *c, int prec, const void *bo, const void *xe, void *xo)
{
    Exec e = c->ex();
    HopCall r = hopcall(c, HOP_RECON, prec, 1);
    r.in = xe;
    r.in2 = bo;
    r.out = xo;
    r.clov = Cip(c, prec);
    hop(e, r);
}

// The reconstruction of Eq. 2 together with the full system's residual r = b - D x
// (prec FP64 or df64): x_o = D_oo^{-1} u with u = b_o - D_oe x_e, and in the same
// launch r_o = u - D_oo x_o; then r_e = b_e - D_ee x_e - D_eo x_o in one launch.
void op_reconstruct_residual(lq_ctx *c, int prec, const void *be, const void *bo, const void *xe, void *xo,
                             void *re, void *ro)
{
    Exec e = c->ex();
    HopCall r = hopcall(c, HOP_RECON_RES, prec, 1);
    r.in = xe;
    r.in2 = bo;
    r.out = xo;
    r.clov = Cip(c, prec);
    r.clov2 = Cp(c, prec, 1);
    r.out2 = ro;
    hop(e, r);
    HopCall q = hopcall(c, HOP_RES, prec, 0);
    q.in = xo;
    q.in2 = xe;
    q.b = be;
    q.out = re;
    q.clov = Cp(c, prec, 0);
    hop(e, q);
}

// ---- Krylov solvers ---------------------------------------------------------------

struct KResult {
    int cycles = 0;
    int iters = 0;
    double relres = 0.0;   // last residual estimate or recomputed value, relative to ||b||
    bool converged = false;
};

// Givens-rotation least squares of the Arnoldi relation, on the host
struct Hess {
    int m;
    std::vector<cd> H;   // column-major (m+1) x m
    std::vector<double> cs;
    std::vector<cd> sn;
    std::vector<cd> gv;
    explicit Hess(int m_) : m(m_), H((size_t)(m_ + 1) * m_), cs(m_), sn(m_), gv(m_ + 1) {}
    cd &h(int i, int j) { return H[(size_t)j * (m + 1) + i]; }
    void reset(double beta)
    {
        std::fill(gv.begin(), gv.end(), cd(0));
        gv[0] = beta;
    }
    // rotate column k (entries 0..k+1 already stored); returns |g_{k+1}|
    double rotate(int k)
    {
        for (int i = 0; i < k; i++) {
            cd a = h(i, k), b = h(i + 1, k);
            h(i, k) = cs[i] * a + sn[i] * b;
            h(i + 1, k) = -std::conj(sn[i]) * a + cs[i] * b;
        }
        cd a = h(k, k), b = h(k + 1, k);
        double t = std::sqrt(std::norm(a) + std::norm(b));
        if (std::abs(a) == 0.0) {
            cs[k] = 0.0;
            sn[k] = 1.0;
        } else {
            cs[k] = std::abs(a) / t;
            sn[k] = (a / std::abs(a)) * std::conj(b) / t;
        }
        h(k, k) = cs[k] * a + sn[k] * b;
        h(k + 1, k) = 0.0;
        cd gk = gv[k];
        gv[k] = cs[k] * gk;
        gv[k + 1] = -std::conj(sn[k]) * gk;
        return std::abs(gv[k + 1]);
    }
    // back-substitution R y = g for the first n columns
    std::vector<cd> solve(int n)
    {
        std::vector<cd> y(n);
        for (int i = n - 1; i >= 0; i--) {
            cd acc = gv[i];
            for (int j = i + 1; j < n; j++) acc -= h(i, j) * y[j];
            y[i] = acc / h(i, i);
        }
        return y;
    }
};

void upload_coef(lq_ctx *c, const std::vector<cd> &y)
{
    std::vector<double> v(2 * y.size());
    for (size_t j = 0; j < y.size(); j++) {
        v[2 * j] = y[j].real();
        v[2 * j + 1] = y[j].imag();
    }
    // kernel arguments: nothing to stage, so nothing to wait for
    put_values(c->ex(), v.data(), (int)v.size(), c->d_coef);
    ck_launch(c, "upload_coef");
}

// Arnoldi step: w <- w orthogonalised against V[0..k] by CGS2; returns the
// Hessenberg column h[0..k] and h_{k+1,k} = ||w|| (not yet normalised)
// The FP64-class solvers orthogonalise twice (CGS2); the FP32 solvers, which
// only ever serve as preconditioners or smoothers under an FP64-class outer
// iteration, orthogonalise once (classical Gram-Schmidt: one multi-dot and one
// multi-axpy with the new norm fused), half the basis sweeps of CGS2.
double arnoldi_cgs2(lq_ctx *c, int prec, void *V, int k, void *w, Hess &H)
{
    Exec e = c->ex();
    const int n = k + 1;
    if (prec == P32) {
        multi_dot(e, prec, V, n, w, c->red, 0);
        reduce_finish(e, c->red, 0, n);
        multi_axpy(e, prec, V, n, c->red.out, -1, w, &c->red, n);
        reduce_finish(e, c->red, n, 1);
        ck_launch(c, "arnoldi");
        const double *hv = fetch(c, 0, n + 1);
        for (int j = 0; j < n; j++) H.h(j, k) = cd(hv[2 * j], hv[2 * j + 1]);
        const double nrm2 = hv[2 * n];
        if (!std::isfinite(nrm2)) fail(c, LQ_ERR_NAN, "NaN/Inf in the Arnoldi process");
        return std::sqrt(nrm2);
    }
    multi_dot(e, prec, V, n, w, c->red, 0);
    reduce_finish(e, c->red, 0, n);
    multi_axpy(e, prec, V, n, c->red.out, -1, w, nullptr, 0);
    multi_dot(e, prec, V, n, w, c->red, n);
    reduce_finish(e, c->red, n, n);
    multi_axpy(e, prec, V, n, c->red.out + 2 * n, -1, w, &c->red, 2 * n);
    reduce_finish(e, c->red, 2 * n, 1);
    ck_launch(c, "arnoldi");
    const double *hv = fetch(c, 0, 2 * n + 1);
    for (int j = 0; j < n; j++) H.h(j, k) = cd(hv[2 * j] + hv[2 * (n + j)], hv[2 * j + 1] + hv[2 * (n + j) + 1]);
    const double nrm2 = hv[4 * n];
    if (!std::isfinite(nrm2)) fail(c, LQ_ERR_NAN, "NaN/Inf in the Arnoldi process");
    return std::sqrt(nrm2);
}

// The FP32 GMRES keeps its basis unnormalised: v_j = s_j V_j with the scales
// s_j on the host, which saves the pass that would scale each new vector by
// 1 / ||w||.  set_scale passes s_j^2 to the device for the CGS coefficients.
void set_scale(lq_ctx *c, int j, double s)
{
    const double s2 = s * s;
    put_values(c->ex(), &s2, 1, c->d_s2 + j);
    ck_launch(c, "set_scale");
}

// Arnoldi step on the unnormalised FP32 basis: w = D_S V_k = D_S v_k / s_k.
// In the v's, h_jk = (v_j, D_S v_k) = s_j s_k (V_j, w) and CGS removes
// sum_j h_jk v_j, i.e. w -= sum_j s_j^2 (V_j, w) V_j (the reduction applies
// s_j^2); the new vector V_{k+1} = w has s_{k+1} = 1 / ||w||, and the true
// h_{k+1,k} = s_k ||w||, which is returned.
double arnoldi_scaled(lq_ctx *c, void *V, int k, void *w, Hess &H, double *s)
{
    Exec e = c->ex();
    const int n = k + 1;
    multi_dot_finish(e, V, n, w, c->red, c->d_s2);   // s_j^2 (V_j, w) into red.out
    multi_axpy_finish(e, V, n, c->red, -1, w, n);    // w -= sum_j ..., ||w||^2 into red.out[n]
    ck_launch(c, "arnoldi");
    const double *hv = fetch(c, 0, n + 1);
    for (int j = 0; j < n; j++) H.h(j, k) = cd(hv[2 * j], hv[2 * j + 1]) * (s[k] / s[j]);
    const double nrm2 = hv[2 * n];
    if (!std::isfinite(nrm2)) fail(c, LQ_ERR_NAN, "NaN/Inf in the Arnoldi process");
    const double nrm = std::sqrt(nrm2);
    s[k + 1] = nrm > 0 ? 1.0 / nrm : 0.0;
    return s[k] * nrm;
}

// Restarted GMRES(m) on D_S in precision `prec`: b, x internal even fields.
// x_zero: x is known to be zero on entry (skips the first residual product).
// tol > 0 stops at ||b - D_S x|| <= tol ||b||; tol == 0 runs max_cycles full cycles.
// confirm: a cycle whose least-squares estimate reaches the tolerance is
// confirmed by the recomputed residual before returning (the next cycle's
// first step); without it the call returns on the estimate, for callers that
// check the result themselves (the odd-even solve recomputes the full
// system's residual) or only precondition with it.
KResult gmres(lq_ctx *c, int prec, const void *b, void *x, int m, int max_cycles, double tol, bool x_zero,
              const char *wsname, double bnorm_hint = -1.0, bool confirm = true)
{
    Exec e = c->ex();
    KResult R;
    void *V = basis(c, prec, wsname, m + 1);
    void *t = field(c, prec, (std::string(wsname) + ":t").c_str());
    const double bnorm = bnorm_hint >= 0 ? bnorm_hint : std::sqrt(norm2_of(c, prec, b));
    if (!std::isfinite(bnorm)) fail(c, LQ_ERR_NAN, "NaN/Inf in the right-hand side");
    if (bnorm == 0.0) {
        zero(e, prec, x);
        R.converged = true;
        return R;
    }
    Hess H(m);
    for (int cyc = 0; cyc < max_cycles; cyc++) {
        void *v0 = vec_at(c, prec, V, 0);
        double beta;
        if (x_zero) {
            copy(e, prec, b, v0);
            beta = bnorm;
        } else {
            op_schur(c, prec, x, v0, t);
            axpby(e, prec, 1.0, 0.0, b, -1.0, 0.0, v0);   // v0 = b - D_S x
            beta = std::sqrt(norm2_of(c, prec, v0));
            if (!std::isfinite(beta)) fail(c, LQ_ERR_NAN, "NaN/Inf in the residual");
        }
        R.relres = beta / bnorm;
        if (tol > 0 && beta <= tol * bnorm) {
            R.converged = true;
            return R;
        }
        R.cycles++;
        // FP32: v0 = s_0 V_0 kept unnormalised; otherwise normalised in place
        const bool scaled = prec == P32;
        double s[MAX_RESTART + 1];
        if (scaled) {
            s[0] = 1.0 / beta;
            set_scale(c, 0, s[0]);
        } else {
            axpby(e, prec, 0.0, 0.0, v0, 1.0 / beta, 0.0, v0);
        }
        H.reset(beta);
        int nk = 0;
        for (int k = 0; k < m; k++) {
            void *w = vec_at(c, prec, V, k + 1);
            op_schur(c, prec, vec_at(c, prec, V, k), w, t);
            const double hk1 = scaled ? arnoldi_scaled(c, V, k, w, H, s) : arnoldi_cgs2(c, prec, V, k, w, H);
            double colnorm2 = hk1 * hk1;
            for (int j = 0; j <= k; j++) colnorm2 += std::norm(H.h(j, k));
            H.h(k + 1, k) = hk1;
            const double est = H.rotate(k);
            nk = k + 1;
            R.iters++;
            R.relres = est / bnorm;
            const bool breakdown = hk1 <= 1e-14 * std::sqrt(colnorm2);
            if (breakdown || (tol > 0 && est <= tol * bnorm) || k == m - 1) break;
            if (scaled) set_scale(c, k + 1, s[k + 1]);
            else axpby(e, prec, 0.0, 0.0, w, 1.0 / hk1, 0.0, w);
        }
        std::vector<cd> y = H.solve(nk);
        if (scaled)   // x += sum_j y_j v_j = sum_j (y_j s_j) V_j
            for (int j = 0; j < nk; j++) y[j] *= s[j];
        upload_coef(c, y);
        multi_axpy(e, prec, V, nk, c->d_coef, +1, x, nullptr, 0);
        ck_launch(c, "gmres update");
        x_zero = false;
        if (tol > 0 && R.relres <= tol) {
            if (!confirm) {   // the estimate reached the tolerance: the caller checks
                R.converged = true;
                return R;
            }
            continue;   // confirm with the recomputed residual before declaring convergence
        }
    }
    if (tol > 0) {
        void *r = vec_at(c, prec, V, 0);
        op_schur(c, prec, x, r, t);
        axpby(e, prec, 1.0, 0.0, b, -1.0, 0.0, r);
        R.relres = std::sqrt(norm2_of(c, prec, r)) / bnorm;
        R.converged = R.relres <= tol;
    }
    return R;
}

// Richardson(n) from x = 0 on D_S in precision prec (Algorithm 4)
void richardson(lq_ctx *c, int prec, const void *b, void *x, int n, double omega, const char *wsname)
{
    Exec e = c->ex();
    if (n <= 0) {
        zero(e, prec, x);
        return;
    }
    void *t = field(c, prec, (std::string(wsname) + ":t").c_str());
    axpby(e, prec, omega, 0.0, b, 0.0, 0.0, x);   // first sweep: x = 0 + omega (b - D_S 0)
    for (int i = 1; i < n; i++) op_rich_sweep(c, prec, x, b, omega, t);
}

// ---- SAP(n, m), Algorithm 1 ------------------------------------------------------

// block extents of the SAP decomposition: params->sap_block, or 4 along every
// direction that allows it (and the whole extent of a direction of length 2)
void sap_dims(lq_ctx *c, const lq_solver_params *p, int b[4])
{
    const int *L = c->lat.L;
    for (int mu = 0; mu < 4; mu++) {
        int v = p->sap_block[mu];
        if (v == 0) v = (L[mu] % 4 == 0 && (L[mu] / 4 == 1 || (L[mu] / 4) % 2 == 0)) ? 4 : (L[mu] == 2 ? 2 : -1);
        if (v < 2 || v % 2 || L[mu] % v) fail(c, LQ_ERR_ARG, "SAP block extents must be even and divide the lattice");
        const int n = L[mu] / v;
        if (n != 1 && n % 2) fail(c, LQ_ERR_ARG, "SAP needs an even number of blocks (or one) along each direction");
        b[mu] = v;
    }
    if ((long long)b[0] * b[1] * b[2] * b[3] > 256) fail(c, LQ_ERR_ARG, "SAP blocks hold at most 256 sites");
}

// the first site of every block of each colour (colour = parity of the block
// coordinates' sum), rebuilt when the block extents change
void sap_tables(lq_ctx *c, const int b[4])
{
    if (c->sap_origin[0] && std::equal(b, b + 4, c->sap_b)) return;
    const int *L = c->lat.L;
    std::vector<int4> org[2];
    for (int t = 0; t < L[3] / b[3]; t++)
        for (int z = 0; z < L[2] / b[2]; z++)
            for (int y = 0; y < L[1] / b[1]; y++)
                for (int x = 0; x < L[0] / b[0]; x++)
                    org[(x + y + z + t) & 1].push_back(make_int4(x * b[0], y * b[1], z * b[2], t * b[3]));
    for (int col = 0; col < 2; col++) {
        const size_t bytes = sizeof(int4) * (org[col].size() ? org[col].size() : 1);
        c->sap_origin[col] = (int4 *)ws(c, col ? "sap:org1" : "sap:org0", bytes);
        if (!org[col].empty())
            ck(c, cudaMemcpy(c->sap_origin[col], org[col].data(), sizeof(int4) * org[col].size(),
                             cudaMemcpyHostToDevice),
               "cudaMemcpy H2D");
        c->sap_count[col] = (int)org[col].size();
    }
    std::copy(b, b + 4, c->sap_b);
}

// The block-major copies of the FP32 links and clover fields that the SAP
// block solves read, made on first use for a gauge field and block shape.
void need_sap_block_major(lq_ctx *c, const int b[4])
{
    if (std::equal(b, b + 4, c->sapbm_b)) return;
    Exec e = c->ex();
    const size_t lb = (size_t)4 * 3 * c->g.stride * 16, cb = (size_t)2 * 9 * c->g.stride * 16;
    for (int p = 0; p < 2; p++) {
        sap_block_major(e, b, p, 12, c->U32[p], ws(c, p ? "sap:Ub1" : "sap:Ub0", lb));
        sap_block_major(e, b, p, 18, p ? c->Ci32 : c->C32[0], ws(c, p ? "sap:Cb1" : "sap:Cb0", cb));
    }
    std::copy(b, b + 4, c->sapbm_b);
}

// x = SAP(n, m) b from x = 0 on the full lattice, FP32 internal fields
void sap_apply(lq_ctx *c, const lq_solver_params *p, const void *be, const void *bo, void *xe, void *xo)
{
    int b[4];
    sap_dims(c, p, b);
    sap_tables(c, b);
    need_sap_block_major(c, b);
    Exec e = c->ex();
    zero(e, P32, xe);
    zero(e, P32, xo);
    SapLaunch L;
    std::copy(b, b + 4, L.b);
    L.U[0] = c->U32[0];
    L.U[1] = c->U32[1];
    const size_t lb = (size_t)4 * 3 * c->g.stride * 16, cb = (size_t)2 * 9 * c->g.stride * 16;
    L.Ub[0] = ws(c, "sap:Ub0", lb);
    L.Ub[1] = ws(c, "sap:Ub1", lb);
    L.Ce = ws(c, "sap:Cb0", cb);
    L.Ci = ws(c, "sap:Cb1", cb);
    L.x[0] = xe;
    L.x[1] = xo;
    // the blocks' even residual and each colour's last correction, on the
    // sites of that colour's blocks
    void *res_e = field(c, P32, "sap:re");
    void *corr[2] = {field(c, P32, "sap:e0"), field(c, P32, "sap:e1")};
    L.rout_e = res_e;
    L.eout[0] = corr[0];
    L.eout[1] = corr[1];
    L.ro = field(c, P32, "sap:ro");
    L.m = p->smooth_m;
    for (int i = 0; i < p->smooth_n; i++)
        for (int col = 0; col < 2; col++) {
            // a colour's first sweep starts from r = b on its blocks (x is zero
            // there); later sweeps from the residual its last sweep left
            L.rin[0] = i == 0 ? be : res_e;
            L.rin[1] = i == 0 ? bo : nullptr;
            // no correction of the other colour exists before the first launch
            const bool first = i == 0 && col == 0;
            L.eface[0] = first ? nullptr : corr[0];
            L.eface[1] = first ? nullptr : corr[1];
            L.origin = c->sap_origin[col];
            L.count = c->sap_count[col];
            sap_blocks(e, L);
        }
    ck_launch(c, "SAP");
}

// the preconditioner / smoother on D_S: z = M v, both in precision q
long long smoother_schur(lq_ctx *c, const lq_solver_params *p, int q, const void *v, void *z)
{
    if (p->smoother == LQ_SMOOTH_SAP) {
        // the even half of SAP applied to (v, 0): D^{-1} restricted to the even
        // sites is D_S^{-1}
        if (q != P32) fail(c, LQ_ERR_ARG, "SAP runs in LQ_F32 (inner_prec)");
        void *zo = field(c, P32, "sap:zo"), *vo = field(c, P32, "sap:vo");
        zero(c->ex(), P32, vo);
        sap_apply(c, p, v, vo, z, zo);
        return p->smooth_n;
    }
    if (p->smoother == LQ_SMOOTH_RICHARDSON) {
        richardson(c, q, v, z, p->smooth_n, p->omega, "rich");
        return p->smooth_n;
    }
    if (p->smoother == LQ_SMOOTH_GMRES) {
        Exec e = c->ex();
        zero(e, q, z);
        KResult r = gmres(c, q, v, z, p->smooth_m, p->smooth_n, p->smooth_tol, true, "inner", -1.0, false);
        return r.iters;
    }
    copy(c->ex(), q, v, z);
    return 0;
}

// Flexible GMRES(m) in precision W (FP64 or df64), right-preconditioned by the
// smoother in inner_prec.  Stops at ||b - D_S x|| <= tol * bnorm_ref (bnorm_ref < 0:
// the norm of b itself).
KResult fgmres(lq_ctx *c, const lq_solver_params *p, const void *b, void *x, long long *inner_iters,
               double bnorm_ref = -1.0, bool confirm = true, int max_cycles = -1)
{
    if (max_cycles < 0) max_cycles = p->max_restarts;
    Exec e = c->ex();
    KResult R;
    const int m = p->restart;
    const int q = p->inner_prec;
    const int W = p->prec;
    void *V = basis(c, W, "outerV", m + 1);
    void *Z = basis(c, W, "outerZ", m);
    void *t = field(c, W, "outer:t");
    void *vq = q == W ? nullptr : field(c, q, "prec:v");
    void *zq = q == W ? nullptr : field(c, q, "prec:z");
    const double bnorm = bnorm_ref >= 0 ? bnorm_ref : std::sqrt(norm2_of(c, W, b));
    if (!std::isfinite(bnorm)) fail(c, LQ_ERR_NAN, "NaN/Inf in the right-hand side");
    if (bnorm == 0.0) {
        zero(e, W, x);
        R.converged = true;
        return R;
    }
    Hess H(m);
    for (int cyc = 0; cyc < max_cycles; cyc++) {
        void *v0 = vec_at(c, W, V, 0);
        op_schur(c, W, x, v0, t);
        axpby(e, W, 1.0, 0.0, b, -1.0, 0.0, v0);
        const double beta = std::sqrt(norm2_of(c, W, v0));
        if (!std::isfinite(beta)) fail(c, LQ_ERR_NAN, "NaN/Inf in the residual");
        R.relres = beta / bnorm;
        if (beta <= p->tol * bnorm) {
            R.converged = true;
            return R;
        }
        R.cycles++;
        axpby(e, W, 0.0, 0.0, v0, 1.0 / beta, 0.0, v0);
        H.reset(beta);
        int nk = 0;
        for (int k = 0; k < m; k++) {
            void *vk = vec_at(c, W, V, k);
            void *zk = vec_at(c, W, Z, k);
            if (q == W) {
                *inner_iters += smoother_schur(c, p, W, vk, zk);
            } else {
                convert(e, W, vk, q, vq);
                *inner_iters += smoother_schur(c, p, q, vq, zq);
                convert(e, q, zq, W, zk);
            }
            void *w = vec_at(c, W, V, k + 1);
            op_schur(c, W, zk, w, t);
            const double hk1 = arnoldi_cgs2(c, W, V, k, w, H);
            double colnorm2 = hk1 * hk1;
            for (int j = 0; j <= k; j++) colnorm2 += std::norm(H.h(j, k));
            H.h(k + 1, k) = hk1;
            const double est = H.rotate(k);
            nk = k + 1;
            R.iters++;
            R.relres = est / bnorm;
            const bool breakdown = hk1 <= 1e-14 * std::sqrt(colnorm2);
            if (breakdown || est <= p->tol * bnorm || k == m - 1) break;
            axpby(e, W, 0.0, 0.0, w, 1.0 / hk1, 0.0, w);
        }
        std::vector<cd> y = H.solve(nk);
        upload_coef(c, y);
        multi_axpy(e, W, Z, nk, c->d_coef, +1, x, nullptr, 0);
        ck_launch(c, "fgmres update");
        if (!confirm && R.relres <= p->tol) {   // the estimate reached the tolerance: the caller checks
            R.converged = true;
            return R;
        }
    }
    void *r = vec_at(c, W, V, 0);
    op_schur(c, W, x, r, t);
    axpby(e, W, 1.0, 0.0, b, -1.0, 0.0, r);
    R.relres = std::sqrt(norm2_of(c, W, r)) / bnorm;
    R.converged = R.relres <= p->tol;
    return R;
}

void check_params(lq_ctx *c, const lq_solver_params *p, bool solve)
{
    if (!p) fail(c, LQ_ERR_ARG, "params is NULL");
    if (solve) {
        if (p->solver != LQ_SOLVER_GMRES && p->solver != LQ_SOLVER_FGMRES) fail(c, LQ_ERR_ARG, "bad solver");
        if (p->restart < 1 || p->restart > MAX_RESTART) fail(c, LQ_ERR_ARG, "restart out of range 1..256");
        if (p->max_restarts < 1) fail(c, LQ_ERR_ARG, "max_restarts < 1");
        if (!(p->tol > 0.0) || !std::isfinite(p->tol)) fail(c, LQ_ERR_ARG, "tol must be positive");
        if (!valid_prec(p->prec)) fail(c, LQ_ERR_ARG, "bad prec");
        if (p->solver == LQ_SOLVER_FGMRES && p->prec == LQ_F32)
            fail(c, LQ_ERR_ARG, "the FGMRES outer iteration needs LQ_F64 or LQ_DF64");
    }
    if (p->smoother < LQ_SMOOTH_NONE || p->smoother > LQ_SMOOTH_SAP) fail(c, LQ_ERR_ARG, "bad smoother");
    if (p->smoother == LQ_SMOOTH_SAP && (p->inner_prec != LQ_F32 || p->smooth_m < 0))
        fail(c, LQ_ERR_ARG, "SAP runs in LQ_F32 with smooth_m >= 0 Minimal Residual steps");
    if (!valid_prec(p->inner_prec) && p->inner_prec != LQ_BF16) fail(c, LQ_ERR_ARG, "bad inner_prec");
    if (p->inner_prec == LQ_BF16 && p->smoother != LQ_SMOOTH_RICHARDSON)
        fail(c, LQ_ERR_ARG, "LQ_BF16 storage is offered for the Richardson smoother");
    if (p->smoother != LQ_SMOOTH_NONE && p->smooth_n < 0) fail(c, LQ_ERR_ARG, "smooth_n < 0");
    if (p->smoother == LQ_SMOOTH_GMRES && (p->smooth_m < 1 || p->smooth_m > MAX_RESTART))
        fail(c, LQ_ERR_ARG, "smooth_m out of range 1..256");
    if (p->smoother == LQ_SMOOTH_RICHARDSON && !std::isfinite(p->omega)) fail(c, LQ_ERR_ARG, "omega not finite");
    if (p->smoother == LQ_SMOOTH_GMRES && !(p->smooth_tol >= 0.0)) fail(c, LQ_ERR_ARG, "smooth_tol < 0");
}

// ---- batched right-hand sides over one or several lattices -------------------------

// out = D_S in for N consecutive fields of one lattice: one batched K1 and one
// batched K2 launch (the df64 defect of the batched solve)
void op_schur_n(lq_ctx *c, int prec, const void *in, void *out, void *t, int N)
{
    Exec e = c->ex();
    HopCall k1 = hopcall(c, HOP_K1, prec, 1);
    k1.in = in;
    k1.out = t;
    k1.clov = Cip(c, prec);
    k1.nrhs = N;
    hop(e, k1);
    HopCall k2 = hopcall(c, HOP_K2, prec, 0);
    k2.in = t;
    k2.in2 = in;
    k2.out = out;
    k2.clov = Cp(c, prec, 0);
    k2.nrhs = N;
    hop(e, k2);
}

}  // namespace

// A batched solve over the right-hand sides of one or several lattices (contexts
// on one device).  The inner FP32 GMRES treats every right-hand side of every
// member as one system of a batch: each operator launch is one persistent grid
// walking a work table over all members' sites and right-hand sides, the BLAS
// launches cover all systems, and the Givens bookkeeping runs on the device, so
// that a cycle is a short sequence of captured CUDA graphs.  The outer df64
// defect correction runs per member.
struct lq_group {
    std::vector<lq_ctx *> mem;
    cudaStream_t user = nullptr;   // stream of the group's calls
    cudaStream_t st = nullptr;     // private stream (graph capture)
    cudaEvent_t ev = nullptr;
    bool autotune = true;
    int pin_spt = 32, pin_rpt = 1, pin_factor = 2;   // the shape used without autotuning
    // layout of the current signature: right-hand sides per member, cycle length
    std::vector<int> nrhs;
    int N = 0, m = 0;
    long long mf = 0;              // float4 vectors per multi-field
    std::vector<long long> off;    // first field of each member in a multi-field
    std::vector<int> first;        // first system of each member
    Segs S;
    LatDesc *desc = nullptr;
    int4 *tiles = nullptr;
    int ntiles = 0, max_tiles = 0, blas_default = 1, blas_max = 1;
    double k1_bytes = 0, k2_bytes = 0, k1_flops = 0, k2_flops = 0;
    struct {
        int spt = 32, rpt = 1, grid = 0, blas = 0;
        float hop_ms = 0.0f, blas_ms = 0.0f;
        bool tuned = false;
    } tune;
    void *V = nullptr, *T = nullptr, *X = nullptr, *B = nullptr;
    BatchRed br{};
    KState ks{};
    std::vector<BatchRed> mbr;     // per-member df64 norms of the outer iteration
    std::vector<cudaGraphExec_t> gexec;
    std::vector<long long> cap_launches;
    std::vector<double> cap_bytes;
    double *h = nullptr;           // pinned: est / norms [N], targets [N], norms [N]
    int *hact = nullptr;           // pinned: active flags [N]
    double *h_dev = nullptr;       // device mappings of h and hact (written by get_values / get_ints)
    int *hact_dev = nullptr;
    std::vector<void *> owned;
};

namespace {

// the context that records the group's errors, launches and profile: member 0
lq_ctx *gctx(lq_group *G) { return G->mem[0]; }

Exec gexec(lq_group *G)
{
    lq_ctx *c = G->mem[0];
    return Exec{c->g, G->st, &c->ctr, &c->prof};
}

void *galloc(lq_group *G, size_t bytes)
{
    lq_ctx *c = gctx(G);
    void *p = nullptr;
    ck(c, cudaMalloc(&p, bytes), "cudaMalloc");
    G->owned.push_back(p);
    ck(c, cudaMemsetAsync(p, 0, bytes, G->st), "cudaMemsetAsync");
    return p;
}

// drop everything that depends on the layout
void group_release(lq_group *G)
{
    if (G->st) cudaStreamSynchronize(G->st);
    for (cudaGraphExec_t g : G->gexec)
        if (g) cudaGraphExecDestroy(g);
    G->gexec.clear();
    G->cap_launches.clear();
    G->cap_bytes.clear();
    for (void *p : G->owned) cudaFree(p);
    G->owned.clear();
    if (G->h) cudaFreeHost(G->h);
    if (G->hact) cudaFreeHost(G->hact);
    G->h = nullptr;
    G->hact = nullptr;
    G->nrhs.clear();
    G->N = G->m = 0;
    G->tune.tuned = false;
}

// the work table of the batched hop for `spt` sites per tile: per member, per
// site block, its right-hand-side groups (so the tiles of one site block follow
// one another)
void group_tiles(lq_group *G, int spt, int per_thread = 1)
{
    // right-hand sides per tile; the staged form (per_thread 0) covers all of them
    const int rpt = per_thread * (kHopBlock / spt);
    std::vector<int4> t;
    for (size_t l = 0; l < G->mem.size(); l++) {
        const long long sb = (G->mem[l]->g.Vh + spt - 1) / spt;
        const int groups = per_thread == 0 ? 1 : (G->nrhs[l] + rpt - 1) / rpt;
        for (long long b = 0; b < sb; b++)
            for (int q = 0; q < groups; q++) t.push_back(make_int4((int)l, (int)b, q * rpt, 0));
    }
    lq_ctx *c = gctx(G);
    if ((int)t.size() > G->max_tiles) fail(c, LQ_ERR_STATE, "work table larger than its buffer");
    ck(c, cudaMemcpyAsync(G->tiles, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice, G->st),
       "cudaMemcpyAsync H2D");
    ck(c, cudaStreamSynchronize(G->st), "cudaStreamSynchronize");
    G->ntiles = (int)t.size();
    G->tune.spt = spt;
    G->tune.rpt = per_thread;
}

// persistent grid: `factor` times the resident blocks of the whole GPU (0: one
// block per tile)
int group_grid(lq_group *G, int factor)
{
    if (factor == 0) return G->ntiles;
    int sms = 0;
    ck(gctx(G), cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, gctx(G)->device), "cudaDeviceGetAttribute");
    const long long g = (long long)factor * hop_group_resident(G->tune.rpt, G->tune.spt) * sms;
    return (int)(g < G->ntiles ? g : G->ntiles);
}

void group_setup(lq_group *G, const std::vector<int> &nrhs, int m)
{
    lq_ctx *c = gctx(G);
    if (!G->st) {
        ck(c, cudaStreamCreateWithFlags(&G->st, cudaStreamNonBlocking), "cudaStreamCreate");
        ck(c, cudaEventCreateWithFlags(&G->ev, cudaEventDisableTiming), "cudaEventCreate");
    }
    if (G->nrhs == nrhs && G->m == m) return;
    group_release(G);
    const int M = (int)G->mem.size();
    int N = 0;
    long long mf = 0, maxfs = 0;
    double sites = 0.0;
    G->off.assign(M, 0);
    G->first.assign(M, 0);
    std::vector<longlong2> seg;
    std::vector<LatDesc> desc(M);
    G->k1_bytes = G->k2_bytes = G->k1_flops = G->k2_flops = 0.0;
    long long max_tiles = 0;
    for (int l = 0; l < M; l++) {
        lq_ctx *ml = G->mem[l];
        const long long fs = 6 * ml->g.stride;
        G->off[l] = mf;
        G->first[l] = N;
        for (int r = 0; r < nrhs[l]; r++) seg.push_back(make_longlong2(mf + r * fs, fs));
        LatDesc &d = desc[l];
        d.g = ml->g;
        d.U[0] = (const float4 *)ml->U32[0];
        d.U[1] = (const float4 *)ml->U32[1];
        d.clov[0] = (const float4 *)ml->C32[0];
        d.clov[1] = (const float4 *)ml->Ci32;
        d.off = mf;
        d.fs = fs;
        d.nrhs = nrhs[l];
        mf += nrhs[l] * fs;
        N += nrhs[l];
        maxfs = fs > maxfs ? fs : maxfs;
        sites += (double)nrhs[l] * ml->g.Vh;
        G->k1_bytes += hop_bytes(HOP_K1, P32, nrhs[l], (double)ml->g.Vh);
        G->k2_bytes += hop_bytes(HOP_K2, P32, nrhs[l], (double)ml->g.Vh);
        G->k1_flops += hop_flops(HOP_K1, (double)ml->g.Vh * nrhs[l]);
        G->k2_flops += hop_flops(HOP_K2, (double)ml->g.Vh * nrhs[l]);
        max_tiles += (ml->g.Vh + 15) / 16 * ((nrhs[l] + 7) / 8) + (ml->g.Vh + 127) / 128 * nrhs[l] +
                     (ml->g.Vh + 63) / 64 * ((nrhs[l] + 1) / 2) + (ml->g.Vh + 31) / 32 * ((nrhs[l] + 3) / 4) +
                     (ml->g.Vh + 31) / 32;
    }
    G->N = N;
    G->m = m;
    G->mf = mf;
    G->max_tiles = (int)max_tiles;
    G->blas_default = batch_blocks(maxfs, N);
    G->blas_max = 2 * G->blas_default;
    G->S.seg = (const longlong2 *)galloc(G, sizeof(longlong2) * N);
    ck(c, cudaMemcpyAsync((void *)G->S.seg, seg.data(), sizeof(longlong2) * N, cudaMemcpyHostToDevice, G->st),
       "cudaMemcpyAsync H2D");
    G->desc = (LatDesc *)galloc(G, sizeof(LatDesc) * M);
    ck(c, cudaMemcpyAsync(G->desc, desc.data(), sizeof(LatDesc) * M, cudaMemcpyHostToDevice, G->st),
       "cudaMemcpyAsync H2D");
    ck(c, cudaStreamSynchronize(G->st), "cudaStreamSynchronize");
    G->S.n = 0;
    G->S.sites = sites;
    G->S.blocks = G->blas_default;
    G->tiles = (int4 *)galloc(G, sizeof(int4) * (size_t)max_tiles);
    const size_t mfb = (size_t)mf * 16;
    G->V = galloc(G, (size_t)(m + 1) * mfb);
    G->T = galloc(G, mfb);
    G->X = galloc(G, mfb);
    G->B = galloc(G, mfb);
    G->br.blocks = G->blas_default;
    G->br.pitch = 2 * (2 * m + 2);
    G->br.partial = (double *)galloc(G, sizeof(double) * (size_t)N * G->blas_max * G->br.pitch);
    G->br.out = (double *)galloc(G, sizeof(double) * (size_t)N * G->br.pitch);
    KState &k = G->ks;
    k.N = N;
    k.m = m;
    k.H = (double2 *)galloc(G, sizeof(double2) * (size_t)N * (m + 1) * m);
    k.cs = (double *)galloc(G, sizeof(double) * (size_t)N * m);
    k.sn = (double2 *)galloc(G, sizeof(double2) * (size_t)N * m);
    k.g = (double2 *)galloc(G, sizeof(double2) * (size_t)N * (m + 1));
    k.y = (double2 *)galloc(G, sizeof(double2) * (size_t)N * m);
    k.active = (int *)galloc(G, sizeof(int) * N);
    k.kused = (int *)galloc(G, sizeof(int) * N);
    k.nanflag = (int *)galloc(G, sizeof(int));
    k.scale = (double *)galloc(G, sizeof(double) * N);
    k.est = (double *)galloc(G, sizeof(double) * N);
    k.target = (double *)galloc(G, sizeof(double) * N);
    G->mbr.assign(M, BatchRed{});
    for (int l = 0; l < M; l++) {
        BatchRed &b = G->mbr[l];
        b.blocks = batch_blocks(12 * G->mem[l]->g.stride, nrhs[l]);
        b.pitch = 2;
        b.partial = (double *)galloc(G, sizeof(double) * (size_t)nrhs[l] * b.blocks * b.pitch);
        b.out = (double *)galloc(G, sizeof(double) * (size_t)nrhs[l] * b.pitch);
    }
    ck(c, cudaMallocHost((void **)&G->h, sizeof(double) * 3 * N), "cudaMallocHost");
    ck(c, cudaMallocHost((void **)&G->hact, sizeof(int) * N), "cudaMallocHost");
    ck(c, cudaHostGetDevicePointer((void **)&G->h_dev, G->h, 0), "cudaHostGetDevicePointer");
    ck(c, cudaHostGetDevicePointer((void **)&G->hact_dev, G->hact, 0), "cudaHostGetDevicePointer");
    G->nrhs = nrhs;
    group_tiles(G, G->pin_spt, G->pin_rpt);
    G->tune.grid = group_grid(G, G->pin_factor);
    G->tune.blas = G->blas_default;
    G->tune.tuned = false;
}

// out = D_S in for every system (two persistent launches over the work table)
void group_schur(lq_group *G, const void *in, void *out)
{
    Exec e = gexec(G);
    hop_group(e, HOP_K1, G->desc, G->tiles, G->ntiles, G->tune.grid, G->tune.spt, G->tune.rpt, in, nullptr, G->T,
              G->k1_bytes, G->k1_flops);
    hop_group(e, HOP_K2, G->desc, G->tiles, G->ntiles, G->tune.grid, G->tune.spt, G->tune.rpt, G->T, in, out,
              G->k2_bytes, G->k2_flops);
}

void group_set_blas(lq_group *G, int blocks)
{
    G->tune.blas = blocks;
    G->S.blocks = blocks;
    G->br.blocks = blocks;
}

// The autotuner: times every candidate launch shape on the group's own buffers
// (CUDA events, after a warm-up launch) and keeps the fastest.
//   batched hop: one or two right-hand sides per thread x sites per tile 16,
//     32, 64, 128 (with 8, 4, 2, 1 threads along the right-hand sides) x grid =
//     1 or 2 times the resident blocks (persistent) or one block per tile;
//   batched BLAS: blocks per system 1/2, 1, 2 times the default, on a
//     multi-dot and a multi-axpy over min(m, 8) basis vectors.
// Launch counts and bytes of the trials are not recorded.
void group_tune(lq_group *G)
{
    lq_ctx *c = gctx(G);
    const Counters saved = c->ctr;
    const bool prof = c->prof.on;
    c->prof.on = false;
    cudaEvent_t a = nullptr, b = nullptr;
    ck(c, cudaEventCreate(&a), "cudaEventCreate");
    ck(c, cudaEventCreate(&b), "cudaEventCreate");
    auto timed = [&](auto fn) {
        fn();
        cudaEventRecord(a, G->st);
        for (int i = 0; i < 3; i++) fn();
        cudaEventRecord(b, G->st);
        ck(c, cudaEventSynchronize(b), "cudaEventSynchronize");
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        return ms / 3.0f;
    };
    float best = 1e30f;
    int best_spt = 32, best_rpt = 1, best_factor = 2;
    for (int rpt : {1, 2, 0})
        for (int spt : {32, 64, 16, 128}) {
            if (rpt == 0 && spt != 32 && spt != 64) continue;   // staged form: 32 or 64 sites per tile
            group_tiles(G, spt, rpt);
            for (int factor : {1, 2, 0}) {
                G->tune.grid = group_grid(G, factor);
                const float t = timed([&] { group_schur(G, G->X, G->V); });
                if (t < best) {
                    best = t;
                    best_spt = spt;
                    best_rpt = rpt;
                    best_factor = factor;
                }
            }
        }
    group_tiles(G, best_spt, best_rpt);
    G->tune.grid = group_grid(G, best_factor);
    G->tune.hop_ms = best;
    const int nv = G->m < 8 ? G->m : 8;
    Exec e = gexec(G);
    float bbest = 1e30f;
    int bblocks = G->blas_default;
    for (int blocks : {G->blas_default, G->blas_default / 2, 2 * G->blas_default}) {
        if (blocks < 1 || blocks > G->blas_max) continue;
        group_set_blas(G, blocks);
        const float t = timed([&] {
            bdot(e, G->S, G->V, G->mf, nv, G->T, G->N, G->br, 0);
            baxpy(e, G->S, G->V, G->mf, nv, G->br.out, G->br.pitch / 2, -1, G->T, G->N, &G->br, nv);
        });
        if (t < bbest) {
            bbest = t;
            bblocks = blocks;
        }
    }
    group_set_blas(G, bblocks);
    G->tune.blas_ms = bbest;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ck(c, cudaMemsetAsync(G->T, 0, (size_t)G->mf * 16, G->st), "cudaMemsetAsync");
    ck(c, cudaStreamSynchronize(G->st), "cudaStreamSynchronize");
    c->ctr = saved;
    c->prof.on = prof;
    G->tune.tuned = true;
}

// One cycle of batched GMRES(m) in FP32 on D_S (Algorithm 2 for each system), in
// three kinds of segment, each a fixed launch sequence without host
// synchronisation:
//   start:  r = B - D_S X, beta = ||r||, g = beta e_1, V_0 = r / beta
//   steps:  Arnoldi steps [k0, k1): w = D_S v_k, one Gram-Schmidt pass with the
//           new norm fused, Givens on the device, v_{k+1}
//   finish: y = R^{-1} g, X += V y
static constexpr int BATCH_SEG = 4;   // Arnoldi steps per segment

void group_start(lq_group *G)
{
    Exec e = gexec(G);
    group_schur(G, G->X, G->V);
    bxmy(e, G->S, G->B, G->V, G->N);   // V_0 = B - D_S X
    bnorm(e, P32, G->S, G->V, G->N, G->br, 0);
    bfinish(e, G->br, G->N, 0, 1);
    ks_init(e, G->ks, G->br.out, G->br.pitch);
    bscale(e, G->S, G->V, G->ks.scale, G->V, G->N);
}

void group_steps(lq_group *G, int k0, int k1)
{
    Exec e = gexec(G);
    auto Vj = [&](int j) { return (char *)G->V + (size_t)j * G->mf * 16; };
    for (int k = k0; k < k1; k++) {
        group_schur(G, Vj(k), Vj(k + 1));
        const int nv = k + 1;
        bdot(e, G->S, G->V, G->mf, nv, Vj(k + 1), G->N, G->br, 0);
        bfinish(e, G->br, G->N, 0, nv);
        baxpy(e, G->S, G->V, G->mf, nv, G->br.out, G->br.pitch / 2, -1, Vj(k + 1), G->N, &G->br, nv);
        bfinish(e, G->br, G->N, nv, 1);
        ks_step(e, G->ks, k, 1, G->br.out, G->br.pitch);
        bscale(e, G->S, Vj(k + 1), G->ks.scale, Vj(k + 1), G->N);
    }
}

void group_finish(lq_group *G)
{
    Exec e = gexec(G);
    ks_solve(e, G->ks);
    baxpy(e, G->S, G->V, G->mf, G->m, (const double *)G->ks.y, G->m, +1, G->X, G->N, nullptr, 0);
}

// Segment `id` (0 start, 1..nseg steps, nseg+1 finish): replayed from its CUDA
// graph, captured on first use; launched eagerly while per-launch profiling is
// on.  Launches and bytes are counted on every replay.
void group_segment(lq_group *G, int id)
{
    lq_ctx *c = gctx(G);
    const int nseg = (G->m + BATCH_SEG - 1) / BATCH_SEG;
    auto body = [&]() {
        if (id == 0) group_start(G);
        else if (id <= nseg) group_steps(G, (id - 1) * BATCH_SEG, std::min(G->m, id * BATCH_SEG));
        else group_finish(G);
    };
    if (c->prof.on) {
        body();
        ck_launch(c, "batched segment");
        return;
    }
    if ((int)G->gexec.size() < nseg + 2) {
        G->gexec.resize(nseg + 2, nullptr);
        G->cap_launches.resize(nseg + 2, 0);
        G->cap_bytes.resize(nseg + 2, 0.0);
    }
    if (!G->gexec[id]) {
        const long long l0 = c->ctr.launches;
        const double b0 = c->ctr.bytes;
        ck(c, cudaStreamBeginCapture(G->st, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        body();
        cudaGraph_t graph = nullptr;
        const cudaError_t err = cudaStreamEndCapture(G->st, &graph);
        ck(c, err, "cudaStreamEndCapture");
        const cudaError_t ierr = cudaGraphInstantiate(&G->gexec[id], graph, 0);
        cudaGraphDestroy(graph);
        ck(c, ierr, "cudaGraphInstantiate");
        G->cap_launches[id] = c->ctr.launches - l0;
        G->cap_bytes[id] = c->ctr.bytes - b0;
        c->ctr.launches = l0;
        c->ctr.bytes = b0;
    }
    ck(c, cudaGraphLaunch(G->gexec[id], G->st), "cudaGraphLaunch");
    c->ctr.launches += G->cap_launches[id];
    c->ctr.bytes += G->cap_bytes[id];
}

// One inner cycle: start, step segments until every system has left the cycle
// (host check of the active flags between segments), finish.  Returns the
// Arnoldi steps launched.
int group_run_cycle(lq_group *G)
{
    lq_ctx *c = gctx(G);
    const int nseg = (G->m + BATCH_SEG - 1) / BATCH_SEG;
    group_segment(G, 0);
    int steps = 0;
    for (int j = 1; j <= nseg; j++) {
        get_ints(gexec(G), G->ks.active, G->N, G->hact_dev);
        ck_launch(c, "active flags");
        ck(c, cudaStreamSynchronize(G->st), "cudaStreamSynchronize");
        bool any = false;
        for (int r = 0; r < G->N; r++) any = any || G->hact[r];
        if (!any) break;
        group_segment(G, j);
        steps += std::min(G->m, j * BATCH_SEG) - (j - 1) * BATCH_SEG;
    }
    group_segment(G, nseg + 1);
    return steps;
}

// Runs a group solve on the group's private stream (capturable), with every
// member's work redirected there; ordered after the group's stream and every
// member's stream on entry, and before them on exit.
struct OnGroupStream {
    lq_group *G;
    std::vector<cudaStream_t> saved;
    explicit OnGroupStream(lq_group *G_) : G(G_)
    {
        lq_ctx *c = gctx(G);
        ck(c, cudaEventRecord(G->ev, G->user), "cudaEventRecord");
        ck(c, cudaStreamWaitEvent(G->st, G->ev, 0), "cudaStreamWaitEvent");
        for (lq_ctx *m : G->mem) {
            ck(c, cudaEventRecord(G->ev, m->st), "cudaEventRecord");
            ck(c, cudaStreamWaitEvent(G->st, G->ev, 0), "cudaStreamWaitEvent");
        }
        for (lq_ctx *m : G->mem) {
            saved.push_back(m->st);
            m->st = G->st;
        }
    }
    ~OnGroupStream()
    {
        cudaEventRecord(G->ev, G->st);
        for (size_t i = 0; i < G->mem.size(); i++) {
            G->mem[i]->st = saved[i];
            cudaStreamWaitEvent(saved[i], G->ev, 0);
        }
        cudaStreamWaitEvent(G->user, G->ev, 0);
    }
};

template <typename F>
lq_status guarded(lq_ctx *c, F &&f)
{
    if (!c) return LQ_ERR_ARG;
    try {
        int dev = -1;
        cudaGetDevice(&dev);
        if (dev != c->device) ck(c, cudaSetDevice(c->device), "cudaSetDevice");
        f();
        ck(c, cudaGetLastError(), "kernel launch");
        return LQ_OK;
    } catch (const Fail &f) {
        return f.s;
    } catch (const std::bad_alloc &) {
        c->err = "host allocation failed";
        return LQ_ERR_OOM;
    }
}

}  // namespace

// =====================================================================================
// C ABI
// =====================================================================================

namespace lq {
// readers of the index-check flags of every translation unit (checked build)
static std::vector<unsigned (*)(unsigned *)> &bounds_readers()
{
    static std::vector<unsigned (*)(unsigned *)> v;
    return v;
}
void bounds_register(unsigned (*read_clear)(unsigned *first)) { bounds_readers().push_back(read_clear); }
}  // namespace lq

extern "C" {

lq_status lq_bounds_check(int *checked, unsigned long long *violations, int *first_code)
{
    unsigned long long total = 0;
    int first = 0;
#ifdef LQ_BOUNDS
    if (checked) *checked = 1;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return LQ_ERR_CUDA;
    }
    for (auto fn : lq::bounds_readers()) {
        unsigned f = 0;
        const unsigned n = fn(&f);
        if (n && !first) first = (int)f;
        total += n;
    }
    if (cudaGetLastError() != cudaSuccess) return LQ_ERR_CUDA;
#else
    if (checked) *checked = 0;
#endif
    if (violations) *violations = total;
    if (first_code) *first_code = first;
    return total ? LQ_ERR_BOUNDS : LQ_OK;
}

const char *lq_status_string(lq_status s)
{
    switch (s) {
    case LQ_OK: return "LQ_OK";
    case LQ_ERR_ARG: return "LQ_ERR_ARG";
    case LQ_ERR_CUDA: return "LQ_ERR_CUDA";
    case LQ_ERR_OOM: return "LQ_ERR_OOM";
    case LQ_ERR_NOT_CONVERGED: return "LQ_ERR_NOT_CONVERGED";
    case LQ_ERR_BREAKDOWN: return "LQ_ERR_BREAKDOWN";
    case LQ_ERR_NAN: return "LQ_ERR_NAN";
    case LQ_ERR_STATE: return "LQ_ERR_STATE";
    case LQ_ERR_BOUNDS: return "LQ_ERR_BOUNDS";
    }
    return "LQ_ERR_UNKNOWN";
}

const char *lq_last_error(lq_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

lq_status lq_create(lq_ctx **out, const lq_lattice *lat, void *stream)
{
    if (!out || !lat) return LQ_ERR_ARG;
    *out = nullptr;
    for (int mu = 0; mu < 4; mu++)
        if (lat->L[mu] < 2 || lat->L[mu] % 2) return LQ_ERR_ARG;
    if (lat->t_bc != 1 && lat->t_bc != -1) return LQ_ERR_ARG;
    if (!std::isfinite(lat->m0) || !std::isfinite(lat->csw)) return LQ_ERR_ARG;
    const long long V = (long long)lat->L[0] * lat->L[1] * lat->L[2] * lat->L[3];
    if (V >= (1LL << 31)) return LQ_ERR_ARG;   // one FP64 spinor of 2^31 sites would exceed HBM
    lq_ctx *c = new (std::nothrow) lq_ctx();
    if (!c) return LQ_ERR_OOM;
    c->lat = *lat;
    for (int mu = 0; mu < 4; mu++) c->g.L[mu] = lat->L[mu];
    c->g.Lxh = lat->L[0] / 2;
    c->g.tbc = lat->t_bc;
    c->g.V = V;
    c->g.Vh = V / 2;
    c->g.stride = (c->g.Vh + 63) / 64 * 64;
    c->st = (cudaStream_t)stream;
    try {
        ck(c, cudaGetDevice(&c->device), "cudaGetDevice");
        c->red.blocks = reduction_blocks(c->g);
        c->red.maxv = RED_SLOTS;
        c->red.partial = (double *)dev_alloc(c, sizeof(double) * 2 * RED_SLOTS * c->red.blocks);
        c->red.out = (double *)dev_alloc(c, sizeof(double) * 2 * RED_SLOTS);
        c->red.ticket = (unsigned *)dev_alloc(c, sizeof(unsigned));
        c->d_coef = (double *)dev_alloc(c, sizeof(double) * 2 * RED_SLOTS);
        c->d_s2 = (double *)dev_alloc(c, sizeof(double) * RED_SLOTS);
        c->dflag = (int *)dev_alloc(c, sizeof(int));
        // pinned: [0, 2R) red.out mirror, [2R, 4R) coefficients, [4R, 5R) basis scales
        ck(c, cudaMallocHost((void **)&c->h_pin, sizeof(double) * 5 * RED_SLOTS), "cudaMallocHost");
        ck(c, cudaHostGetDevicePointer((void **)&c->h_pin_dev, c->h_pin, 0), "cudaHostGetDevicePointer");
        ck(c, cudaMallocHost((void **)&c->h_int, sizeof(int) * 4), "cudaMallocHost");
        ck(c, cudaHostGetDevicePointer((void **)&c->h_int_dev, c->h_int, 0), "cudaHostGetDevicePointer");
    } catch (const Fail &f) {
        lq_destroy(c);
        return f.s;
    }
    *out = c;
    return LQ_OK;
}

lq_status lq_destroy(lq_ctx *c)
{
    if (!c) return LQ_ERR_ARG;
    if (c->self_group) lq_group_destroy(c->self_group);
    cudaStreamSynchronize(c->st);
    for (void *p : c->owned)
        if (p) cudaFree(p);
    if (c->h_pin) cudaFreeHost(c->h_pin);
    if (c->h_int) cudaFreeHost(c->h_int);
    for (cudaEvent_t ev : c->prof.pool) cudaEventDestroy(ev);
    delete c;
    return LQ_OK;
}

lq_status lq_set_gauge(lq_ctx *c, const void *U)
{
    const NvtxRange range_("lq_set_gauge");
    return guarded(c, [&] {
        if (!U) fail(c, LQ_ERR_ARG, "U is NULL");
        Exec e = c->ex();
        const Geom &g = c->g;
        if (!c->U64[0]) {
            for (int p = 0; p < 2; p++) {
                c->U64[p] = dev_alloc(c, (size_t)4 * 9 * g.stride * 16);
                c->U32[p] = dev_alloc(c, (size_t)4 * 3 * g.stride * 16);
                c->C64[p] = dev_alloc(c, (size_t)2 * 18 * g.stride * 16);
                c->C32[p] = dev_alloc(c, (size_t)2 * 9 * g.stride * 16);
            }
            c->Ci64 = dev_alloc(c, (size_t)2 * 18 * g.stride * 16);
            c->Ci32 = dev_alloc(c, (size_t)2 * 9 * g.stride * 16);
            for (int p = 0; p < 2; p++) {
                c->Udf[p] = dev_alloc(c, (size_t)4 * 9 * g.stride * 16);
                c->Cdf[p] = dev_alloc(c, (size_t)2 * 18 * g.stride * 16);
            }
            c->Cidf = dev_alloc(c, (size_t)2 * 18 * g.stride * 16);
            for (int p = 0; p < 2; p++) c->U16[p] = dev_alloc(c, (size_t)4 * 3 * g.stride * 8);
        }
        c->have_gauge = false;
        c->clover64 = false;
        c->links16 = false;
        c->links64 = false;
        std::fill(c->sapbm_b, c->sapbm_b + 4, 0);
        // links in FP32 and df64; clover and inverse built in df64, their FP32
        // copies rounded by the same kernels (the FP64 links and clover and the
        // BF16 links follow on first use)
        import_links(e, U, nullptr, c->U32, c->Udf);
        const void *udf[2] = {c->Udf[0], c->Udf[1]};
        clover_build(e, udf, c->lat.csw, c->lat.m0, c->Cdf, c->C32, ws(c, "clover:F", (size_t)6 * 9 * 8 * g.V),
                     ws(c, "clover:R", (size_t)6 * 9 * 8 * g.V));
        ck(c, cudaMemsetAsync(c->dflag, 0, sizeof(int), c->st), "cudaMemsetAsync");
        clover_invert(e, c->Cdf[1], c->Cidf, c->Ci32, c->dflag);
        ck_launch(c, "set_gauge kernels");
        get_ints(e, c->dflag, 1, c->h_int_dev);
        ck_launch(c, "set_gauge flag");
        sync(c);
        const int flag = c->h_int[0];
        if (flag) fail(c, LQ_ERR_BREAKDOWN, std::to_string(flag) + " clover blocks with a non-positive pivot");
        c->have_gauge = true;
    });
}

lq_status lq_apply(lq_ctx *c, int op, int prec, const void *in, void *out)
{
    const NvtxRange range_("lq_apply");
    return guarded(c, [&] {
        if (!in || !out) fail(c, LQ_ERR_ARG, "NULL field");
        if (!valid_prec(prec) && prec != LQ_BF16) fail(c, LQ_ERR_ARG, "bad precision");
        if (prec == LQ_BF16 && op != LQ_OP_SCHUR && op != LQ_OP_SCHUR_DAG)
            fail(c, LQ_ERR_ARG, "LQ_BF16 applies LQ_OP_SCHUR and LQ_OP_SCHUR_DAG");
        need_gauge(c);
        Exec e = c->ex();
        void *a = field(c, prec, "apply:a"), *b = field(c, prec, "apply:b");
        void *d = field(c, prec, "apply:d"), *f = field(c, prec, "apply:f");
        switch (op) {
        case LQ_OP_FULL:
            import_full(e, prec, in, a, b);
            op_full(c, prec, a, b, d, f);
            export_full(e, prec, d, f, out);
            break;
        case LQ_OP_SCHUR:
            import_half(e, prec, in, a);
            op_schur(c, prec, a, d, b);
            export_half(e, prec, d, out);
            break;
        case LQ_OP_SCHUR_DAG:
            import_half(e, prec, in, a);
            gamma5(e, prec, a, a);
            op_schur(c, prec, a, d, b);
            gamma5(e, prec, d, d);
            export_half(e, prec, d, out);
            break;
        case LQ_OP_EE:
            import_half(e, prec, in, a);
            clover_mul(e, prec, Cp(c, prec, 0), a, d);
            export_half(e, prec, d, out);
            break;
        case LQ_OP_OO_INV:
            import_half(e, prec, in, a);
            clover_mul(e, prec, Cip(c, prec), a, d);
            export_half(e, prec, d, out);
            break;
        default:
            fail(c, LQ_ERR_ARG, "bad op");
        }
    });
}

lq_status lq_prepare(lq_ctx *c, const void *b, void *bhat_e)
{
    const NvtxRange range_("lq_prepare");
    return guarded(c, [&] {
        if (!b || !bhat_e) fail(c, LQ_ERR_ARG, "NULL field");
        need_gauge(c);
        Exec e = c->ex();
        void *be = field(c, P64, "prep:be"), *bo = field(c, P64, "prep:bo");
        void *t = field(c, P64, "prep:t"), *o = field(c, P64, "prep:o");
        import_full(e, P64, b, be, bo);
        op_prepare(c, P64, be, bo, o, t);
        export_half(e, P64, o, bhat_e);
    });
}

lq_status lq_reconstruct(lq_ctx *c, const void *b, const void *x_e, void *x)
{
    const NvtxRange range_("lq_reconstruct");
    return guarded(c, [&] {
        if (!b || !x_e || !x) fail(c, LQ_ERR_ARG, "NULL field");
        need_gauge(c);
        Exec e = c->ex();
        void *be = field(c, P64, "prep:be"), *bo = field(c, P64, "prep:bo");
        void *xe = field(c, P64, "prep:t"), *xo = field(c, P64, "prep:o");
        import_full(e, P64, b, be, bo);
        import_half(e, P64, x_e, xe);
        op_reconstruct(c, P64, bo, xe, xo);
        export_full(e, P64, xe, xo, x);
    });
}

lq_status lq_estimate_norm(lq_ctx *c, int prec, int iters, const void *v0, double *out)
{
    const NvtxRange range_("lq_estimate_norm");
    return guarded(c, [&] {
        if (!v0 || !out || iters < 1) fail(c, LQ_ERR_ARG, "bad argument");
        if (!valid_prec(prec)) fail(c, LQ_ERR_ARG, "bad precision");
        need_gauge(c);
        Exec e = c->ex();
        void *v = field(c, prec, "pow:v"), *w = field(c, prec, "pow:w");
        void *u = field(c, prec, "pow:u"), *t = field(c, prec, "pow:t");
        import_half(e, prec, v0, v);
        double n0 = norm2_of(c, prec, v);
        if (!(n0 > 0.0) || !std::isfinite(n0)) fail(c, LQ_ERR_ARG, "v0 is zero or not finite");
        axpby(e, prec, 0.0, 0.0, v, 1.0 / std::sqrt(n0), 0.0, v);
        double lam = 0.0;
        for (int i = 0; i < iters; i++) {
            op_schur(c, prec, v, u, t);             // u = D_S v
            gamma5(e, prec, u, u);
            op_schur(c, prec, u, w, t);             // w = D_S^+ D_S v = g5 D_S g5 D_S v
            gamma5(e, prec, w, w);
            lam = std::sqrt(norm2_of(c, prec, w));
            if (!std::isfinite(lam) || lam == 0.0) fail(c, LQ_ERR_NAN, "power iteration produced 0/NaN");
            axpby(e, prec, 1.0 / lam, 0.0, w, 0.0, 0.0, v);
        }
        *out = std::sqrt(lam);
    });
}

lq_status lq_norm2(lq_ctx *c, const void *v, long long n_sites, double *out)
{
    const NvtxRange range_("lq_norm2");
    return guarded(c, [&] {
        if (!v || !out || n_sites < 0) fail(c, LQ_ERR_ARG, "bad argument");
        Exec e = c->ex();
        nat_norm2(e, v, n_sites, c->red, 0);
        reduce_finish(e, c->red, 0, 1);
        ck_launch(c, "norm2");
        *out = fetch(c, 0, 1)[0];
    });
}

lq_status lq_smooth(lq_ctx *c, const lq_solver_params *p, const void *r, void *eo)
{
    const NvtxRange range_("lq_smooth");
    return guarded(c, [&] {
        if (!r || !eo) fail(c, LQ_ERR_ARG, "NULL field");
        check_params(c, p, false);
        need_gauge(c);
        Exec e = c->ex();
        if (p->smoother == LQ_SMOOTH_SAP) {   // Algorithm 1 on the full lattice
            void *be = field(c, P32, "sm:be"), *bo = field(c, P32, "sm:bo");
            void *xe = field(c, P32, "sm:xe"), *xo = field(c, P32, "sm:xo");
            import_full(e, P32, r, be, bo);
            sap_apply(c, p, be, bo, xe, xo);
            export_full(e, P32, xe, xo, eo);
            return;
        }
        const int q = p->inner_prec;
        const int W = p->prec;
        if (W != LQ_F64 && W != LQ_DF64) fail(c, LQ_ERR_ARG, "prec (prepare/reconstruct) must be LQ_F64 or LQ_DF64");
        void *re = field(c, W, "sm:re"), *ro = field(c, W, "sm:ro");
        void *rh = field(c, W, "sm:rh"), *t = field(c, W, "sm:t");
        void *ee = field(c, W, "sm:ee"), *eodd = field(c, W, "sm:eo");
        import_full(e, W, r, re, ro);
        op_prepare(c, W, re, ro, rh, t);
        if (q == W) {
            smoother_schur(c, p, W, rh, ee);
        } else {
            void *rq = field(c, q, "sm:rq"), *eq = field(c, q, "sm:eq");
            convert(e, W, rh, q, rq);
            smoother_schur(c, p, q, rq, eq);
            convert(e, q, eq, W, ee);
        }
        op_reconstruct(c, W, ro, ee, eodd);
        export_full(e, W, ee, eodd, eo);
    });
}

lq_status lq_solve(lq_ctx *c, const lq_solver_params *p, const void *b, void *x, lq_stats *stats)
{
    const NvtxRange range_("lq_solve");
    bool not_conv = false;
    auto t0 = std::chrono::steady_clock::now();
    const long long l0 = c ? c->ctr.launches : 0;
    const double b0 = c ? c->ctr.bytes : 0.0;
    lq_stats st{};
    lq_status s = guarded(c, [&] {
        if (!b || !x) fail(c, LQ_ERR_ARG, "NULL field");
        check_params(c, p, true);
        need_gauge(c);
        Exec e = c->ex();
        // precision of prepare, reconstruct and the true residual: FP64 or df64
        const int W = p->prec == LQ_F32 ? (int)P64 : p->prec;
        void *be = field(c, W, "sol:be"), *bo = field(c, W, "sol:bo");
        void *xe = field(c, W, "sol:xe"), *xo = field(c, W, "sol:xo");
        void *bh = field(c, W, "sol:bh"), *t = field(c, W, "sol:t");
        import_full(e, W, b, be, bo);
        import_full(e, W, x, xe, xo);
        op_prepare(c, W, be, bo, bh, t);
        // The tolerance is on the full system, ||b - D x|| <= tol ||b||.  After the
        // reconstruction of Eq. 2 the odd residual vanishes and the even one is
        // b_hat_e - D_S x_e, so the Schur solve is measured against ||b||, not ||b_hat_e||.
        norm2(e, W, be, c->red, 0);
        norm2(e, W, bo, c->red, 1);
        reduce_finish(e, c->red, 0, 2);
        ck_launch(c, "norm of b");
        const double *hb = fetch(c, 0, 2);
        const double bfull = std::sqrt(hb[0] + hb[2]);
        // The Krylov solver returns once its least-squares estimate reaches the
        // tolerance; the check is the full system's residual recomputed after
        // the reconstruction (which is also the reported true residual).  Should
        // it miss the tolerance, the solve resumes from the current x_e.
        void *ye = field(c, W, "sol:ye"), *yo = field(c, W, "sol:yo");
        KResult R;
        long long inner = 0;
        int cycles_left = p->max_restarts;
        bool conv = false, est_conv = false;
        double rel_true = 0.0;
        for (;;) {
            KResult r;
            if (p->solver == LQ_SOLVER_GMRES) {
                if (p->prec != LQ_F32) {
                    r = gmres(c, W, bh, xe, p->restart, cycles_left, p->tol, false, "outerV", bfull, false);
                } else {
                    void *bq = field(c, P32, "sol:bq"), *xq = field(c, P32, "sol:xq");
                    convert(e, W, bh, P32, bq);
                    convert(e, W, xe, P32, xq);
                    r = gmres(c, P32, bq, xq, p->restart, cycles_left, p->tol, false, "outerV", bfull, false);
                    convert(e, P32, xq, W, xe);
                }
            } else {
                r = fgmres(c, p, bh, xe, &inner, bfull, false, cycles_left);
            }
            R.cycles += r.cycles;
            R.iters += r.iters;
            R.relres = r.relres;
            est_conv = r.converged;
            cycles_left -= r.cycles;
            // x_o and the true residual on the full lattice, in W
            op_reconstruct_residual(c, W, be, bo, xe, xo, ye, yo);
            norm2(e, W, ye, c->red, 0);
            norm2(e, W, yo, c->red, 1);
            reduce_finish(e, c->red, 0, 2);
            ck_launch(c, "true residual");
            const double *hv = fetch(c, 0, 2);
            rel_true = bfull > 0 ? std::sqrt(hv[0] + hv[2]) / bfull : 0.0;
            if (!std::isfinite(rel_true)) fail(c, LQ_ERR_NAN, "NaN/Inf in the true residual");
            conv = rel_true <= p->tol;
            // stop when converged, when the solver ran out of cycles without reaching
            // the tolerance, or when it can make no progress
            if (conv || !r.converged || cycles_left <= 0 || r.cycles == 0) break;
        }
        export_full(e, W, xe, xo, x);
        st.rel_resid_true = rel_true;
        st.cycles = R.cycles;
        st.iters = R.iters;
        st.inner_iters = inner;
        // the Schur residual: recomputed by a solver that ran out of cycles; after a
        // stop on the estimate it equals the full residual just computed
        st.rel_resid = est_conv ? rel_true : R.relres;
        not_conv = !conv;
    });
    if (c) {
        st.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        st.launches = c->ctr.launches - l0;
        st.bytes = c->ctr.bytes - b0;
    }
    if (stats) *stats = st;
    if (s == LQ_OK && not_conv) {
        c->err = "tolerance not reached within max_restarts";
        return LQ_ERR_NOT_CONVERGED;
    }
    return s;
}

// ---- batched solves over one or several lattices ------------------------------------

lq_status lq_group_create(lq_group **out, lq_ctx *const *members, int n_members, void *stream)
{
    if (!out || !members || n_members < 1 || n_members > 64) return LQ_ERR_ARG;
    for (int i = 0; i < n_members; i++) {
        if (!members[i]) return LQ_ERR_ARG;
        if (members[i]->device != members[0]->device) {
            members[0]->err = "group members must share one device";
            return LQ_ERR_ARG;
        }
        for (int j = 0; j < i; j++)
            if (members[j] == members[i]) {
                members[0]->err = "a context appears twice in the group";
                return LQ_ERR_ARG;
            }
    }
    lq_group *G = new (std::nothrow) lq_group;
    if (!G) return LQ_ERR_OOM;
    G->mem.assign(members, members + n_members);
    G->user = (cudaStream_t)stream;
    *out = G;
    return LQ_OK;
}

lq_status lq_group_destroy(lq_group *G)
{
    if (!G) return LQ_ERR_ARG;
    group_release(G);
    if (G->ev) cudaEventDestroy(G->ev);
    if (G->st) cudaStreamDestroy(G->st);
    delete G;
    return LQ_OK;
}

lq_status lq_group_set_autotune(lq_group *G, int on)
{
    if (!G) return LQ_ERR_ARG;
    return guarded(gctx(G), [&] {
        G->autotune = on != 0;
        if (!G->autotune) {   // the fixed default shape
            G->pin_spt = 32;
            G->pin_rpt = 1;
            G->pin_factor = 2;
        }
        group_release(G);   // the next solve lays out, tunes (or not) and captures afresh
    });
}

lq_status lq_group_set_shape(lq_group *G, int sites_per_tile, int rhs_per_thread, int grid_factor)
{
    if (!G) return LQ_ERR_ARG;
    return guarded(gctx(G), [&] {
        const int spt = sites_per_tile;
        const bool staged = rhs_per_thread == 0 && (spt == 32 || spt == 64);
        const bool threads = (spt == 16 || spt == 32 || spt == 64 || spt == 128) &&
                             (rhs_per_thread == 1 || rhs_per_thread == 2);
        if (!(staged || threads) || grid_factor < 0 || grid_factor > 2)
            fail(gctx(G), LQ_ERR_ARG, "bad launch shape");
        G->autotune = false;
        G->pin_spt = spt;
        G->pin_rpt = rhs_per_thread;
        G->pin_factor = grid_factor;
        group_release(G);
    });
}

lq_status lq_group_tuning(lq_group *G, int *sites_per_tile, int *rhs_per_thread, int *grid, int *blas_blocks,
                          double *hop_ms, double *blas_ms)
{
    if (!G) return LQ_ERR_ARG;
    if (!G->N) {
        gctx(G)->err = "no solve has run on this group yet";
        return LQ_ERR_STATE;
    }
    if (sites_per_tile) *sites_per_tile = G->tune.spt;
    if (rhs_per_thread) *rhs_per_thread = G->tune.rpt;
    if (grid) *grid = G->tune.grid;
    if (blas_blocks) *blas_blocks = G->tune.blas;
    if (hop_ms) *hop_ms = G->tune.tuned ? G->tune.hop_ms : 0.0;
    if (blas_ms) *blas_ms = G->tune.tuned ? G->tune.blas_ms : 0.0;
    return LQ_OK;
}

lq_status lq_solve_group(lq_group *G, const lq_solver_params *p, const int *n_rhs, const void *const *b,
                         void *const *x, lq_stats *stats)
{
    const NvtxRange range_("lq_solve_group");
    if (!G) return LQ_ERR_ARG;
    lq_ctx *c = gctx(G);
    const int M = (int)G->mem.size();
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<long long> l0(M);
    std::vector<double> by0(M);
    for (int l = 0; l < M; l++) {
        l0[l] = G->mem[l]->ctr.launches;
        by0[l] = G->mem[l]->ctr.bytes;
    }
    int Ntot = 0;
    if (n_rhs)
        for (int l = 0; l < M; l++) Ntot += n_rhs[l] > 0 ? n_rhs[l] : 0;
    std::vector<lq_stats> st(Ntot);
    bool not_conv = false;
    lq_status s = guarded(c, [&] {
        if (!b || !x || !p || !n_rhs) fail(c, LQ_ERR_ARG, "bad argument");
        for (int l = 0; l < M; l++) {
            if (n_rhs[l] < 1 || n_rhs[l] > 256 || !b[l] || !x[l]) fail(c, LQ_ERR_ARG, "bad right-hand sides");
            need_gauge(G->mem[l]);
        }
        if (Ntot > 1024) fail(c, LQ_ERR_ARG, "more than 1024 systems");
        if (p->restart < 1 || p->restart > 64) fail(c, LQ_ERR_ARG, "restart (inner cycle length) out of range 1..64");
        if (p->max_restarts < 1) fail(c, LQ_ERR_ARG, "max_restarts < 1");
        if (!(p->tol > 0.0) || !std::isfinite(p->tol)) fail(c, LQ_ERR_ARG, "tol must be positive");
        if (p->prec != LQ_DF64) fail(c, LQ_ERR_ARG, "the batched outer iteration runs in LQ_DF64");
        if (p->inner_prec != LQ_F32) fail(c, LQ_ERR_ARG, "the batched inner solver runs in LQ_F32");
        if (p->smooth_n < 1) fail(c, LQ_ERR_ARG, "smooth_n (inner cycles) < 1");
        if (!(p->smooth_tol > 0.0 && p->smooth_tol < 1.0)) fail(c, LQ_ERR_ARG, "smooth_tol must be in (0, 1)");
        group_setup(G, std::vector<int>(n_rhs, n_rhs + M), p->restart);
        OnGroupStream on(G);
        if (G->autotune && !G->tune.tuned) group_tune(G);
        const int N = G->N;
        // per member: df64 workspaces of its right-hand sides
        struct MW {
            char *BE, *BO, *BH, *XE, *XO, *R, *T, *E;
            size_t fw, nat;
        };
        std::vector<MW> w(M);
        for (int l = 0; l < M; l++) {
            lq_ctx *ml = G->mem[l];
            const int n = n_rhs[l];
            MW &q = w[l];
            q.fw = spinor_bytes(ml->g, PDF);
            q.nat = (size_t)ml->g.V * 12 * sizeof(double2);
            q.BE = (char *)ws(ml, "bw:be", n * q.fw);
            q.BO = (char *)ws(ml, "bw:bo", n * q.fw);
            q.BH = (char *)ws(ml, "bw:bh", n * q.fw);
            q.XE = (char *)ws(ml, "bw:xe", n * q.fw);
            q.XO = (char *)ws(ml, "bw:xo", n * q.fw);
            q.R = (char *)ws(ml, "bw:r", n * q.fw);
            q.T = (char *)ws(ml, "bw:t", n * q.fw);
            q.E = (char *)ws(ml, "bw:e", n * q.fw);
            Exec e = ml->ex();
            // prepare (Eq. 2) every right-hand side
            for (int r = 0; r < n; r++) {
                import_full(e, PDF, (const char *)b[l] + r * q.nat, q.BE + r * q.fw, q.BO + r * q.fw);
                import_full(e, PDF, (const char *)x[l] + r * q.nat, q.XE + r * q.fw, q.XO + r * q.fw);
                op_prepare(ml, PDF, q.BE + r * q.fw, q.BO + r * q.fw, q.BH + r * q.fw, q.T);
            }
        }
        // df64 norms of one field per right-hand side, all members, into out[N]
        auto norms = [&](char *MW::*f, std::vector<double> &out) {
            for (int l = 0; l < M; l++) {
                lq_ctx *ml = G->mem[l];
                Exec e = ml->ex();
                Segs S1;
                S1.n = 12 * ml->g.stride;
                S1.sites = (double)n_rhs[l] * ml->g.Vh;
                bnorm(e, PDF, S1, w[l].*f, n_rhs[l], G->mbr[l], 0);
                bfinish(e, G->mbr[l], n_rhs[l], 0, 1);
                ck(c, cudaMemcpy2DAsync(G->h + 2 * N + G->first[l], sizeof(double), G->mbr[l].out,
                                        sizeof(double) * G->mbr[l].pitch, sizeof(double), n_rhs[l],
                                        cudaMemcpyDeviceToHost, G->st),
                   "cudaMemcpy2DAsync");
            }
            ck(c, cudaStreamSynchronize(G->st), "cudaStreamSynchronize");
            out.resize(N);
            for (int k = 0; k < N; k++) out[k] = std::sqrt(G->h[2 * N + k]);
        };
        // reference norm of each system: its full right-hand side, so that the stop
        // ||b_hat - D_S x|| <= tol ||b|| is the full system's relative residual after
        // the reconstruction of Eq. 2 (the odd residual vanishes there)
        std::vector<double> bn, bo_n, rn;
        norms(&MW::BE, bn);
        norms(&MW::BO, bo_n);
        for (int k = 0; k < N; k++) bn[k] = std::sqrt(bn[k] * bn[k] + bo_n[k] * bo_n[k]);
        std::vector<int> outer(N, 0);
        std::vector<long long> inner(N, 0);
        bool all = false;
        for (int it = 0; it <= p->max_restarts; it++) {
            // defect: R = b_hat - D_S x in df64, per member
            for (int l = 0; l < M; l++) {
                lq_ctx *ml = G->mem[l];
                op_schur_n(ml, PDF, w[l].XE, w[l].R, w[l].T, n_rhs[l]);
                axpby(ml->ex(), PDF, 1.0, 0.0, w[l].BH, -1.0, 0.0, w[l].R, n_rhs[l]);
            }
            norms(&MW::R, rn);
            all = true;
            for (int k = 0; k < N; k++) {
                if (!std::isfinite(rn[k])) fail(c, LQ_ERR_NAN, "NaN/Inf in a residual");
                st[k].rel_resid = bn[k] > 0 ? rn[k] / bn[k] : 0.0;
                if (st[k].rel_resid > p->tol) all = false;
            }
            if (all || it == p->max_restarts) break;
            // correction: D_S e = R to smooth_tol (relative) with batched FP32 GMRES
            for (int l = 0; l < M; l++) {
                Exec e = G->mem[l]->ex();
                const long long fs = 6 * G->mem[l]->g.stride;
                for (int r = 0; r < n_rhs[l]; r++)
                    convert(e, PDF, w[l].R + r * w[l].fw, P32, (float4 *)G->B + G->off[l] + r * fs);
            }
            ck(c, cudaMemsetAsync(G->X, 0, (size_t)G->mf * 16, G->st), "cudaMemsetAsync");
            for (int k = 0; k < N; k++) {
                const bool done = st[k].rel_resid <= p->tol;
                G->h[N + k] = done ? rn[k] * 2.0 : p->smooth_tol * rn[k];   // converged ones stay idle
                if (!done) outer[k]++;
            }
            put_values(gexec(G), G->h + N, N, G->ks.target);
            ck_launch(c, "inner targets");
            ck(c, cudaMemsetAsync(G->ks.nanflag, 0, sizeof(int), G->st), "cudaMemsetAsync");
            for (int cyc = 0; cyc < p->smooth_n; cyc++) {
                const int steps = group_run_cycle(G);
                get_values(gexec(G), G->ks.est, N, G->h_dev);
                ck_launch(c, "inner estimates");
                ck(c, cudaStreamSynchronize(G->st), "cudaStreamSynchronize");
                bool inner_done = true;
                for (int k = 0; k < N; k++) {
                    if (st[k].rel_resid > p->tol) inner[k] += steps;
                    if (G->h[k] > G->h[N + k]) inner_done = false;
                }
                if (inner_done) break;
            }
            get_ints(gexec(G), G->ks.nanflag, 1, G->hact_dev);
            ck_launch(c, "NaN flag");
            ck(c, cudaStreamSynchronize(G->st), "cudaStreamSynchronize");
            if (G->hact[0]) fail(c, LQ_ERR_NAN, "NaN/Inf in the batched inner solve");
            for (int l = 0; l < M; l++) {
                lq_ctx *ml = G->mem[l];
                Exec e = ml->ex();
                const long long fs = 6 * ml->g.stride;
                for (int r = 0; r < n_rhs[l]; r++)
                    convert(e, P32, (const float4 *)G->X + G->off[l] + r * fs, PDF, w[l].E + r * w[l].fw);
                axpby(e, PDF, 1.0, 0.0, w[l].E, 1.0, 0.0, w[l].XE, n_rhs[l]);
            }
        }
        not_conv = !all;
        // reconstruct (Eq. 2), export, true residual of every right-hand side
        for (int l = 0; l < M; l++) {
            lq_ctx *ml = G->mem[l];
            Exec e = ml->ex();
            const MW &q = w[l];
            void *ye = field(ml, PDF, "bw:ye"), *yo = field(ml, PDF, "bw:yo");
            for (int r = 0; r < n_rhs[l]; r++) {
                const int k = G->first[l] + r;
                op_reconstruct_residual(ml, PDF, q.BE + r * q.fw, q.BO + r * q.fw, q.XE + r * q.fw,
                                        q.XO + r * q.fw, ye, yo);
                export_full(e, PDF, q.XE + r * q.fw, q.XO + r * q.fw, (char *)x[l] + r * q.nat);
                norm2(e, PDF, ye, ml->red, 0);
                norm2(e, PDF, yo, ml->red, 1);
                norm2(e, PDF, q.BE + r * q.fw, ml->red, 2);
                norm2(e, PDF, q.BO + r * q.fw, ml->red, 3);
                reduce_finish(e, ml->red, 0, 4);
                const double *hv = fetch(ml, 0, 4);
                const double bb = hv[4] + hv[6];
                st[k].rel_resid_true = bb > 0 ? std::sqrt((hv[0] + hv[2]) / bb) : 0.0;
                if (!std::isfinite(st[k].rel_resid_true)) fail(c, LQ_ERR_NAN, "NaN/Inf in a true residual");
                st[k].cycles = outer[k];
                st[k].iters = outer[k];
                st[k].inner_iters = inner[k];
            }
        }
        ck(c, cudaStreamSynchronize(G->st), "cudaStreamSynchronize");
    });
    if (stats) {
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        long long nl = 0;
        double nb = 0.0;
        for (int l = 0; l < M; l++) {
            nl += G->mem[l]->ctr.launches - l0[l];
            nb += G->mem[l]->ctr.bytes - by0[l];
        }
        for (int k = 0; k < Ntot; k++) {
            st[k].time_ms = ms;
            st[k].launches = nl;
            st[k].bytes = nb;
            stats[k] = st[k];
        }
    }
    if (s == LQ_OK && not_conv) {
        c->err = "tolerance not reached within max_restarts";
        return LQ_ERR_NOT_CONVERGED;
    }
    return s;
}

lq_status lq_solve_batch(lq_ctx *c, const lq_solver_params *p, int n_rhs, const void *b, void *x, lq_stats *stats)
{
    const NvtxRange range_("lq_solve_batch");
    if (!c) return LQ_ERR_ARG;
    if (!c->self_group) {
        lq_ctx *one[1] = {c};
        const lq_status s = lq_group_create(&c->self_group, one, 1, c->st);
        if (s != LQ_OK) return s;
    }
    c->self_group->user = c->st;
    void *xs[1] = {x};
    const void *bs[1] = {b};
    return lq_solve_group(c->self_group, p, &n_rhs, bs, xs, stats);
}

lq_status lq_export_clover(lq_ctx *c, int which, void *out)
{
    const NvtxRange range_("lq_export_clover");
    return guarded(c, [&] {
        if (!out || (which != 0 && which != 1)) fail(c, LQ_ERR_ARG, "bad argument");
        need_gauge(c);
        need_clover64(c);
        Exec e = c->ex();
        if (which == 0) clover_export(e, c->C64[0], c->C64[1], out);
        else clover_export(e, nullptr, c->Ci64, out);
    });
}

// G = coef grad_U Re(Y^+ D X) for natural full spinors X, Y (df64 throughout)
static void force_apply(lq_ctx *c, const void *X, const void *Y, double coef, void *G)
{
    Exec e = c->ex();
    void *xe = field(c, PDF, "force:xe"), *xo = field(c, PDF, "force:xo");
    void *ye = field(c, PDF, "force:ye"), *yo = field(c, PDF, "force:yo");
    import_full(e, PDF, X, xe, xo);
    import_full(e, PDF, Y, ye, yo);
    const void *Xs[2] = {xe, xo}, *Ys[2] = {ye, yo};
    const void *U[2] = {c->Udf[0], c->Udf[1]};
    void *gam = ws(c, "clover:F", (size_t)6 * 9 * 8 * c->g.V);
    force_insertion(e, Xs, Ys, c->lat.csw, gam);
    force_links(e, U, Xs, Ys, gam, coef, G);
    ck_launch(c, "force");
}

lq_status lq_force(lq_ctx *c, const void *X, const void *Y, double coef, void *G)
{
    const NvtxRange range_("lq_force");
    return guarded(c, [&] {
        if (!X || !Y || !G) fail(c, LQ_ERR_ARG, "NULL field");
        need_gauge(c);
        force_apply(c, X, Y, coef, G);
    });
}

// the two solves of the pseudofermion action; X, Y natural full spinors
static lq_status action_solves(lq_ctx *c, const lq_solver_params *p, const void *phi, void *X, void *Y, double *S,
                               lq_stats st[2], bool *not_conv)
{
    return guarded(c, [&] {
        if (!p || !phi || !X || !Y || !S) fail(c, LQ_ERR_ARG, "bad argument");
        need_gauge(c);
        Exec e = c->ex();
        const size_t nb = (size_t)c->g.V * 12 * 16;
        void *w = ws(c, "force:w", nb);
        auto solve = [&](const void *rhs, void *sol, lq_stats *out) {
            ck(c, cudaMemsetAsync(sol, 0, nb, c->st), "cudaMemsetAsync");
            const lq_status r = lq_solve(c, p, rhs, sol, out);
            if (r == LQ_ERR_NOT_CONVERGED) *not_conv = true;
            else if (r != LQ_OK) throw Fail{r};
        };
        // D^+ = g5 D g5: Y = D^{-+} phi = g5 D^{-1} g5 phi, then X = D^{-1} Y
        gamma5_nat(e, phi, Y);
        solve(Y, w, &st[0]);
        gamma5_nat(e, w, Y);
        solve(Y, X, &st[1]);
        nat_norm2(e, Y, c->g.V, c->red, 0);
        reduce_finish(e, c->red, 0, 1);
        ck_launch(c, "norm2");
        *S = fetch(c, 0, 1)[0];
    });
}

lq_status lq_fermion_action(lq_ctx *c, const lq_solver_params *p, const void *phi, void *X, void *Y, double *S,
                            lq_stats *stats)
{
    const NvtxRange range_("lq_fermion_action");
    lq_stats st[2] = {};
    bool not_conv = false;
    const lq_status s = action_solves(c, p, phi, X, Y, S, st, &not_conv);
    if (stats) {
        stats[0] = st[0];
        stats[1] = st[1];
    }
    if (s == LQ_OK && not_conv) {
        c->err = "tolerance not reached within max_restarts";
        return LQ_ERR_NOT_CONVERGED;
    }
    return s;
}

lq_status lq_fermion_force(lq_ctx *c, const lq_solver_params *p, const void *phi, double *S, void *G,
                           lq_stats *stats)
{
    const NvtxRange range_("lq_fermion_force");
    lq_stats st[2] = {};
    bool not_conv = false;
    lq_status s = guarded(c, [&] {
        if (!G) fail(c, LQ_ERR_ARG, "NULL gradient");
        need_gauge(c);
        const size_t nb = (size_t)c->g.V * 12 * 16;
        void *y = ws(c, "force:y", nb), *x = ws(c, "force:x", nb);
        const lq_status r = action_solves(c, p, phi, x, y, S, st, &not_conv);
        if (r != LQ_OK) throw Fail{r};
        force_apply(c, x, y, -2.0, G);
        sync(c);
    });
    if (stats) {
        stats[0] = st[0];
        stats[1] = st[1];
    }
    if (s == LQ_OK && not_conv) {
        c->err = "tolerance not reached within max_restarts";
        return LQ_ERR_NOT_CONVERGED;
    }
    return s;
}

lq_status lq_profile(lq_ctx *c, int on)
{
    if (!c) return LQ_ERR_ARG;
    c->prof.recs.clear();
    c->prof.next = 0;
    c->prof.on = on != 0;
    return LQ_OK;
}

lq_status lq_profile_read(lq_ctx *c, int cls, long long *launches, double *ms, double *bytes, double *flops)
{
    return guarded(c, [&] {
        if (cls < 0 || cls >= K_COUNT) fail(c, LQ_ERR_ARG, "bad kernel class");
        sync(c);
        long long n = 0;
        double t = 0.0, b = 0.0, f = 0.0;
        for (const auto &r : c->prof.recs) {
            if (r.cls != cls) continue;
            float dt = 0.0f;
            ck(c, cudaEventElapsedTime(&dt, r.a, r.b), "cudaEventElapsedTime");
            n++;
            t += dt;
            b += r.bytes;
            f += r.flops;
        }
        if (launches) *launches = n;
        if (ms) *ms = t;
        if (bytes) *bytes = b;
        if (flops) *flops = f;
    });
}

const char *lq_kernel_class_name(int cls)
{
    static const char *names[K_COUNT] = {"hop_k1_f64", "hop_k1_f32", "hop_k2_f64", "hop_k2_f32", "hop_other",
                                         "clover", "layout", "dot_f64", "dot_f32", "axpy_f64", "axpy_f32",
                                         "norm", "reduce_finish", "copy", "hop_k1_df64", "hop_k2_df64",
                                         "dot_df64", "axpy_df64", "clover_field", "force", "sap",
                                         "hop_k1_bf16", "hop_k2_bf16"};
    return (cls >= 0 && cls < K_COUNT) ? names[cls] : "";
}

lq_status lq_counters(lq_ctx *c, long long *launches, double *bytes)
{
    if (!c) return LQ_ERR_ARG;
    if (launches) *launches = c->ctr.launches;
    if (bytes) *bytes = c->ctr.bytes;
    return LQ_OK;
}

}  // extern "C"
