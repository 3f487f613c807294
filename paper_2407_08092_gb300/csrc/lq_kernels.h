// Host-side launchers of the library's kernels (internal; not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "lq_internal.cuh"

namespace lq {

// Internal precisions: native FP64, FP32, double-float (df64: FP64-accurate
// arithmetic on the FP32 units, stored as float pairs in the FP64 layouts), and
// BF16 storage of spinors and links with FP32 arithmetic and FP32 clover.
enum Prec { P64 = 0, P32 = 1, PDF = 2, P16 = 3 };

// Kernel classes for the per-class device timing (mirrors lq_kernel_class of
// the public header).
enum KClass {
    K_HOP_K1_F64 = 0, K_HOP_K1_F32, K_HOP_K2_F64, K_HOP_K2_F32, K_HOP_OTHER, K_CLOVER, K_LAYOUT,
    K_DOT_F64, K_DOT_F32, K_AXPY_F64, K_AXPY_F32, K_NORM, K_FINISH, K_COPY,
    K_HOP_K1_DF, K_HOP_K2_DF, K_DOT_DF, K_AXPY_DF, K_CLOVER_FIELD, K_FORCE, K_SAP, K_HOP_K1_BF16,
    K_HOP_K2_BF16, K_COUNT
};

// Optional CUDA-event timing of every launch (enabled by lq_profile).
struct Prof {
    bool on = false;
    struct Rec {
        int cls;
        cudaEvent_t a, b;
        double bytes, flops;
    };
    std::vector<cudaEvent_t> pool;
    size_t next = 0;
    std::vector<Rec> recs;
    cudaEvent_t get();
};

// Execution context of a launcher: geometry, stream, counters of launches and
// algorithmic bytes, and the optional profiler.
struct Exec {
    Geom g;
    cudaStream_t st;
    Counters *ctr;
    Prof *prof;
};

// Accounts one launch: records a start event at construction and an end
// event, the launch count, the algorithmic bytes and the algorithmic flops
// (FP64-equivalent for df64 kernels) at destruction.  Kernel launches count
// toward `launches`; memsets (K_COPY without `kernel_`) do not.
struct Launch {
    const Exec &e;
    int cls;
    double bytes, flops;
    cudaEvent_t a = nullptr;
    bool kernel;   // a kernel of the library (counted in `launches`)
    Launch(const Exec &e_, int cls_, double bytes_, double flops_ = 0.0, bool kernel_ = false)
        : e(e_), cls(cls_), bytes(bytes_), flops(flops_), kernel(kernel_ || cls_ != K_COPY)
    {
        if (e.prof && e.prof->on) {
            a = e.prof->get();
            cudaEventRecord(a, e.st);
        }
    }
    ~Launch()
    {
        if (kernel) e.ctr->launches++;
        e.ctr->bytes += bytes;
        if (a) {
            cudaEvent_t b = e.prof->get();
            cudaEventRecord(b, e.st);
            e.prof->recs.push_back({cls, a, b, bytes, flops});
        }
    }
};

// Bytes of one internal per-parity spinor field in a precision.
inline size_t spinor_bytes(const Geom &g, int prec)
{
    return (size_t)24 * g.stride * (prec == P32 ? 4 : prec == P16 ? 2 : 8);
}

// ---- layout (layout.cu) ----------------------------------------------------
// natural complex-double gauge field -> per-parity internal link copies (the
// FP64 ones only when U64 is non-null)
void import_links(const Exec &e, const void *U_nat, void *U64[2], void *U32[2], void *Udf[2]);
// out = hi + lo for n df64 complex slots (FP64 copies rounded from df64 ones)
void df64_to_f64(const Exec &e, const void *in, void *out, long long n);
// BF16 12-real links of one parity from the FP32 ones
void links_to_bf16(const Exec &e, const void *U32, void *U16);
// BF16 fields (bf16.cu): conversions (one side BF16), natural half spinors,
// gamma5 and axpby; the generic launchers below dispatch here for P16
void bf16_convert(const Exec &e, int from, const void *in, int to, void *out);
void bf16_import_half(const Exec &e, const void *nat, void *f);
void bf16_export_half(const Exec &e, const void *f, void *nat);
void bf16_gamma5(const Exec &e, const void *in, void *out);
void bf16_axpby(const Exec &e, double ar, double ai, const void *x, double br, double bi, void *y, int nfields);
// natural half spinor [Vh][12] c128 <-> internal field of one parity
void import_half(const Exec &e, int prec, const void *nat, void *f);
void export_half(const Exec &e, int prec, const void *f, void *nat);
// natural full spinor [V][12] c128 <-> internal even and odd fields
void import_full(const Exec &e, int prec, const void *nat, void *fe, void *fo);
void export_full(const Exec &e, int prec, const void *fe, const void *fo, void *nat);
// precision conversion between internal fields
void convert(const Exec &e, int from, const void *in, int to, void *out);
// out = g5 in (negates spins 2 and 3); in == out allowed
void gamma5(const Exec &e, int prec, const void *in, void *out);

// ---- clover (clover.cu) ----------------------------------------------------
// C(x) of every site from the internal df64 links: packed blocks per parity in
// df64 and, rounded, FP32; Fscratch, Rscratch: device scratch of 6 * 9 * V * 8
// bytes each (the six field strengths and the half-clover sums of the passes)
void clover_build(const Exec &e, const void *Udf[2], double csw, double m0, void *Cdf[2], void *C32[2],
                  void *Fscratch, void *Rscratch);
// inverse of the blocks of one parity by LDL^+ in df64, written in df64 and
// FP32; *flag += failures
void clover_invert(const Exec &e, const void *Cdf, void *Cidf, void *Ci32, int *flag);
// FP64 copy of one parity's df64 blocks (both 6x6 blocks), rounded
void clover_to_f64(const Exec &e, const void *Cdf, void *C64);
// natural export: out[V][2][6][6] c128 from FP64 packed blocks (null parity pointer -> zeros)
void clover_export(const Exec &e, const void *Ce, const void *Co, void *out);

// ---- SAP block solves (sap.cu) ----------------------------------------------
// One launch solves every block of one colour (FP32): for each block (origin
// in lattice coordinates), odd-even Minimal Residual on the block operator
// with m steps against the residual r, then x += e on the block's sites.
struct SapLaunch {
    int b[4];                 // block extents: even, dividing the lattice, b0 b1 b2 b3 <= 256
    const int4 *origin;       // device: first site of each block of the colour
    int count;                // blocks of the colour
    const void *U[2];         // FP32 links by parity, lattice order
    const void *Ub[2];        // FP32 links by parity, block-major order (sap_block_major)
    const void *Ce;           // FP32 C of the even sites, block-major order
    const void *Ci;           // FP32 C^{-1} of the odd sites, block-major order
    const void *rin[2];       // FP32 residual of the blocks before the face update (rin[1] null: zero)
    const void *eface[2];     // FP32 last correction of the other colour (null: none yet)
    void *rout_e;             // FP32 out: the blocks' even residual after the solve
    void *eout[2];            // FP32 out: the blocks' correction
    void *x[2];               // FP32 solution by parity (x += e)
    void *ro;                 // FP32 scratch field for the odd residual
    int m;
};
void sap_blocks(const Exec &e, const SapLaunch &s);
// Block-major copy of a parity-`parity` FP32 field of `rows` float4 rows (the
// links: 12, a clover field: 18) for the blocks with extents b: the blocks in
// lexicographic order of their block coordinates, each block's sites in its
// local checkerboard order.  dst has the size and row stride of src.
void sap_block_major(const Exec &e, const int b[4], int parity, int rows, const void *src, void *dst);

// ---- fermion force (force.cu) ----------------------------------------------
// X, Y: internal df64 full fields (even, odd).  Gam: device scratch of
// 6 * 9 * V * 8 bytes.  G: natural c128 [V][4][3][3], G = coef grad_U Re(Y^+ D X).
void force_insertion(const Exec &e, const void *X[2], const void *Y[2], double csw, void *Gam);
void force_links(const Exec &e, const void *Udf[2], const void *X[2], const void *Y[2], const void *Gam,
                 double coef, void *G);
// out = g5 in on natural full spinors (in == out allowed)
void gamma5_nat(const Exec &e, const void *in, void *out);

// ---- hopping term (dslash.cu) ----------------------------------------------
// Modes of the fused hopping kernel; acc = sum of the eight hops into x (the
// hopping term H of the operator) read from the opposite-parity field `in`.
enum HopMode {
    HOP_K1 = 0,     // out = Cinv (-1/2 acc)               t_o = D_oo^{-1} D_oe x_e
    HOP_K2 = 1,     // out = C in2 + 1/2 acc               y_e = D_ee x_e - D_eo t_o
    HOP_RICH = 2,   // out = in2 + w (b - (C in2 + 1/2 acc))   Richardson sweep on D_S
    HOP_FULL = 3,   // out = C in2 - 1/2 acc               D on one parity
    HOP_PREP = 4,   // out = in2 + 1/2 acc                 b_e - D_eo t_o
    HOP_RECON = 5,  // out = Cinv (in2 + 1/2 acc)          D_oo^{-1} (b_o - D_oe x_e)
    // the full system's residual after a solve (FP64 and df64 only):
    HOP_RES = 6,        // out = b - (C in2 - 1/2 acc)               r_e = b_e - D_ee x_e - D_eo x_o
    HOP_RECON_RES = 7   // u = in2 + 1/2 acc: out = Cinv u,          x_o = D_oo^{-1} (b_o - D_oe x_e)
                        //                    out2 = u - clov2 out   r_o = b_o - D_oe x_e - D_oo x_o
};
struct HopCall {
    int mode;
    int prec;
    int pout;              // parity of the output sites
    const void *in;        // opposite-parity field (the hops' source)
    const void *in2;       // same-parity field (mode dependent)
    const void *b;         // HOP_RICH right-hand side
    void *out;
    const void *U[2];      // link copies of both parities (this precision)
    const void *clov;      // C or C^{-1} of the output parity (this precision)
    const void *clov2 = nullptr;   // HOP_RECON_RES: C of the output parity
    void *out2 = nullptr;          // HOP_RECON_RES: the output parity's residual
    double omega;          // HOP_RICH weight
    int nrhs = 1;          // right-hand sides: in, in2, b, out are nrhs consecutive fields
};
void hop(const Exec &e, const HopCall &c);

// One member lattice of a batched solve over lattices of different sizes: its
// geometry, FP32 links and clover, and where its right-hand sides' fields sit
// in a multi-field (nrhs consecutive fields of fs vectors from `off`).
struct LatDesc {
    Geom g;
    const float4 *U[2];      // 12-real FP32 links of both parities
    const float4 *clov[2];   // clov[1]: C^{-1} of the odd sites (K1); clov[0]: C of the even sites (K2)
    long long off;           // float4 vectors
    long long fs;            // float4 vectors per field (6 * stride)
    int nrhs;
};
// threads per block of the hopping kernels
constexpr int kHopBlock = 128;
// resident blocks per SM of the batched hopping kernel with rpt (1 or 2)
// right-hand sides per thread, or of the staged form (rpt 0) with spt sites
// per tile (for a persistent grid)
int hop_group_resident(int rpt, int spt);
// One work-table entry of the batched hopping launch: lattice, site block (of
// blockDim.x sites) and first right-hand side (of rpt * blockDim.y, rpt
// right-hand sides per thread sharing each link load).  rpt 0 selects the staged
// form: one entry per (lattice, site block of spt = 32 or 64 sites), whose links
// and clover blocks are staged in shared memory and applied to every
// right-hand side of the lattice (first right-hand side 0).
// A persistent grid of `grid` blocks of (spt, kHopBlock / spt) threads
// walks the table; mode HOP_K1 (odd output) or HOP_K2 (even output), FP32.
void hop_group(const Exec &e, int mode, const LatDesc *desc, const int4 *tiles, int ntiles, int grid, int spt,
               int rpt, const void *in, const void *in2, void *out, double bytes, double flops);
// FP32 hopping-launch byte and flop counts of `sites` output sites with nrhs
// right-hand sides sharing links and clover
double hop_bytes(int mode, int prec, int nrhs, double sites);
double hop_flops(int mode, double site_rhs);
// out = C in (site-diagonal apply of packed blocks of one parity)
void clover_mul(const Exec &e, int prec, const void *clov, const void *in, void *out);

// ---- BLAS-1 and reductions (blas.cu) ----------------------------------------
// All vectors are internal fields of one parity (or n_vec of them spaced by
// spinor_bytes apart).  Complex scalars are (re, im) pairs.
void zero(const Exec &e, int prec, void *x);
void copy(const Exec &e, int prec, const void *x, void *y);
// y = x for `bytes` (a multiple of 16) of device memory, by a kernel
void copy_bytes(const Exec &e, const void *x, void *y, size_t bytes);
// Small host <-> device transfers by kernels (see blas.cu): put_values copies
// n host doubles (passed as kernel arguments, kSmallVals per launch) to device
// memory; get_values / get_ints copy n device values into pinned host memory
// given by its device-mapped address.  The host reads them after a stream sync.
constexpr int kSmallVals = 64;
void put_values(const Exec &e, const double *h, int n, double *d);
void get_values(const Exec &e, const double *d, int n, double *h_mapped);
void get_ints(const Exec &e, const int *d, int n, int *h_mapped);
// y = a x + b y  (complex a, b; host scalars)
void axpby(const Exec &e, int prec, double ar, double ai, const void *x, double br, double bi,
           void *y, int nfields = 1);
// Reduction scratch: per-block partials and the finished values, in device
// memory owned by the context.  Slot i holds a complex value at [2i, 2i+1].
struct RedScratch {
    double *partial;   // [blocks][2 * maxv]
    double *out;       // [2 * maxv]
    int blocks;
    int maxv;
    unsigned *ticket = nullptr;   // zero between launches: the finishing block count of multi_axpy_finish
};
// y = y - sum_j c_j v_j (sign = -1) or y + sum_j c_j v_j (sign = +1), c in DEVICE
// memory (complex doubles), v_j = V + j * spinor_bytes; with r non-null also the
// partials of ||y_new||^2 into slot `slot`
void multi_axpy(const Exec &e, int prec, const void *V, int nv, const double *c_dev, int sign,
                void *y, const RedScratch *r, int slot);
// FP32 pair of the Arnoldi step on the unnormalised basis, with no separate
// reduction launches: multi_dot_finish writes scale_j * (v_j, w) for j < nv to
// r.out slots 0 .. nv-1 (the last block of each launch sums the partials in a
// fixed order); multi_axpy_finish then forms y = y + sign * sum_j r.out_j v_j and
// writes ||y_new||^2 to r.out slot nrm_slot (summed the same way by its last block)
void multi_dot_finish(const Exec &e, const void *V, int nv, const void *w, const RedScratch &r, const double *scale);
void multi_axpy_finish(const Exec &e, const void *V, int nv, const RedScratch &r, int sign, void *y, int nrm_slot);
// partials of (v_j, w) = sum conj(v_j) w for j < nv into slots slot0 + j
void multi_dot(const Exec &e, int prec, const void *V, int nv, const void *w, const RedScratch &r,
               int slot0);
// ||w||^2 into slot `slot` (real part)
void norm2(const Exec &e, int prec, const void *w, const RedScratch &r, int slot);
// sum the per-block partials of slots [first, first + count) into r.out; with
// `scale` (device, one real per slot, indexed from slot `first`) each complex
// result j is multiplied by scale[j]
void reduce_finish(const Exec &e, const RedScratch &r, int first, int count, const double *scale = nullptr);
// norm of a natural c128 field of n sites (used by lq_norm2)
void nat_norm2(const Exec &e, const void *v, long long n_sites, const RedScratch &r, int slot);
int reduction_blocks(const Geom &g);

// ---- batched right-hand sides (batch.cu) -------------------------------------
// Reduction scratch of a batch: partial[N][blocks][pitch], out[N][pitch]
// (doubles; complex slot i at [2i, 2i+1] of a right-hand side's row).
struct BatchRed {
    double *partial;
    double *out;
    int blocks;
    int pitch;
};
// Device-side Givens state of the batched GMRES: N right-hand sides, cycle m.
struct KState {
    int N, m;
    double2 *H;       // [N][m][m+1] Hessenberg columns (rotated in place)
    double *cs;       // [N][m]
    double2 *sn;      // [N][m]
    double2 *g;       // [N][m+1]
    double2 *y;       // [N][m] least-squares solution
    int *active;      // [N] cycle continues for this right-hand side
    int *kused;       // [N] Arnoldi steps taken this cycle
    int *nanflag;     // NaN/Inf seen
    double *scale;    // [N] normaliser of the newest basis vector (0 when inactive)
    double *est;      // [N] residual estimate |g_{k+1}|
    double *target;   // [N] absolute residual target of the cycle
};
// The systems of a batch inside one buffer (a multi-field): system r's field
// is vectors [off_r, off_r + len_r) (16-byte vectors); seg holds {off, len} per
// system in device memory, or is null for the uniform layout off_r = r * n,
// len_r = n.  blocks: grid of the non-reducing kernels per system; sites: the
// systems' sites of one parity in total (byte accounting).
struct Segs {
    const longlong2 *seg = nullptr;
    long long n = 0;
    int blocks = 1;
    double sites = 0.0;
};
// FP32 batched BLAS; basis vector j of system r at V + j * vjs + off_r
void bdot(const Exec &e, const Segs &S, const void *V, long long vjs, int nv, const void *w, int N, BatchRed &br,
          int slot0);
void baxpy(const Exec &e, const Segs &S, const void *V, long long vjs, int nv, const double *c, int cstride,
           int sign, void *y, int N, BatchRed *br, int slot);
void bnorm(const Exec &e, int prec, const Segs &S, const void *w, int N, BatchRed &br, int slot);   // P32 or PDF
void bfinish(const Exec &e, BatchRed &br, int N, int first, int count);
void bscale(const Exec &e, const Segs &S, const void *x, const double *s, void *y, int N);
void bxmy(const Exec &e, const Segs &S, const void *x, void *y, int N);   // y = x - y
void ks_init(const Exec &e, const KState &k, const double *nrm2, int nstride);
void ks_step(const Exec &e, const KState &k, int step, int passes, const double *dots, int dstride);
void ks_solve(const Exec &e, const KState &k);
int batch_blocks(long long maxlen, int N);   // reduction blocks per system

}  // namespace lq
