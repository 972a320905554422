// Internal interfaces between the slrf translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace slrf {

// Launch bookkeeping: every kernel launch of the library goes through a Ctx,
// which counts launches per class and, when profiling, brackets each launch
// with a pair of CUDA events on the launch stream.
struct Ctx {
    cudaStream_t stream = nullptr;
    int sm_count = 152;
    bool profile = false;
    uint32_t profile_mask = ~0u;  // classes timed when profile is set
    bool rec = false;             // the current launch is being timed
    int64_t launches[SLRF_NKERNEL_CLASSES] = {};
    double bytes[SLRF_NKERNEL_CLASSES] = {};
    double flops[SLRF_NKERNEL_CLASSES] = {};
    struct EvPair { cudaEvent_t a, b; int kc; };
    std::vector<EvPair> pool;     // all events ever created (reused)
    size_t used = 0;              // pairs recorded since reset
    int cur_kc = -1;

    void reset_counters();
    // Call around each launch.
    void before(int kc, double bytes_, double flops_);
    void after();
    // Sum event times per class (synchronises the stream).
    void harvest(double ms_out[SLRF_NKERNEL_CLASSES]);
    void destroy();
};

// Pole data passed by value to kernels.
template <typename T> struct PoleSet {
    int N;
    T re[SLRF_MAX_POLES];
    T im[SLRF_MAX_POLES];
};

// Device pencil.
struct DevPencil {
    int n = 0;
    int64_t nnz = 0;
    int32_t *rowptr = nullptr, *col = nullptr;
    double *a = nullptr, *b = nullptr;      // FP64 values
    float2 *ab32 = nullptr;                 // interleaved (a, b), FP32
    double2 *ab64 = nullptr;                // interleaved (a, b), FP64
    double *diag_a = nullptr, *diag_b = nullptr;
    // row-group form of the shifted SpMM (rg_rows consecutive rows per group,
    // union column list per group, rg_rows (a, b) pairs per union entry)
    int rg_rows = 1, rg_ngroups = 0;
    int64_t rg_nnz = 0;
    int32_t *rg_ptr = nullptr, *rg_col = nullptr;
    float2 *rg_ab32 = nullptr;
    double2 *rg_ab64 = nullptr;
    // staged form of the FP32 row-group product: per union entry and row the
    // pair as (a, a, b, b) (the operand layout of the packed FP32x2 FMA), the
    // position of each row's own column in its group's union list, and the
    // longest union list
    float4 *rg_ab4 = nullptr;
    uint8_t *rg_dpos = nullptr;
    int rg_emax = 0;
    // shifted product kernel: SPMM_ROWGROUP or SPMM_STAGED, and the staged
    // kernel's row groups per CTA; dev_err receives a device-side wait timeout
    int spmm_kind = 0;
    int spmm_gpb = 0;
    int32_t *dev_err = nullptr;
    // node-block form (3-dof nodes whose mass couples equal dofs only, as the
    // consistent mass of vector Lagrange elements does): per row group (node)
    // the neighbour nodes, and per neighbour the 3 x 3 stiffness block and
    // the 3 mass weights, packed as 3 float4 (a00 a01 a02 a10 | a11 a12 a20
    // a21 | a22 b0 b1 b2)
    int32_t *nb_ptr = nullptr, *nb_node = nullptr;
    float4 *nb_coef = nullptr;
    // SELL-C-sigma form (FP32): rows permuted by length within windows of
    // sigma rows, chunks of C rows padded to their longest row, entries
    // slot-major within a chunk (entry k of the chunk's row r at
    // sell_cptr[chunk] + k C + r); per permuted row its original index and
    // length
    int sell_c = 0, sell_sigma = 0, sell_nchunks = 0;
    int64_t sell_slots = 0;
    int32_t *sell_cptr = nullptr, *sell_col = nullptr, *sell_perm = nullptr, *sell_rlen = nullptr;
    float2 *sell_ab = nullptr;
};
enum { SPMM_ROWGROUP = 1, SPMM_STAGED = 2, SPMM_NODEBLOCK = 3, SPMM_SELL = 4 };
// Dynamic shared memory of the staged kernel for this pencil (0: the staged
// kernel cannot run it: no row groups, or a union list too long).
size_t spmm_staged_smem(const DevPencil &A);

// ---------------------------------------------------------------- krylov.cu
// Column-block layout of the Krylov state: complex n x W, W = N * Lp, row
// stride W, pole j in columns [j*Lp, j*Lp + Lp), Lp even.
struct KrylovDims {
    int n, N, Lp, m;       // m <= Lp live columns per pole
    double frac = 1.0;     // active fraction of the W columns (byte accounting)
    int W() const { return N * Lp; }
};

// Per-column scalars of the Krylov solve (device arrays of length W).
template <typename T> struct KrylovScalars {
    cplx<T> *alpha, *rho, *beta, *ua;   // ua = 2 * coef_jc * alpha_jc
    double *bnorm2, *rnorm2;
    int32_t *flag;                       // 1 active, 0 converged, 2 breakdown, 3 maxit, 4 skipped
    int32_t *iters;
    cplx<double> *coef;                  // coef_jc = w_j * d_jc (d = 1 in the plain filter)
    T *part;                             // [gy][W][4] partial sums
    int32_t *active_count;               // 1 int
};

template <typename T>
struct KrylovBuffers {
    cplx<T> *P, *Q, *R;                  // n x W each
    cplx<T> *dinv;                       // n x N Jacobi inverse diagonal
    T *Uacc;                             // n x Lp accumulation of the filter output
    cplx<T> *Z = nullptr;                // n x W preconditioned residual (multigrid); nullptr: Jacobi
    const cplx<T> *mgd = nullptr;        // multigrid: finest damped Jacobi diagonal (n x N); the
                                         // update then also writes y = mgd r into Q (Q is dead there)
    KrylovScalars<T> s;
    int gy;                              // row groups of the kernels
};

int krylov_row_groups(const Ctx &ctx, const KrylovDims &d, int prec_fp32);

template <typename T>
void krylov_dinv(Ctx &ctx, const DevPencil &A, const PoleSet<T> &ps, int precond, cplx<T> *dinv);

// r = p = z = M^{-1} b from a real block shared by all poles (rhs: n x m, ld)
// or, if rhs_c != nullptr, a complex block per pole (layout of the state).
template <typename T>
void krylov_init(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb, const double *rhs, int64_t ldr,
                 const cplx<double> *rhs_c);
template <typename T>
void krylov_reduce_init(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb);
template <typename T>
void krylov_spmm(Ctx &ctx, const KrylovDims &d, const DevPencil &A, const cplx<T> *sig_dev,
                 const cplx<T> *P, cplx<T> *Q, const int32_t *flag, T *part, int gy);
template <typename T>
void krylov_reduce_alpha(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb);
template <typename T>
void krylov_update(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb);
template <typename T>
void krylov_reduce_beta(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb, double tol2, int maxit);
// p = z + beta p (z = Z, or M^{-1} r with the Jacobi diagonal); init: p = z
template <typename T>
void krylov_direction(Ctx &ctx, const KrylovDims &d, KrylovBuffers<T> &kb, int init = 0);
void krylov_count_active(Ctx &ctx, int W, const int32_t *flag, int32_t *count);
// mu[c] = sum over row groups of part slot 0/1 -> complex (for the SpMM step API)
template <typename T>
void krylov_reduce_mu(Ctx &ctx, const KrylovDims &d, const T *part, int gy, cplx<T> *mu);

// ---------------------------------------------------------------- bicgstab.cu
// Extra state of block BiCGStab (n x W each) and its per-column omega.
template <typename T> struct BcgBuffers {
    cplx<T> *Rh, *V, *Y, *Z, *Tt;        // shadow residual, A y, M^{-1} p, M^{-1} s, A z
    cplx<T> *omega, *ua2;                // omega and 2 coef omega (W each)
};
// r^ = r, p = r, partials for rho = (r^, r) and |b|^2 (then krylov_reduce_init)
template <typename T> void bicgstab_init(Ctx &, const KrylovDims &, KrylovBuffers<T> &, BcgBuffers<T> &);
template <typename T>
void bicgstab_precond_jacobi(Ctx &, const KrylovDims &, KrylovBuffers<T> &, const cplx<T> *In, cplx<T> *Out);
// alpha = rho / (r^, v)
template <typename T> void bicgstab_alpha(Ctx &, const KrylovDims &, KrylovBuffers<T> &, BcgBuffers<T> &);
// s = r - alpha v (in R); jacobi: also Z = D s
template <typename T> void bicgstab_s(Ctx &, const KrylovDims &, KrylovBuffers<T> &, BcgBuffers<T> &, bool jacobi);
// omega = (t, s) / (t, t)
template <typename T> void bicgstab_omega(Ctx &, const KrylovDims &, KrylovBuffers<T> &, BcgBuffers<T> &);
// U += filter terms of alpha y + omega z; r = s - omega t; partials of (r^, r), |r|^2
template <typename T> void bicgstab_update(Ctx &, const KrylovDims &, KrylovBuffers<T> &, BcgBuffers<T> &);
// p = r + (beta alpha / omega)(p - omega v) (after krylov_reduce_beta)
template <typename T> void bicgstab_direction(Ctx &, const KrylovDims &, KrylovBuffers<T> &, BcgBuffers<T> &);

// ---------------------------------------------------------------- mg.cu
// Device view of the multigrid hierarchy for one Krylov precision T.  Level 0
// is the caller's pencil (row-group form); levels 1.. are Galerkin pencils in
// CSR (R = 1).  Transfers P_l (n_l x n_{l+1}) and R_l = P_l^T are stored as
// CSR with real values.  r/z/t are the per-solve level blocks (levels >= 1),
// dinv the damped Jacobi inverse n_l x N.
constexpr int MG_MAX_LEVELS = 16;
template <typename T> struct MgLevel {
    int n = 0, R = 1, ngroups = 0;
    int64_t nnz_union = 0;
    const int32_t *gptr = nullptr, *gcol = nullptr;
    const cplx<T> *ab = nullptr;              // R (a, b) pairs per union entry
    const double *diag_a = nullptr, *diag_b = nullptr;
    int64_t p_nnz = 0, r_nnz = 0;
    const int32_t *pptr = nullptr, *pcol = nullptr, *rptr = nullptr, *rcol = nullptr;
    const T *pval = nullptr, *rval = nullptr;
    cplx<T> *r = nullptr, *z = nullptr, *t = nullptr, *dinv = nullptr;
    double rho = 1.0;                         // spectral radius of D^{-1} A on this level
    // level 0 with a next level: F = (M - D^{-1}) P in pair form (F_a, F_b),
    // F_a = A P - (rho/omega) diag(a) P, F_b = B P - (rho/omega) diag(b) P,
    // by fine row groups (the R rows of the level's groups, union coarse
    // columns, R pairs per entry: "up") and by coarse rows (F^T: "down").
    // f_q holds the unfolded FP64 pieces (A P, B P) and (a_ii P, b_ii P) per
    // stored pair, up entries first; f_ab the folded pairs in that order.
    int64_t fu_nnz = 0, fd_nnz = 0;
    const int32_t *fu_ptr = nullptr, *fu_col = nullptr, *fd_ptr = nullptr, *fd_col = nullptr;
    const double2 *f_q = nullptr;
    cplx<T> *f_ab = nullptr;
};
template <typename T> struct MgSolve {
    int nlev = 0, nc = 0;
    int nu = 1, gamma = 1;        // coarse-level sweeps per side, coarse visits per level
    double omega = 4.0 / 3.0;     // Jacobi damping on level l: omega / rho_l
    MgLevel<T> lv[MG_MAX_LEVELS];
    const T *V = nullptr;         // coarsest eigenvectors, nc x nc row-major
    cplx<T> *cinv = nullptr;      // nc x N: 1 / (lambda_k - sigma_j)
    // FP32 cycles may instead stop at a level solved by its dense shifted
    // inverses (N matrices nc x nc, formed per solve by coarse_inverse);
    // cublas is the handle's cuBLAS handle for their GEMMs
    const cplx<T> *Minv = nullptr;
    void *cublas = nullptr;
    // tensor-core application of those inverses (coarse_tc.cu): the split
    // panels of the inverses, the per-apply workspace and the mapped word
    // that records a bounded wait that gave up; Mpan == nullptr: cuBLAS
    const void *Mpan = nullptr;
    void *ct_work = nullptr;
    int32_t *ct_err = nullptr;
};
template <typename T>
void mg_dinv(Ctx &ctx, MgSolve<T> &mg, const PoleSet<T> &ps);

// ---------------------------------------------------------------- coarse.cu
// Dense shifted inverses of one level: Minv_j = (A - sigma_j B)^{-1}, j < N,
// n x n each (symmetric), from the level's CSR pairs, by blocked Gauss-Jordan
// (GEMMs through cuBLAS handle `cublas`); work: coarse_inverse_work_bytes.
size_t coarse_inverse_work_bytes(int n, int N);
int coarse_inverse(Ctx &ctx, void *cublas, int n, const PoleSet<float> &ps, const int32_t *ptr, const int32_t *col,
                   const float2 *ab, float2 *Minv, void *work);
// Z_j = Minv_j R_j for every pole's columns of the level block (layout of the state)
int coarse_inverse_apply(Ctx &ctx, void *cublas, const KrylovDims &d, int n, const float2 *Minv, const float2 *R,
                         float2 *Z);

// ---------------------------------------------------------------- coarse_tc.cu
// The same application on the tcgen05 tensor cores (three-way bf16 split of
// both operands, six part products into one FP32 accumulator): the panels of
// the inverses are formed once per solve (coarse_tc_panels, coarse_tc_panel_bytes
// bytes), each application splits the level block into work
// (coarse_tc_work_bytes) and writes Z; Lp <= 256 (coarse_tc_fits).
bool coarse_tc_fits(int Lp);
size_t coarse_tc_panel_bytes(int n, int N);
size_t coarse_tc_work_bytes(int n, int N, int Lp);
void coarse_tc_panels(Ctx &ctx, int n, int N, const float2 *Minv, void *Mpan);
void coarse_tc_apply(Ctx &ctx, const KrylovDims &d, int n, const void *Mpan, const float2 *R, float2 *Z, void *work,
                     int32_t *err);
// Z0 = cycle(R0) for all active columns of the state; part receives the
// partial sums r^T z (slots 0, 1).  Y0 = D R0 with the finest level's
// damped Jacobi diagonal (mg.lv[0].dinv), if the caller has it (the COCG
// update forms it); otherwise it is formed into T0, an n x W scratch block
// (also the scratch of a single-level hierarchy).
template <typename T>
void mg_apply(Ctx &ctx, const KrylovDims &d, MgSolve<T> &mg, const cplx<T> *sig, const int32_t *flag, T *part,
              int gy, const cplx<T> *R0, cplx<T> *Z0, cplx<T> *T0, const cplx<T> *Y0 = nullptr);
// part = partial sums r^T z per column (slots 0, 1) of two state blocks
template <typename T>
void mg_rz(Ctx &ctx, const KrylovDims &d, int gy, const cplx<T> *R, const cplx<T> *Z, const int32_t *flag, T *part);

// ---------------------------------------------------------------- ilu.cu
// No-fill incomplete L D L^T of every shifted matrix A - sigma_j B (pencil
// pattern), built per solve by fixed-point sweeps and applied by Jacobi
// sweeps of the two triangular solves.  Pattern arrays are built once per
// handle (lower part by rows and by columns), factor values per solve.
struct IluPattern {
    int n = 0;
    int64_t nnzl = 0;                          // strictly lower entries
    const int32_t *lptr = nullptr, *lcol = nullptr;  // lower part by rows (CSR, sorted columns)
    const int32_t *lrow = nullptr;             // row of each lower entry
    const int32_t *lsrc = nullptr;             // pencil CSR index of each lower entry
    const int32_t *tptr = nullptr, *trow = nullptr;  // lower part by columns (rows of L^T)
    const int32_t *tidx = nullptr;             // lower-entry index of each L^T entry
};
// Host build of the pattern arrays from the pencil's CSR, concatenated in
// the order lptr (n+1), lcol, lrow, lsrc (nnzl each), tptr (n+1), trow, tidx.
std::vector<int32_t> ilu_pattern_host(int n, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci,
                                      int64_t *nnzl);
// Device views of the concatenated arrays.
void ilu_pattern_views(const int32_t *dev, int n, int64_t nnzl, IluPattern &pat);
template <typename T> struct IluFactor {
    int N = 0;
    const cplx<T> *L = nullptr;    // N x nnzl, pole-major
    const cplx<T> *Dinv = nullptr; // n x N, 1 / d
};
size_t ilu_factor_work_bytes(const IluPattern &pat, int N);
// Factor values of all poles (FP64 sweeps; stored as T in `out`, sized
// N * nnzl + n * N complex T, after the FP64 work in `work`).
template <typename T>
void ilu_factor(Ctx &ctx, const DevPencil &A, const IluPattern &pat, const PoleSet<double> &ps, int sweeps,
                void *work, cplx<T> *out, IluFactor<T> &fac);
// Out = P^T D^{-1} P In (tri_sweeps each side) for the active columns;
// F and Ys are n x W scratch blocks; part receives In^T Out partials when
// non-null.
template <typename T>
void ilu_apply(Ctx &ctx, const KrylovDims &d, const IluPattern &pat, const IluFactor<T> &fac, int tri_sweeps,
               int gy, const int32_t *flag, const cplx<T> *In, cplx<T> *Out, cplx<T> *F, cplx<T> *Ys, T *part);

// ---------------------------------------------------------------- dense.cu
// Y = A X and/or Z = B X, FP64, row-major n x m.
void spmm_real(Ctx &ctx, const DevPencil &A, int m, const double *X, int64_t ldx, double *Y,
               int64_t ldy, double *Z, int64_t ldz);
// C = op(A) op(B) (+ beta C), row-major; opA/opB: 0 = N, 1 = T.
// Dimensions: op(A) is M x K, op(B) is K x N.  split > 1 splits K into
// `split` slices whose partial products go to work[split][M][N] and are then
// summed in a fixed order.
void dgemm(Ctx &ctx, int opA, int opB, int M, int N, int K, const double *A, int64_t lda,
           const double *B, int64_t ldb, double beta, double *C, int64_t ldc, int split = 1,
           double *work = nullptr, int kc = KC_TALL_GEMM);
// Choose a split for a Gram of n rows.
int gram_split(const Ctx &ctx, int m, int64_t n);
// Residual of the Ritz pairs: Rout = BX diag(theta) - AX (if Rout != nullptr),
// rho[c] = ||R_c|| / (|theta_c| ||BX_c||), rho_ax[c] = ||R_c|| / ||AX_c||.
void residual(Ctx &ctx, int n, int m, const double *AX, const double *BX, int64_t ld,
              const double *theta, double *Rout, int64_t ldr, double *rho, double *rho_ax,
              double *work);
// U = X diag(phi) + Ucorr(T, ld Lp)  (FP64 out)
template <typename T>
void filter_combine(Ctx &ctx, int n, int m, const double *X, int64_t ldx, const double *phi,
                    const T *Ucorr, int ldc, double *U, int64_t ldu);
void fill_zero(Ctx &ctx, void *p, size_t bytes);
// Copy a strided row-major block (device).
void copy_block(Ctx &ctx, int n, int m, const double *src, int64_t lds, double *dst, int64_t ldd);

// ---------------------------------------------------------------- ozaki.cu
// G = X^T Y (m x m, row-major, ld m) from int8 tensor-core digit products.
size_t ozaki_gram_work_bytes(int64_t n, int m, int sm_count);
// symmetric: X^T Y is known to be symmetric (Y = B X with B symmetric): only
// the tiles on and above the diagonal are computed and mirrored.
// tc_err != nullptr selects the tensor-core (tcgen05, bf16 digits) form; it
// receives a nonzero code if one of that kernel's bounded waits gives up.
void ozaki_gram(Ctx &ctx, int64_t n, int m, const double *X, int64_t ldx, const double *Y, int64_t ldy, double *G,
                void *work, bool symmetric = false, int32_t *tc_err = nullptr);
// C = (A diag(cs)) B, A n x k, B k x m, C n x m (row-major, leading dims),
// cs = nullptr for no column scaling; FP64-accurate from exact digit
// products.  tc_err != nullptr (and k <= 512) selects the tcgen05 form (bf16
// digits, FP32 tensor-memory sums); it receives a nonzero code if one of that
// kernel's bounded waits gives up.  Otherwise int8 mma.sync.
size_t ozaki_tall_work_bytes(int64_t n, int k, int m);
bool ozaki_tall_fits(int k);
void ozaki_tall(Ctx &ctx, int64_t n, int k, int m, const double *A, int64_t lda, const double *cs, const double *B,
                int64_t ldb, double *C, int64_t ldc, void *work, int kc, int32_t *tc_err = nullptr);

// ---------------------------------------------------------------- small.cu
// All m x m matrices row-major, device.  status: device int, set nonzero on
// failure (Cholesky pivot <= 0 or non-finite).
void small_colscale(Ctx &ctx, int m, double *G, double *s);        // s = 1/sqrt(diag G); G = S G S
// G + s I = R^T R (R upper) into R (may alias G); s = 0, or shift_on_fail if
// the unshifted factorisation breaks down (*status = -1 then).
void small_chol_upper(Ctx &ctx, int m, const double *G, double *R, int32_t *status, double shift_on_fail);
void small_triinv_upper(Ctx &ctx, int m, const double *R, double *Rinv);
void small_scale_rows(Ctx &ctx, int m, const double *s, double *T);  // T = diag(s) T
// Symmetric eigensolver: lam ascending, Q eigenvectors (columns).  mode 1:
// FP32 Jacobi followed by FP64 refinement; 0: FP64 Jacobi.
cudaError_t small_syev(Ctx &ctx, int m, const double *S, double *lam, double *Q, double *work, int mode);
size_t small_syev_work_bytes(int m);

// ---------------------------------------------------------------- api.cu
// Upper bound of the device bytes a handle needs for a solve of subspace size
// L with N poles (pencil copies + Krylov state + projection workspace + the
// staging of the host-buffer entry point; mg_coarse > 0: plus the multigrid
// hierarchy and its level blocks, mg_coarse being the coarsest-size target;
// krylov = SLRF_KRYLOV_BICGSTAB: plus its extra blocks).
size_t workspace_estimate(int64_t n, int64_t nnz, int L, int N, int precision, int sm_count, int mg_coarse,
                          int krylov);
int handle_device(const slrf_handle *h);

}  // namespace slrf
